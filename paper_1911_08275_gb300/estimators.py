"""Correlation-function estimators on top of the pair counts (host-only, numpy).

Sec. 1.1: the correlation function compares the data pair counts N_DD with the
counts N_RR expected for randomly distributed points in the same bins,
xi(r) = N_DD / N_RR - 1 (Eq. "xi"); the projected function is the line-of-sight
integral wp(rp) = 2 * integral_0^pimax xi(rp, pi) dpi.  For a periodic cube the
random counts are analytic (the expected number of pairs of uniform points in
each bin), so only the auto-correlation DD has to be counted; for other
geometries the DR and RR terms are counted as well, and the counts combine in
the Landy-Szalay form below.

All counts here are ORDERED pairs, as the library returns them: an
auto-correlation of N points counts N (N - 1) pairs in total, a cross-correlation
N1 N2.  Bins are [e_k, e_{k+1}) in r (or rp) and [P_m, P_{m+1}) in pi = |dz| with
P_m = pimax * m / npibins.
"""
from __future__ import annotations

import math

import numpy as np


def _pairs(n1: int, n2: int | None) -> float:
    """Ordered pairs of an auto (n2 None) or cross correlation."""
    return float(n1) * (float(n1) - 1.0) if n2 is None else float(n1) * float(n2)


def rr_analytic_xi(edges, n1: int, box: float, n2: int | None = None) -> np.ndarray:
    """Expected ordered pair counts per r bin for uniform points in a periodic cube.

    The pairs of uniform points are spread evenly over the box volume V = box^3,
    so the count in the spherical shell e_k <= r < e_{k+1} is
    pairs / V * (4/3) pi (e_{k+1}^3 - e_k^3).  Valid while e_B < box / 2 (one
    image per pair), which the counting routines require anyway.
    """
    e = np.asarray(edges, dtype=np.float64)
    if e.ndim != 1 or e.size < 2 or np.any(np.diff(e) <= 0) or e[0] < 0:
        raise ValueError("edges must be increasing, non-negative, at least two")
    if not e[-1] < 0.5 * box:
        raise ValueError("largest edge must be below half the box")
    shell = (4.0 / 3.0) * math.pi * (e[1:] ** 3 - e[:-1] ** 3)
    return _pairs(n1, n2) / float(box) ** 3 * shell


def pi_edges(pimax: float, npibins: int) -> np.ndarray:
    """Line-of-sight edges P_m = pimax * m / npibins (P_npibins = pimax)."""
    p = np.array([pimax * m / npibins for m in range(npibins + 1)], dtype=np.float64)
    p[-1] = pimax
    return p


def rr_analytic_rppi(rp_edges, pimax: float, npibins: int, n1: int, box: float,
                     n2: int | None = None) -> np.ndarray:
    """Expected ordered pair counts per (rp, pi) bin for uniform points in a periodic cube.

    The bin rp_k <= rp < rp_{k+1}, P_m <= |dz| < P_{m+1} is a cylindrical shell of
    volume pi (rp_{k+1}^2 - rp_k^2) * 2 (P_{m+1} - P_m) (both signs of dz).
    Returns shape [n_rp_bins, npibins], rp-major like the counts.
    """
    e = np.asarray(rp_edges, dtype=np.float64)
    if e.ndim != 1 or e.size < 2 or np.any(np.diff(e) <= 0) or e[0] < 0:
        raise ValueError("rp edges must be increasing, non-negative, at least two")
    if not (e[-1] < 0.5 * box and pimax < 0.5 * box):
        raise ValueError("largest rp edge and pimax must be below half the box")
    p = pi_edges(pimax, npibins)
    area = math.pi * (e[1:] ** 2 - e[:-1] ** 2)
    return _pairs(n1, n2) / float(box) ** 3 * np.outer(area, 2.0 * np.diff(p))


def xi_natural(dd, rr) -> np.ndarray:
    """xi = N_DD / N_RR - 1 (Sec. 1.1, Eq. "xi"), bin by bin; NaN where N_RR = 0.

    dd and rr must count pairs of catalogues of the same sizes (for example the
    counts of the library and rr_analytic_* for the same N).
    """
    dd = np.asarray(dd, dtype=np.float64)
    rr = np.asarray(rr, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(rr > 0, dd / np.where(rr > 0, rr, 1.0) - 1.0, np.nan)


def wp_from_xi(xi_rppi, pimax: float, npibins: int) -> np.ndarray:
    """wp(rp) = 2 sum_m xi(rp, pi_m) (P_{m+1} - P_m): the line-of-sight integral of
    Sec. 1.1 as a sum over the pi bins (xi constant inside a bin)."""
    x = np.asarray(xi_rppi, dtype=np.float64)
    if x.ndim != 2 or x.shape[1] != npibins:
        raise ValueError("xi(rp, pi) must have shape [n_rp_bins, npibins]")
    return 2.0 * x @ np.diff(pi_edges(pimax, npibins))


def xi_landy_szalay(dd, dr, rr, nd: int, nr: int, rd=None) -> np.ndarray:
    """Landy-Szalay estimator from counted DD, DR and RR (surveys, where N_RR and
    N_DR cannot be written down and are counted, Sec. 1.1):

        xi = (DD / n_dd - DR / n_dr - RD / n_dr + RR / n_rr) / (RR / n_rr)

    with the ordered-pair normalisations n_dd = nd (nd - 1), n_dr = nd nr,
    n_rr = nr (nr - 1).  RD defaults to DR (a cross count is symmetric).  NaN
    where RR = 0.
    """
    dd = np.asarray(dd, dtype=np.float64)
    dr = np.asarray(dr, dtype=np.float64)
    rr = np.asarray(rr, dtype=np.float64)
    rd = dr if rd is None else np.asarray(rd, dtype=np.float64)
    fdd = dd / _pairs(nd, None)
    fdr = dr / _pairs(nd, nr)
    frd = rd / _pairs(nd, nr)
    frr = rr / _pairs(nr, None)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(frr > 0, (fdd - fdr - frd + frr) / np.where(frr > 0, frr, 1.0), np.nan)
