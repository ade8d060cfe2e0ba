"""Estimators on top of the counts (Sec. 1.1): analytic RR, xi, wp, Landy-Szalay.

CPU tests pin the analytic random counts against counted pairs of uniform points
(the oracle), and the estimators against closed forms; the GPU test runs the
whole chain on the library's counts.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1911_08275_gb300 import estimators as est
from paper_1911_08275_gb300 import synth


def _within_noise(counted, expected, nsig=6.0, floor=50.0):
    """Counted ordered pairs of uniform points vs the expectation: each unordered
    pair is counted twice, so the variance is about 2 x expected."""
    m = expected > floor
    z = (counted[m] - expected[m]) / np.sqrt(2.0 * expected[m])
    return np.all(np.abs(z) < nsig), np.max(np.abs(z))


def test_rr_xi_matches_counted_uniform_pairs():
    cat = synth.c1_uniform20k()
    e = synth.log_edges(0.5, 40.0, 12)
    dd = oracle.xi(cat.x, cat.y, cat.z, edges=e, periodic=True, box=synth.BOX)[0].astype(float)
    rr = est.rr_analytic_xi(e, cat.n, synth.BOX)
    ok, worst = _within_noise(dd, rr)
    assert ok, worst
    xi = est.xi_natural(dd, rr)
    assert np.all(np.abs(xi[rr > 1000]) < 0.1)


def test_rr_rppi_matches_counted_uniform_pairs():
    cat = synth.c1_uniform20k()
    e = synth.log_edges(1.0, 40.0, 8)
    dd = oracle.rppi(cat.x, cat.y, cat.z, rp_edges=e, pimax=40.0, npibins=8, periodic=True,
                     box=synth.BOX)[0].astype(float)
    rr = est.rr_analytic_rppi(e, 40.0, 8, cat.n, synth.BOX)
    assert rr.shape == dd.shape == (8, 8)
    ok, worst = _within_noise(dd, rr)
    assert ok, worst


def test_rr_closed_forms():
    # one bin [0, R): all pairs times the sphere's share of the box
    n, box, R = 1000, 100.0, 7.0
    rr = est.rr_analytic_xi([0.0, R], n, box)
    assert rr[0] == pytest.approx(n * (n - 1) * (4.0 / 3.0) * math.pi * R ** 3 / box ** 3, rel=1e-14)
    # cross counts use n1 n2; shells add up to the outer sphere
    e = [0.0, 1.0, 2.5, 7.0]
    assert est.rr_analytic_xi(e, 10, box, n2=30).sum() == pytest.approx(
        10 * 30 * (4.0 / 3.0) * math.pi * 7.0 ** 3 / box ** 3, rel=1e-13)
    # rp-pi: the bins tile the cylinder rp < 7, |dz| < 9
    c = est.rr_analytic_rppi(e, 9.0, 3, n, box)
    assert c.sum() == pytest.approx(n * (n - 1) * math.pi * 49.0 * 18.0 / box ** 3, rel=1e-13)
    with pytest.raises(ValueError):
        est.rr_analytic_xi([0.0, 60.0], n, box)


def test_pi_edges_match_the_counting_convention():
    p = est.pi_edges(37.3, 17)
    assert p[0] == 0.0 and p[-1] == 37.3
    assert all(p[m] == (37.3 * m) / 17 for m in range(17))


def test_wp_closed_forms():
    pimax, npi = 40.0, 20
    xi = np.full((5, npi), 0.25)
    assert np.allclose(est.wp_from_xi(xi, pimax, npi), 2.0 * 0.25 * pimax)
    # xi linear in the bin centre: 2 * sum (a + b pi_m) dpi = 2 (a pimax + b pimax^2 / 2)
    p = est.pi_edges(pimax, npi)
    mid = 0.5 * (p[1:] + p[:-1])
    xi = np.vstack([1.0 + 0.1 * mid, -0.5 + 0.0 * mid])
    assert np.allclose(est.wp_from_xi(xi, pimax, npi),
                       [2.0 * (pimax + 0.1 * pimax ** 2 / 2.0), -pimax])


def test_wp_of_neyman_scott_matches_its_closed_form():
    # Siblings (children of one parent, offsets N(0, sigma^2) per axis) are
    # separated by a Gaussian of sigma * sqrt(2) per axis, so their projected
    # separation falls in the annulus [a, b) with probability
    # P = exp(-a^2 / 4 sigma^2) - exp(-b^2 / 4 sigma^2), and |dz| < pimax almost
    # surely (pimax >> sigma); pairs of different parents are uniform.  With S
    # ordered sibling pairs, xi(rp, pi) = DD / RR - 1 integrates to
    #   E[wp] = S V / (N (N - 1)) * (P / (pi (b^2 - a^2)) - 2 pimax / V).
    npar, lam, sig, box, seed = 5000, 5.0, 2.0, 100.0, 52
    cat = synth.neyman_scott(npar, lam, sig, box, seed)
    cnt = synth.poisson(seed, 3, npar, lam)
    S = float(np.sum(cnt * (cnt - 1.0)))
    N, V = cat.n, box ** 3
    rp_e = synth.log_edges(0.5, 8.0, 8)
    pimax, npi = 20.0, 20
    dd = oracle.rppi(cat.x, cat.y, cat.z, rp_edges=rp_e, pimax=pimax, npibins=npi,
                     periodic=True, box=box)[0].astype(float)
    rr = est.rr_analytic_rppi(rp_e, pimax, npi, N, box)
    wp = est.wp_from_xi(est.xi_natural(dd, rr), pimax, npi)
    a, b = rp_e[:-1], rp_e[1:]
    area = np.pi * (b * b - a * a)
    P = np.exp(-a * a / (4 * sig * sig)) - np.exp(-b * b / (4 * sig * sig))
    want = S * V / (N * (N - 1.0)) * (P / area - 2.0 * pimax / V)
    # scatter of the summed counts: sibling pairs move together within a cluster,
    # background pairs between two clusters (ordered pairs come in twos)
    sib, bg = S * P, N * (N - 1.0) * area * 2.0 * pimax / V
    sd = np.sqrt(2 * sib * (1 + lam) + 2 * bg * (1 + 2 * lam)) * V / (N * (N - 1.0) * area)
    z = (wp - want) / sd
    assert np.all(np.abs(z) < 5.0), z
    # the check has power: a generator with sigma doubled lands several of these
    # (deliberately generous) standard deviations away
    P2 = np.exp(-a * a / (16 * sig * sig)) - np.exp(-b * b / (16 * sig * sig))
    wrong = S * V / (N * (N - 1.0)) * (P2 / area - 2.0 * pimax / V)
    assert np.max(np.abs(wp - wrong) / sd) > 4.0


def test_landy_szalay_identities():
    nd, nr = 100, 1000
    rr = np.array([5000.0, 20000.0, 0.0])
    # counts exactly proportional to their pair totals: no clustering
    dd = rr * (nd * (nd - 1)) / (nr * (nr - 1))
    dr = rr * (nd * nr) / (nr * (nr - 1))
    ls = est.xi_landy_szalay(dd, dr, rr, nd, nr)
    assert np.allclose(ls[:2], 0.0, atol=1e-12) and np.isnan(ls[2])
    # twice the uncorrelated DD, DR unchanged: xi = 1
    assert np.allclose(est.xi_landy_szalay(2.0 * dd, dr, rr, nd, nr)[:2], 1.0)
    # hand example, nd = nr = 2 (n_dd = 2, n_dr = 4, n_rr = 2): fdd = 0.5, fdr = 0.2,
    # frr = 0.1 -> (0.5 - 0.2 - 0.2 + 0.1) / 0.1 = 2
    assert est.xi_landy_szalay([1.0], [0.8], [0.2], 2, 2)[0] == pytest.approx(2.0)


def test_natural_estimator_nan_on_empty_bins():
    xi = est.xi_natural([4.0, 0.0, 3.0], [2.0, 0.0, 0.0])
    assert xi[0] == 1.0 and np.isnan(xi[1]) and np.isnan(xi[2])


@pytest.mark.gpu
def test_xi_and_wp_from_gpu_counts(cuda_device):
    import torch
    import paper_1911_08275_gb300 as cf
    # uniform points: xi ~ 0 within the pair-count noise
    u = synth.c1_uniform20k()
    e = synth.log_edges(0.5, 40.0, 12)
    xyz = [torch.from_numpy(v).cuda() for v in (u.x, u.y, u.z)]
    dd = cf.countpairs_xi(*xyz, e, boxsize=synth.BOX).npairs.astype(float)
    ok, worst = _within_noise(dd, est.rr_analytic_xi(e, u.n, synth.BOX))
    assert ok, worst
    # clustered points (clusters of sigma 2): the estimators of the GPU counts equal
    # those of the oracle's counts (the counts are identical), with a strong
    # small-scale signal
    c = synth.neyman_scott(2000, 20.0, 2.0, 200.0, seed=91)
    xyz = [torch.from_numpy(v).cuda() for v in (c.x, c.y, c.z)]
    dd = cf.countpairs_xi(*xyz, e, boxsize=200.0).npairs.astype(float)
    ref = oracle.xi(c.x, c.y, c.z, edges=e, periodic=True, box=200.0)[0].astype(float)
    xi = est.xi_natural(dd, est.rr_analytic_xi(e, c.n, 200.0))
    assert np.array_equal(xi, est.xi_natural(ref, est.rr_analytic_xi(e, c.n, 200.0)))
    assert xi[0] > 5.0 and xi[0] > xi[5] > xi[-1]
    rp = synth.log_edges(0.5, 20.0, 6)
    ddp = cf.countpairs_rp_pi(*xyz, rp, 30.0, 30, boxsize=200.0).npairs.astype(float)
    refp = oracle.rppi(c.x, c.y, c.z, rp_edges=rp, pimax=30.0, npibins=30, periodic=True,
                       box=200.0)[0].astype(float)
    rrp = est.rr_analytic_rppi(rp, 30.0, 30, c.n, 200.0)
    wp = est.wp_from_xi(est.xi_natural(ddp, rrp), 30.0, 30)
    assert np.array_equal(wp, est.wp_from_xi(est.xi_natural(refp, rrp), 30.0, 30))
    assert wp[0] > 10.0 and wp[0] > wp[-1]
