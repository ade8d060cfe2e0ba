"""Host logic of the float32 path: thresholds and bin table (no GPU).

The float32 paths bin a squared separation d2~ computed in float32 and must
reach the bin of the binary64 definition (bins [e_k, e_{k+1}) tested on
squares, Sec. 2.2).  The library's host code builds thresholds lo_k <= E2_k <=
hi_k from an error bound and a byte table over cells of float32 values.  These
tests check them against things other than the builder itself:

* every table entry against the threshold definition, on float32 values at
  every cell boundary, next to every threshold and at random (the cell of a
  value is computed here exactly from the stated cell rule);
* the decision the thresholds take for float32 distances computed here with
  the float32 operations the kernels use (exact emulation, one rounding per
  operation, fused multiply-adds rounded once) against the binary64
  definition, on pairs placed within a few float32 ulps of every edge.
"""
import zlib
from fractions import Fraction

import numpy as np
import pytest

import paper_1911_08275_gb300 as cf

F32 = np.float32
FLAGGED = 0xFF  # the entry of a cell that the thresholds must settle


def log_edges(lo, hi, nb):
    return 10.0 ** np.linspace(np.log10(lo), np.log10(hi), nb + 1)


CASES = {
    # name: (edges, ncomp, coord_max, shift_max)
    "xi_log_0.1_25_periodic420": (log_edges(0.1, 25.0, 20), 3, 420.0, 420.0),
    "xi_log_1e-3_30_wide": (log_edges(1e-3, 30.0, 40), 3, 200.0, 200.0),
    "xi_linear_from_zero_open": (np.linspace(0.0, 50.0, 11), 3, 1000.0, 0.0),
    "xi_64_bins": (log_edges(0.01, 100.0, 64), 3, 1000.0, 1000.0),
    "xi_tiny_edges": (np.array([1e-4, 2e-4, 1e-3, 0.5]), 3, 10.0, 10.0),
    "rp_log_0.1_25_periodic420": (log_edges(0.1, 25.0, 14), 2, 420.0, 420.0),
    # narrow ranges: cells on float bit patterns are the finer shape there
    "xi_narrow_10_12": (np.linspace(10.0, 12.0, 9), 3, 200.0, 200.0),
    "rp_narrow_10_12": (np.linspace(10.0, 12.0, 5), 2, 200.0, 200.0),
    "rp_10_12_open": (np.linspace(10.0, 12.0, 5), 2, 200.0, 0.0),
    "xi_narrow_5_5.5": (np.array([5.0, 5.25, 5.5]), 3, 100.0, 100.0),
}


def tables(name):
    e, ncomp, M, Ls = CASES[name]
    T, tab, info = cf.debug_bin_tables(e, ncomp=ncomp, coord_max=M, shift_max=Ls)
    return e, ncomp, M, Ls, T, tab, info


def cell_of(v, info, lut_n):
    """Cell of float32 values v >= 0 (NaN allowed) under the stated cell rule."""
    v = np.asarray(v, dtype=F32)
    last = lut_n - 1
    out = np.full(v.shape, last, dtype=np.int64)
    ok = ~np.isnan(v)
    if info["lin"]:
        # float32 x float32 is exact in binary64 (48 significant bits); rint
        # rounds half to even, as the float32 sum with 2^23 does
        q = np.rint(v[ok].astype(np.float64) * np.float64(F32(info["lscale"])))
        out[ok] = np.minimum(q, last).astype(np.int64)
    else:
        b = v[ok].view(np.uint32).astype(np.int64)
        q = ((b >> info["shift"]) - int(info["u0"])) % (1 << 32)
        out[ok] = np.minimum(q, last)
    return out


def sample_values(T, tab, info, seed):
    rng = np.random.default_rng(seed)
    top = float(T[-1])
    vals = [np.array([0.0, 1e-45, 1e-30, top, 2 * top, 4 * top, np.inf, np.nan], dtype=F32)]
    t = T[T > 0].astype(F32)
    for k in range(1, 4):  # next to every threshold
        vals += [np.nextafter(t, F32(np.inf)), np.nextafter(t, F32(0))]
        t = np.nextafter(t, F32(np.inf))
    vals.append(T[T >= 0].astype(F32))
    n = tab.size
    if info["lin"]:  # both sides of every cell boundary (q + 1/2) / lscale
        b = ((np.arange(n) + 0.5) / np.float64(F32(info["lscale"]))).astype(F32)
        for s in (b, np.nextafter(b, F32(0)), np.nextafter(b, F32(np.inf))):
            vals.append(s)
    else:  # first and last bit pattern of every cell
        q = np.arange(n - 1, dtype=np.uint64)
        lo = ((np.uint64(info["u0"]) + q) << np.uint64(info["shift"])).astype(np.uint32)
        hi = (((np.uint64(info["u0"]) + q + np.uint64(1)) << np.uint64(info["shift"])) - np.uint64(1))
        for s in (lo, hi.astype(np.uint32), (lo - np.uint32(1))[lo > 0]):
            vals.append(s.view(F32))
    vals.append(rng.uniform(0.0, 1.2 * top, 200_000).astype(F32))
    vals.append((10.0 ** rng.uniform(-12, np.log10(1.2 * top), 200_000)).astype(F32))
    v = np.concatenate(vals)
    return v[~(v < 0)]


@pytest.mark.parametrize("name", sorted(CASES))
def test_thresholds_bracket_the_squared_edges(name):
    e, ncomp, M, Ls, T, tab, info = tables(name)
    E2 = e * e
    assert T.dtype == F32 and T.size == 2 * e.size
    assert np.all(np.diff(T.astype(np.float64)) >= 0), "thresholds must not decrease"
    lo, hi = T[0::2].astype(np.float64), T[1::2].astype(np.float64)
    assert np.all(lo <= E2) and np.all(E2 <= hi)
    pos = E2 > 0
    assert np.all(lo[pos] < E2[pos]) and np.all(E2[pos] < hi[pos])
    # a band is at least one float32 rounding of E2 wide, and narrow next to
    # the squared edges of size >= 1 (a lo_k of -1 near zero claims nothing)
    assert np.all(hi[pos] > F32(E2[pos]))
    big = E2 >= 1.0
    assert np.all((hi - lo)[big] < 0.01 * E2[big])


@pytest.mark.parametrize("name", sorted(CASES))
def test_wider_error_bounds_only_shrink_what_float32_decides(name):
    # every value that the thresholds of larger coordinate and shift bounds
    # settle in float32 (an even count) is settled the same way by the
    # original thresholds: more error can only send more values to binary64
    e, ncomp, M, Ls, T, tab, info = tables(name)
    T2, _, _ = cf.debug_bin_tables(e, ncomp=ncomp, coord_max=4 * M + 1, shift_max=4 * Ls + 1)
    assert np.all(T2[1::2] >= T[1::2]) and np.any(T2[1::2] > T[1::2])
    v = sample_values(np.concatenate([T, T2]), tab, info, seed=7)
    v = v[~np.isnan(v)].astype(np.float64)
    c = np.searchsorted(T.astype(np.float64), v, side="right")
    c2 = np.searchsorted(T2.astype(np.float64), v, side="right")
    even2 = (c2 & 1) == 0
    assert np.array_equal(c[even2], c2[even2])
    assert np.sum(c & 1) <= np.sum(c2 & 1)


@pytest.mark.parametrize("name", sorted(CASES))
def test_every_table_entry_agrees_with_the_thresholds(name):
    e, ncomp, M, Ls, T, tab, info = tables(name)
    nb = e.size - 1
    assert np.all((tab <= nb) | (tab == FLAGGED))
    assert tab[-1] == nb, "out-of-range values must land on the not-counted entry"
    v = sample_values(T, tab, info, seed=zlib.crc32(name.encode()))
    cell = cell_of(v, info, tab.size)
    ent = tab[cell].astype(np.int64)
    c = np.searchsorted(T.astype(np.float64), v.astype(np.float64), side="right")
    nan = np.isnan(v)
    binned = ent < nb
    # a bin entry: the value is safely inside that bin, outside every band
    assert np.array_equal(c[binned], 2 * ent[binned] + 2), (
        name, v[binned][c[binned] != 2 * ent[binned] + 2][:5])
    # the not-counted entry: below lo_0 or at / above hi_B (or NaN)
    dummy = ent == nb
    assert np.all((c[dummy] == 0) | (c[dummy] == T.size) | nan[dummy])
    # the table settles most values: flagged cells hold a small part of the range
    assert np.mean(tab[:-1] == FLAGGED) < 0.05


@pytest.mark.parametrize("name", sorted(CASES))
def test_both_cell_shapes_are_exercised(name):
    # the builder keeps the shape whose flagged cells hold less pair mass:
    # cells linear in d2 for edges from near zero to Rmax (their width is
    # Rmax^2 / 16383 everywhere), cells on float bit patterns for a narrow
    # range of edges (their width is relative, fine there)
    _, _, _, _, _, _, info = tables(name)
    assert info["lin"] == (0 if "narrow" in name else 1)


def bad(**kw):
    args = dict(edges=[1.0, 2.0], ncomp=3, coord_max=10.0, shift_max=0.0)
    args.update(kw)
    e = args.pop("edges")
    with pytest.raises(cf.CfError) as ei:
        cf.debug_bin_tables(e, **args)
    return ei.value


@pytest.mark.parametrize("kw,msg", [
    (dict(edges=[1.0]), "2 to 65"),
    (dict(edges=list(np.arange(1.0, 67.0))), "2 to 65"),
    (dict(edges=[2.0, 1.0]), "increasing"),
    (dict(edges=[-1.0, 1.0]), ">= 0"),
    (dict(edges=[0.0, np.inf]), "finite"),
    (dict(ncomp=4), "ncomp"),
    (dict(coord_max=-1.0), "bounds"),
    (dict(shift_max=np.nan), "bounds"),
])
def test_bad_arguments_rejected(kw, msg):
    err = bad(**kw)
    assert err.status == cf.CF_EINVAL and msg in str(err)


# ---- the decision on float32 distances computed as the kernels do

def f32_round(fr):
    """Round a Fraction to the nearest float32 (ties to even), exactly."""
    if fr == 0:
        return F32(0.0)
    sign = -1 if fr < 0 else 1
    a = abs(fr)
    ex = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** ex > a:
        ex -= 1
    ex = max(ex, -126)  # subnormal spacing below 2^-126
    m = round(a / Fraction(2) ** (ex - 23))  # round half to even
    return F32(sign * float(m * Fraction(2) ** (ex - 23)))


def fr(v):
    return Fraction(float(v))


def kernel_d2(xi, xj, S, ncomp, periodic, origin):
    """float32 squared separation as the float32 kernels compute it: frame
    coordinates fl32(X) (periodic) or fl32(X - origin) (open box), primary
    shifted by fl32(S), dx = fl32(x_j - x^_i), then (ncomp 3)
    fma(dz, dz, fma(dy, dy, dx * dx)) or (ncomp 2) fma(dy, dy, dx * dx)."""
    d = []
    for a in range(3):
        if periodic:
            ti, tj = F32(xi[a]), F32(xj[a])
        else:
            ti, tj = F32(xi[a] - origin[a]), F32(xj[a] - origin[a])
        hi_ = f32_round(fr(ti) - fr(F32(S[a])))
        d.append(f32_round(fr(tj) - fr(hi_)))
    p = f32_round(fr(d[0]) * fr(d[0]))
    q = f32_round(fr(d[1]) * fr(d[1]) + fr(p))
    if ncomp == 2:
        return q
    return f32_round(fr(d[2]) * fr(d[2]) + fr(q))


def canonical_d2(xi, xj, box, ncomp):
    """The binary64 definition: dx = x_j - x_i, minimum image, then
    (dx^2 + dy^2) + dz^2 with one rounding per operation."""
    d = []
    for a in range(3):
        dx = np.float64(xj[a]) - np.float64(xi[a])
        if box is not None:
            if dx > box / 2:
                dx = dx - box
            elif dx < -box / 2:
                dx = dx + box
        d.append(dx)
    s = d[0] * d[0] + d[1] * d[1]
    return s if ncomp == 2 else s + d[2] * d[2]


def near_edge_pairs(e, box, rng, per_edge):
    pts = []
    for ek in e[e > 0]:
        for _ in range(per_edge):
            xi = rng.uniform(0.0, box, 3)
            u = rng.normal(size=3)
            u /= np.linalg.norm(u)
            # relative offsets from 1e-8 (inside every band) to 1e-3 (outside)
            r = ek * (1.0 + rng.choice([-1.0, 1.0]) * 10.0 ** rng.uniform(-8, -3))
            xj = xi + r * u
            pts.append((xi, xj))
    return pts


@pytest.mark.parametrize("ncomp", [3, 2])
@pytest.mark.parametrize("periodic", [True, False])
def test_threshold_decision_matches_binary64_near_every_edge(ncomp, periodic):
    rng = np.random.default_rng(11 + ncomp + 2 * periodic)
    box = 420.0
    e = log_edges(0.1, 25.0, 20 if ncomp == 3 else 14)
    origin = np.zeros(3)
    pairs = near_edge_pairs(e, box, rng, per_edge=60)
    if periodic:
        pairs = [(xi, np.mod(xj, box)) for xi, xj in pairs]
        M, Ls = box, box
    else:
        allx = np.array([p for pr in pairs for p in pr])
        origin = allx.min(axis=0)
        M, Ls = float((allx.max(axis=0) - origin).max()), 0.0
    T, _, _ = cf.debug_bin_tables(e, ncomp=ncomp, coord_max=M, shift_max=Ls)
    Td = T.astype(np.float64)
    E2 = e * e
    nb = e.size - 1
    decided = 0
    for xi, xj in pairs:
        S = np.zeros(3)
        if periodic:  # the kernels' image shift: dx = x_j - (x_i - S)
            dx = xj - xi
            S = np.where(dx > box / 2, -box, np.where(dx < -box / 2, box, 0.0))
        d2f = float(kernel_d2(xi, xj, S, ncomp, periodic, origin))
        d2 = canonical_d2(xi, xj, box if periodic else None, ncomp)
        c = int(np.searchsorted(Td, d2f, side="right"))
        if c & 1:
            continue  # inside a band: settled in binary64 by the kernels
        decided += 1
        k32 = (c - 2) // 2 if 2 <= c <= 2 * nb else -1
        k64 = int(np.searchsorted(E2, d2, side="right")) - 1
        k64 = k64 if 0 <= k64 < nb else -1
        assert k32 == k64, (xi, xj, d2f, d2)
    assert decided > len(pairs) // 10


# ---- the pi-bin decision of the float32 DD(rp, pi) path

def pi_decision(dzf, pscale, pband, npi):
    """The kernels' float32 pi bin of one pair from its float32 dz~: the bin m,
    -1 (not counted) or None (re-checked in binary64).  t' = fma(|dz~|, pscale,
    -1/2) rounded once; m = round(t') half to even (t' + 1.5 * 2^23 in float32);
    g = fl32(pband - |t' - m|) and a set sign bit sends the pair to binary64."""
    t = f32_round(fr(abs(dzf)) * fr(pscale) - Fraction(1, 2))
    m = round(fr(t))
    g = f32_round(fr(pband) - abs(fr(t) - m))
    if g < 0:
        return None
    return m if m < npi else -1


def canonical_pi_bin(zi, zj, box, pimax, npi):
    dz = np.float64(zj) - np.float64(zi)
    if box is not None:
        if dz > box / 2:
            dz = dz - box
        elif dz < -box / 2:
            dz = dz + box
    p = abs(dz)
    if not p < pimax:
        return -1
    P = [(pimax * m) / npi for m in range(npi)]
    return max(m for m in range(npi) if P[m] <= p)


@pytest.mark.parametrize("periodic,pimax,npi", [(True, 40.0, 40), (False, 10.5, 7)])
def test_pi_decision_matches_binary64_near_every_pi_edge(periodic, pimax, npi):
    rng = np.random.default_rng(5 + npi)
    box = 420.0
    edges = [(pimax * m) / npi for m in range(1, npi)] + [pimax]
    zs = []
    for pe in edges:
        for _ in range(40):
            zi = rng.uniform(0.0, box)
            dz = pe * (1.0 + rng.choice([-1.0, 1.0]) * 10.0 ** rng.uniform(-8, -3))
            zj = zi + rng.choice([-1.0, 1.0]) * dz
            zs.append((zi, np.mod(zj, box) if periodic else zj))
    if periodic:
        origin, M, Ls = 0.0, box, box
    else:
        allz = np.array(zs).ravel()
        origin = float(allz.min())
        M, Ls = float(allz.max() - origin), 0.0
    pscale, pband = cf.debug_pi_band(pimax, npi, coord_max=M, shift_max=Ls)
    assert pscale == F32(npi / pimax) and 0.0 < pband < 0.5
    decided = 0
    for zi, zj in zs:
        if periodic:
            kz = -box if zj - zi > box / 2 else (box if zj - zi < -box / 2 else 0.0)
            ti, tj = F32(zi), F32(zj)
        else:
            kz = 0.0
            ti, tj = F32(zi - origin), F32(zj - origin)
        zh = f32_round(fr(ti) - fr(F32(kz)))
        dzf = f32_round(fr(tj) - fr(zh))
        m32 = pi_decision(dzf, pscale, pband, npi)
        if m32 is None:
            continue
        decided += 1
        assert m32 == canonical_pi_bin(zi, zj, box if periodic else None, pimax, npi), (zi, zj)
    assert decided > len(zs) // 10


def test_pi_band_arguments():
    with pytest.raises(cf.CfError):
        cf.debug_pi_band(0.0, 10, coord_max=1.0)
    with pytest.raises(cf.CfError):
        cf.debug_pi_band(10.0, 0, coord_max=1.0)
    with pytest.raises(cf.CfError):
        cf.debug_pi_band(10.0, 10, coord_max=-1.0)
    # larger error bounds leave a narrower trusted interval
    _, b1 = cf.debug_pi_band(40.0, 40, coord_max=420.0, shift_max=420.0)
    _, b2 = cf.debug_pi_band(40.0, 40, coord_max=4200.0, shift_max=4200.0)
    assert b2 < b1
