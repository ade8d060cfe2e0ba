"""Pins for the CPU oracle: facts that do not come from the oracle itself.

* hand-enumerated tiny inputs with dyadic coordinates (every binary64
  operation exact), pairs exactly on squared edges, across the periodic
  boundary, duplicates, N in {0, 1, 2};
* SciPy's KD-tree pair counter (an independent implementation of the same
  counting problem, periodic and not, weighted and not) and SciPy's pdist for
  the 2-D rp-pi histogram;
* closed forms: total pair count when Rmax spans the box, and the expected
  uniform-box counts N(N-1)/V * (4/3)pi(r_hi^3 - r_lo^3) (Sec. 1.1, analytic
  randoms for a periodic cube) within Poisson scatter;
* invariants: auto == cross(D, D) when e_0 > 0, permutation and periodic
  translation invariance, unit weights give wsum == npairs;
* the clustered input recipe: Neyman-Scott counts equal uniform background
  pairs plus sibling pairs whose separation follows the Maxwell law of a 3-D
  Gaussian with sigma * sqrt(2) per axis, within a conservative scatter.
"""
import numpy as np
import pytest
from scipy.spatial import cKDTree
from scipy.spatial.distance import pdist

import oracle
from paper_1911_08275_gb300 import synth


@pytest.fixture
def orc():
    """The oracle under test (the mutation test passes modified builds)."""
    return oracle.Oracle(oracle._load())


def pts(*rows):
    a = np.array(rows, dtype=np.float64)
    return a[:, 0].copy(), a[:, 1].copy(), a[:, 2].copy()


# ---------------------------------------------------------------- hand-enumerated

def test_pair_exactly_on_squared_edge_goes_to_upper_bin(orc):
    # (0,0,0)-(3,4,0): r^2 = 25 = 5^2 exactly -> bin [5, 6), never [1, 5).
    x, y, z = pts((0, 0, 0), (3, 4, 0))
    n, _, _ = orc.xi(x, y, z, edges=[1.0, 5.0, 6.0], periodic=False)
    assert n.tolist() == [0, 2]
    n, _, _ = orc.xi(x, y, z, edges=[1.0, 5.0], periodic=False)
    assert n.tolist() == [0]          # r = Rmax is excluded
    n, _, _ = orc.xi(x, y, z, edges=[5.0, 6.0], periodic=False)
    assert n.tolist() == [2]          # r = Rmin is included


def test_three_points_on_a_line_auto_and_cross(orc):
    # separations 1, 2, 3 -> one unordered pair per bin.
    x, y, z = pts((0, 0, 0), (1, 0, 0), (3, 0, 0))
    e = [0.5, 1.5, 2.5, 3.5]
    n, _, _ = orc.xi(x, y, z, edges=e, periodic=False)
    assert n.tolist() == [2, 2, 2]
    n, _, _ = orc.xi(x[:1], y[:1], z[:1], x2=x[1:], y2=y[1:], z2=z[1:], edges=e,
                        autocorr=False, periodic=False)
    assert n.tolist() == [1, 0, 1]    # d(p0,p1) = 1, d(p0,p2) = 3


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_periodic_minimum_image(orc, axis):
    a = [0.0, 0.0, 0.0]
    b = [0.0, 0.0, 0.0]
    a[axis], b[axis] = 0.5, 9.5        # raw difference 9, image difference -1
    x, y, z = pts(a, b)
    e = [0.5, 1.5, 8.5, 9.5]
    n, _, _ = orc.xi(x, y, z, edges=e, periodic=True, box=10.0)
    assert n.tolist() == [2, 0, 0]
    n, _, _ = orc.xi(x, y, z, edges=e, periodic=False)
    assert n.tolist() == [0, 0, 2]


def test_periodic_wrap_is_strict_at_half_box(orc):
    # raw difference exactly L/2 = 5 is not wrapped (wrap only when |d| > L/2)
    x, y, z = pts((0, 0, 0), (5, 0, 0))
    n, _, _ = orc.xi(x, y, z, edges=[4.5, 5.5], periodic=True, box=10.0)
    assert n.tolist() == [2]


def test_diagonal_wrap_all_axes(orc):
    # (0.25,0.25,0.25)-(9.75,9.75,9.75) in box 10: image offsets (-0.5)^3 -> r^2 = 0.75
    x, y, z = pts((0.25, 0.25, 0.25), (9.75, 9.75, 9.75))
    n, _, _ = orc.xi(x, y, z, edges=[0.5, 0.8660254037844386, 1.0], periodic=True, box=10.0)
    # 0.8660254037844386^2 rounds to 0.7499999999999999 < 0.75 -> upper bin
    assert n.tolist() == [0, 2]


def test_duplicates_and_zero_edge(orc):
    x, y, z = pts((1, 1, 1), (1, 1, 1))
    n, _, _ = orc.xi(x, y, z, edges=[0.0, 1.0], periodic=False)
    assert n.tolist() == [2]          # coincident distinct points count iff e_0 = 0
    n, _, _ = orc.xi(x, y, z, edges=[0.125, 1.0], periodic=False)
    assert n.tolist() == [0]
    # cross-correlation of a point with itself: the (i, i) pair has r = 0
    n, _, _ = orc.xi(x[:1], y[:1], z[:1], x2=x[:1], y2=y[:1], z2=z[:1], edges=[0.0, 1.0],
                        autocorr=False, periodic=False)
    assert n.tolist() == [1]


@pytest.mark.parametrize("n", [0, 1])
def test_empty_and_single(orc, n):
    x, y, z = (np.zeros(n),) * 3
    cnt, _, _ = orc.xi(x, y, z, edges=[0.0, 1.0, 2.0], periodic=True, box=10.0)
    assert cnt.tolist() == [0, 0]


def test_rppi_hand_enumerated(orc):
    # rp^2 = 3^2 + 4^2 = 25, pi = |dz| = 2.5
    x, y, z = pts((0, 0, 0), (3, 4, 2.5))
    n, _, _ = orc.rppi(x, y, z, rp_edges=[1.0, 5.0, 6.0], pimax=4.0, npibins=4, periodic=False)
    want = np.zeros((2, 4), dtype=np.uint64)
    want[1, 2] = 2                     # rp in [5,6), pi in [2,3)
    assert np.array_equal(n, want)
    n, _, _ = orc.rppi(x, y, z, rp_edges=[1.0, 5.0, 6.0], pimax=2.5, npibins=5, periodic=False)
    assert int(n.sum()) == 0           # pi = pimax is excluded
    # periodic line of sight: dz raw 9.5 -> image -0.5 in box 10
    x, y, z = pts((0, 0, 0.25), (3, 4, 9.75))
    n, _, _ = orc.rppi(x, y, z, rp_edges=[1.0, 5.0, 6.0], pimax=4.0, npibins=4, periodic=True,
                          box=10.0)
    assert n[1, 0] == 2 and int(n.sum()) == 2


def test_weights_and_ravg_hand_enumerated(orc):
    x, y, z = pts((0, 0, 0), (3, 4, 0), (0, 0, 12))
    w = np.array([0.5, 2.0, 4.0])
    # pairs: (0,1) r=5 w=1; (0,2) r=12 w=2; (1,2) r=13 w=8
    n, ws, rs = orc.xi(x, y, z, w1=w, edges=[4.0, 6.0, 12.5, 14.0], periodic=False, want_r=True)
    assert n.tolist() == [2, 2, 2]
    assert ws.tolist() == [2.0, 4.0, 16.0]
    assert rs.tolist() == [10.0, 48.0, 208.0]
    n, ws, rs = orc.xi(x, y, z, edges=[4.0, 6.0, 12.5, 14.0], periodic=False, want_r=True)
    assert rs.tolist() == [10.0, 24.0, 26.0] and ws is None


def test_rppi_weights_and_ravg_hand_enumerated(orc):
    # Sec. 1.1 Code 1's weight per pair with the rp-pi separations of Eq.
    # "separations": the mean separation of an (rp, pi) slot is the mean rp,
    # not r.  Dyadic inputs, so every sum below is exact in binary64.
    x, y, z = pts((0, 0, 0), (3, 4, 2.5), (6, 8, 1))
    w = np.array([0.5, 2.0, 4.0])
    # pairs: (0,1) rp=5 pi=2.5 w=1; (1,2) rp=5 pi=1.5 w=8; (0,2) rp=10 pi=1 w=2
    rp, kw = [4.0, 6.0, 11.0], dict(pimax=4.0, npibins=4, periodic=False, want_r=True)
    n, ws, rs = orc.rppi(x, y, z, w1=w, rp_edges=rp, **kw)
    want_n = np.zeros((2, 4), dtype=np.uint64)
    want_w, want_r = np.zeros((2, 4)), np.zeros((2, 4))
    want_n[0, 2], want_w[0, 2], want_r[0, 2] = 2, 2.0, 10.0     # 2 x (w 1, rp 5)
    want_n[0, 1], want_w[0, 1], want_r[0, 1] = 2, 16.0, 80.0    # 2 x (w 8, rp 5 w 8)
    want_n[1, 1], want_w[1, 1], want_r[1, 1] = 2, 4.0, 40.0     # 2 x (w 2, rp 10 w 2)
    assert np.array_equal(n, want_n)
    assert ws.tolist() == want_w.tolist() and rs.tolist() == want_r.tolist()
    n, ws, rs = orc.rppi(x, y, z, rp_edges=rp, **kw)               # unweighted: sum of rp
    assert ws is None and rs[0, 2] == 10.0 and rs[0, 1] == 10.0 and rs[1, 1] == 20.0
    # cross: point 0 against points 1, 2, one ordered pair each
    n, ws, rs = orc.rppi(x[:1], y[:1], z[:1], w1=w[:1], x2=x[1:], y2=y[1:], z2=z[1:], w2=w[1:],
                         rp_edges=rp, autocorr=False, **kw)
    assert n[0, 2] == 1 and n[1, 1] == 1 and int(n.sum()) == 2
    assert ws[0, 2] == 1.0 and ws[1, 1] == 2.0 and rs[0, 2] == 5.0 and rs[1, 1] == 20.0


# ---------------------------------------------------------------- library pins (SciPy)

def _kd_hist(a_xyz, b_xyz, edges, box, w=None):
    ta = cKDTree(np.column_stack(a_xyz), boxsize=box)
    tb = cKDTree(np.column_stack(b_xyz), boxsize=box)
    cum = ta.count_neighbors(tb, np.asarray(edges), weights=w, cumulative=True)
    return np.diff(np.asarray(cum, dtype=np.float64))


@pytest.mark.parametrize("periodic", [True, False])
def test_xi_auto_matches_kdtree(orc, periodic):
    c = synth.uniform_box(3000, 100.0, seed=11)
    e = synth.log_edges(0.5, 30.0, 12)
    n, _, _ = orc.xi(c.x, c.y, c.z, edges=e, periodic=periodic, box=100.0)
    ref = _kd_hist((c.x, c.y, c.z), (c.x, c.y, c.z), e, 100.0 if periodic else None)
    # KD-tree counts ordered pairs including (i, i) at r = 0 < e_0: none in bins.
    assert np.array_equal(n.astype(np.float64), ref)


def test_xi_clustered_auto_matches_kdtree(orc):
    c = synth.neyman_scott(200, 20.0, 2.0, 100.0, seed=12)
    e = synth.log_edges(0.1, 20.0, 20)
    n, _, _ = orc.xi(c.x, c.y, c.z, edges=e, periodic=True, box=100.0)
    ref = _kd_hist((c.x, c.y, c.z), (c.x, c.y, c.z), e, 100.0)
    assert np.array_equal(n.astype(np.float64), ref)


def test_xi_cross_weighted_matches_kdtree(orc):
    a = synth.uniform_box(1500, 60.0, seed=13)
    b = synth.uniform_box(2500, 60.0, seed=14)
    wa = synth.uniform_weights(a.n, 0.5, 1.5, seed=15)
    wb = synth.uniform_weights(b.n, 0.5, 1.5, seed=16)
    e = synth.log_edges(0.3, 25.0, 10)
    for periodic in (True, False):
        box = 60.0 if periodic else None
        n, ws, _ = orc.xi(a.x, a.y, a.z, w1=wa, x2=b.x, y2=b.y, z2=b.z, w2=wb, edges=e,
                             autocorr=False, periodic=periodic, box=60.0)
        ref_n = _kd_hist((a.x, a.y, a.z), (b.x, b.y, b.z), e, box)
        ref_w = _kd_hist((a.x, a.y, a.z), (b.x, b.y, b.z), e, box, w=(wa, wb))
        assert np.array_equal(n.astype(np.float64), ref_n)
        np.testing.assert_allclose(ws, ref_w, rtol=1e-11, atol=0)


def test_rppi_matches_pdist_histogram2d(orc):
    c = synth.uniform_box(2500, 50.0, seed=17)
    rp_e = synth.log_edges(0.5, 12.0, 7)
    pimax, npi = 10.0, 10
    n, _, _ = orc.rppi(c.x, c.y, c.z, rp_edges=rp_e, pimax=pimax, npibins=npi, periodic=False)
    rp = pdist(np.column_stack([c.x, c.y]))
    pi = pdist(c.z[:, None])
    h, _, _ = np.histogram2d(rp, pi, bins=[rp_e, np.arange(npi + 1) * (pimax / npi)])
    assert np.array_equal(n.astype(np.float64), 2 * h)
    # the paper's 1-D wp count: rp bin with the pi < pimax filter
    keep = pi < pimax
    h1, _ = np.histogram(rp[keep], bins=rp_e)
    assert np.array_equal(n.sum(axis=1).astype(np.float64), 2 * h1)


def test_rppi_periodic_projected_matches_2d_kdtree(orc):
    # With pimax > L/2 every minimum-image |dz| passes, so the pi-summed
    # counts are the 2-D periodic rp counts.
    c = synth.uniform_box(3000, 40.0, seed=18)
    rp_e = synth.log_edges(0.25, 15.0, 9)
    n, _, _ = orc.rppi(c.x, c.y, c.z, rp_edges=rp_e, pimax=20.5, npibins=3, periodic=True,
                          box=40.0)
    t = cKDTree(np.column_stack([c.x, c.y]), boxsize=40.0)
    ref = np.diff(t.count_neighbors(t, rp_e).astype(np.float64))
    assert np.array_equal(n.sum(axis=1).astype(np.float64), ref)


# ---------------------------------------------------------------- closed forms

def test_total_count_when_rmax_spans_box(orc):
    c = synth.uniform_box(700, 10.0, seed=19)
    d = synth.uniform_box(300, 10.0, seed=20)
    e = [0.0, 1.0, 5.0, 18.0]          # 18 > sqrt(3) * 10
    n, _, _ = orc.xi(c.x, c.y, c.z, edges=e, periodic=False)
    assert int(n.sum()) == 700 * 699
    n, _, _ = orc.xi(c.x, c.y, c.z, x2=d.x, y2=d.y, z2=d.z, edges=e, autocorr=False,
                        periodic=False)
    assert int(n.sum()) == 700 * 300
    n, _, _ = orc.rppi(c.x, c.y, c.z, rp_edges=[0.0, 15.0], pimax=10.5, npibins=7,
                          periodic=False)
    assert int(n.sum()) == 700 * 699


def test_uniform_xi_closed_form_c1(orc):
    c = synth.c1_uniform20k()
    e = synth.log_edges(0.1, 25.0, 20)
    n, _, _ = orc.xi(c.x, c.y, c.z, edges=e, periodic=True, box=synth.BOX)
    N, V = c.n, synth.BOX ** 3
    mean = N * (N - 1) / V * (4.0 / 3.0) * np.pi * (e[1:] ** 3 - e[:-1] ** 3)
    # ordered counts come in pairs: variance ~ 2 * mean
    z = (n - mean) / np.sqrt(2.0 * mean + 1e-300)
    big = mean > 50
    assert np.all(np.abs(z[big]) < 5.0), z
    assert int(n[~big].sum()) <= 2 * (mean[~big].sum() + 5 * np.sqrt(mean[~big].sum()) + 4)


def test_neyman_scott_counts_background_plus_siblings(orc):
    # Children of one parent are offset by N(0, sigma^2) per axis, so a sibling
    # pair's separation is Maxwell distributed with scale sigma * sqrt(2); two
    # points of different parents are independent and uniform in the periodic
    # box.  Given the children counts c_p (S = sum c_p (c_p - 1) ordered sibling
    # pairs): E[DD_k] = (N (N - 1) - S) V_k / V + S P_k.
    from scipy.special import erf
    npar, lam, sig, box, seed = 2000, 5.0, 2.0, 100.0, 50
    c = synth.neyman_scott(npar, lam, sig, box, seed)
    cnt = synth.poisson(seed, 3, npar, lam)
    S = float(np.sum(cnt * (cnt - 1.0)))
    e = synth.log_edges(0.5, 12.0, 12)
    n, _, _ = orc.xi(c.x, c.y, c.z, edges=e, periodic=True, box=box)
    N, V = c.n, box ** 3
    s = sig * np.sqrt(2.0)

    def maxwell_cdf(r):
        return erf(r / (s * np.sqrt(2.0))) - np.sqrt(2.0 / np.pi) * (r / s) * np.exp(-r * r / (2 * s * s))

    vk = (4.0 / 3.0) * np.pi * (e[1:] ** 3 - e[:-1] ** 3)
    bg = (N * (N - 1) - S) * vk / V
    sib = S * (maxwell_cdf(e[1:]) - maxwell_cdf(e[:-1]))
    # ordered pairs come in twos; clusters correlate both terms (a cluster pair
    # or a cluster moves up to ~lam pairs together): a generous scatter
    sd = np.sqrt(2 * bg * (1 + 2 * lam) + 2 * sib * (1 + lam))
    z = (n - (bg + sib)) / sd
    assert np.all(np.abs(z) < 5.0), z
    # the clustering is visible: between 1 and 2.5 units the counts exceed the
    # background by more than the scatter allowed above
    mid = (e[:-1] >= 1.0) & (e[1:] <= 2.5)
    assert mid.sum() == 3 and np.all((n[mid] - bg[mid]) / sd[mid] > 5.0)


def test_uniform_rppi_closed_form(orc):
    c = synth.uniform_box(20000, 200.0, seed=21)
    rp_e = synth.log_edges(0.5, 20.0, 6)
    pimax, npi = 20.0, 5
    n, _, _ = orc.rppi(c.x, c.y, c.z, rp_edges=rp_e, pimax=pimax, npibins=npi, periodic=True,
                          box=200.0)
    N, V = c.n, 200.0 ** 3
    P = np.arange(npi + 1) * (pimax / npi)
    mean = N * (N - 1) / V * np.pi * np.outer(rp_e[1:] ** 2 - rp_e[:-1] ** 2, 2 * np.diff(P))
    z = (n - mean) / np.sqrt(2.0 * mean)
    assert np.all(np.abs(z) < 5.5), z


# ---------------------------------------------------------------- invariants

def test_auto_equals_cross_with_itself_when_e0_positive(orc):
    c = synth.neyman_scott(100, 20.0, 1.5, 50.0, seed=22)
    e = synth.log_edges(0.05, 10.0, 15)
    a, _, _ = orc.xi(c.x, c.y, c.z, edges=e, periodic=True, box=50.0)
    b, _, _ = orc.xi(c.x, c.y, c.z, x2=c.x, y2=c.y, z2=c.z, edges=e, autocorr=False,
                        periodic=True, box=50.0)
    assert np.array_equal(a, b)
    a, _, _ = orc.rppi(c.x, c.y, c.z, rp_edges=e, pimax=12.0, npibins=12, periodic=True,
                          box=50.0)
    b, _, _ = orc.rppi(c.x, c.y, c.z, x2=c.x, y2=c.y, z2=c.z, rp_edges=e, pimax=12.0,
                          npibins=12, autocorr=False, periodic=True, box=50.0)
    assert np.array_equal(a, b)


def test_permutation_invariance(orc):
    c = synth.neyman_scott(80, 20.0, 2.0, 40.0, seed=23)
    e = synth.log_edges(0.1, 15.0, 12)
    p = np.random.default_rng(0).permutation(c.n)
    a, _, _ = orc.xi(c.x, c.y, c.z, edges=e, periodic=True, box=40.0)
    b, _, _ = orc.xi(c.x[p], c.y[p], c.z[p], edges=e, periodic=True, box=40.0)
    assert np.array_equal(a, b)


def test_periodic_translation_invariance_dyadic(orc):
    # dyadic coordinates on a 1/64 lattice in box 64: every operation is exact,
    # so translating by a lattice vector (mod L) leaves all squared separations unchanged.
    rng = np.random.default_rng(1)
    q = rng.integers(0, 64 * 64, size=(1500, 3)).astype(np.float64) / 64.0
    e = [0.0, 0.5, 1.0, 3.0, 7.5, 20.0]
    a, _, _ = orc.xi(q[:, 0], q[:, 1], q[:, 2], edges=e, periodic=True, box=64.0)
    t = np.mod(q + np.array([17.25, 40.5, 63.984375]), 64.0)
    b, _, _ = orc.xi(t[:, 0], t[:, 1], t[:, 2], edges=e, periodic=True, box=64.0)
    assert np.array_equal(a, b)


def test_unit_weights_give_counts_and_ravg_in_bin(orc):
    c = synth.uniform_box(3000, 80.0, seed=24)
    e = synth.log_edges(0.5, 30.0, 10)
    w = np.ones(c.n)
    n, ws, rs = orc.xi(c.x, c.y, c.z, w1=w, edges=e, periodic=True, box=80.0, want_r=True)
    assert np.array_equal(ws, n.astype(np.float64))
    ok = n > 0
    ravg = rs[ok] / n[ok]
    assert np.all(ravg >= e[:-1][ok]) and np.all(ravg < e[1:][ok])


def test_invalid_arguments_rejected(orc):
    x = np.zeros(3)
    with pytest.raises(ValueError):
        orc.xi(x, x, x, edges=[1.0, 1.0], periodic=False)
    with pytest.raises(ValueError):
        orc.xi(x, x, x, edges=[-1.0, 1.0], periodic=False)
    with pytest.raises(ValueError):
        orc.xi(x, x, x, edges=[1.0], periodic=False)


def test_non_cubic_box_wraps_each_axis_with_its_own_side(orc):
    # box (10, 20, 40): a raw y difference of 19 wraps with Ly = 20 to -1
    x, y, z = pts((1, 0.5, 2), (1, 19.5, 2))
    n, _, _ = orc.xi(x, y, z, edges=[0.5, 1.5, 9.5], periodic=True, box=[10.0, 20.0, 40.0])
    assert n.tolist() == [2, 0]
    x, y, z = pts((1, 1, 0.75), (1, 1, 39.25))      # z: raw 38.5 -> -1.5 with Lz = 40
    n, _, _ = orc.xi(x, y, z, edges=[0.5, 1.75, 9.5], periodic=True, box=[10.0, 20.0, 40.0])
    assert n.tolist() == [2, 0]
    n, _, _ = orc.rppi(x, y, z, rp_edges=[0.0, 1.0], pimax=2.0, npibins=2, periodic=True,
                       box=[10.0, 20.0, 40.0])
    assert n.tolist() == [[0, 2]]


# (test function, keyword arguments) for every pin; the mutation test runs these
# against oracle builds with planted mistakes.
def pin_cases():
    import inspect
    params = {"axis": [0, 1, 2], "periodic": [True, False], "n": [0, 1]}
    out = []
    for name, fn in sorted(globals().items()):
        if not name.startswith("test_") or not callable(fn):
            continue
        if "orc" not in inspect.signature(fn).parameters:
            continue  # checks of the built oracle itself (e.g. across processes)
        extra = [a for a in inspect.signature(fn).parameters if a != "orc"]
        if not extra:
            out.append((fn, {}))
        else:
            (a,) = extra
            out.extend((fn, {a: v}) for v in params[a])
    return out


_THREADS_PROBE = r"""
import json, sys
sys.path.insert(0, {root!r})
import oracle
from paper_1911_08275_gb300 import synth
c = synth.neyman_scott(300, 10.0, 2.0, 60.0, seed=61)
w = synth.uniform_weights(c.n, 0.5, 1.5, seed=62)
e = synth.log_edges(0.2, 12.0, 10)
n, ws, rs = oracle.xi(c.x, c.y, c.z, edges=e, w1=w, periodic=True, box=60.0, want_r=True)
print(json.dumps([oracle.num_threads(), [int(v) for v in n], [float(v).hex() for v in ws],
                  [float(v).hex() for v in rs]]))
"""


def test_sums_do_not_depend_on_the_thread_count():
    # fixed row blocks combined in block order: the binary64 sums are the same
    # bits whatever the number of OpenMP threads
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for t in ("1", "3", "8"):
        env = dict(os.environ, OMP_NUM_THREADS=t)
        r = subprocess.run([sys.executable, "-c", _THREADS_PROBE.format(root=root)], env=env,
                           capture_output=True, text=True, check=True)
        outs.append(json.loads(r.stdout.strip().splitlines()[-1]))
    assert [o[0] for o in outs][:2] == [1, 3]
    assert all(o[1:] == outs[0][1:] for o in outs)
    assert sum(outs[0][1]) > 0
