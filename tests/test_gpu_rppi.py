"""Parity of the CUDA DD(rp, pi) path with the CPU oracle (counts bit-exact).

Calls go through the C ABI (cf_countpairs_rp_pi).  rp^2 = dx^2 + dy^2 is binned
on the rp edges and pi = |dz| on the pi edges P_m = (pimax * m) / npibins
(line of sight = z).  Sizes keep the brute-force oracle at seconds while the GPU
path spans many columns, several z tiles and ragged chunk tails.
"""
import numpy as np
import pytest

import oracle
import paper_1911_08275_gb300 as cf
from paper_1911_08275_gb300 import synth

pytestmark = pytest.mark.gpu

MODES = ["fp32_recheck", "fp64"]


def dev(cat, dtype=np.float64):
    import torch
    c = cat.astype(dtype) if dtype != np.float64 else cat
    return [torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in (c.x, c.y, c.z)], c


def gpu_rppi(cat, e, pimax, npi, dtype=np.float64, **kw):
    (x, y, z), c = dev(cat, dtype)
    return cf.countpairs_rp_pi(x, y, z, e, pimax, npi, **kw), c


def oracle_rppi(c, e, pimax, npi, **kw):
    return oracle.rppi(c.x, c.y, c.z, rp_edges=e, pimax=pimax, npibins=npi, **kw)[0]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_uniform_20k_periodic(cuda_device, mode, dtype):
    cat = synth.c1_uniform20k()
    e = synth.log_edges(0.1, 25.0, 14)
    r, c = gpu_rppi(cat, e, 40.0, 40, dtype, boxsize=synth.BOX, mode=mode)
    ref = oracle_rppi(c, e, 40.0, 40, periodic=True, box=synth.BOX)
    assert r.npairs.shape == (14, 40)
    assert np.array_equal(r.npairs, ref)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("refine", [(1, 1, 1), (2, 2, 1), (3, 3, 2)])
def test_clustered_periodic(cuda_device, mode, refine):
    cat = synth.neyman_scott(1500, 20.0, 2.0, 200.0, seed=51)
    e = synth.log_edges(0.1, 20.0, 12)
    r, c = gpu_rppi(cat, e, 30.0, 30, boxsize=200.0, mode=mode, refine=refine)
    assert np.array_equal(r.npairs, oracle_rppi(c, e, 30.0, 30, periodic=True, box=200.0))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("periodic", [True, False])
def test_cross_correlation(cuda_device, mode, periodic):
    a = synth.neyman_scott(800, 20.0, 2.0, 150.0, seed=52)
    b = synth.uniform_box(25000, 150.0, seed=53)
    e = synth.log_edges(0.2, 20.0, 10)
    (xa, ya, za), _ = dev(a)
    (xb, yb, zb), _ = dev(b)
    r = cf.countpairs_rp_pi(xa, ya, za, e, 25.0, 25, x2=xb, y2=yb, z2=zb, periodic=periodic,
                            boxsize=150.0, mode=mode)
    ref = oracle.rppi(a.x, a.y, a.z, x2=b.x, y2=b.y, z2=b.z, rp_edges=e, pimax=25.0, npibins=25,
                      autocorr=False, periodic=periodic, box=150.0)[0]
    assert np.array_equal(r.npairs, ref)


@pytest.mark.parametrize("mode", MODES)
def test_open_box_non_integer_pi_bins(cuda_device, mode):
    # pimax / npibins = 37.3 / 17 is not a short binary fraction
    cat = synth.neyman_scott(900, 20.0, 3.0, 250.0, seed=54)
    e = synth.log_edges(0.1, 30.0, 16)
    r, c = gpu_rppi(cat, e, 37.3, 17, periodic=False, mode=mode)
    assert np.array_equal(r.npairs, oracle_rppi(c, e, 37.3, 17, periodic=False))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("nrp,npi", [(1, 1), (2, 2000), (64, 64)])
def test_bin_count_extremes(cuda_device, mode, nrp, npi):
    # (2, 2000) and (64, 64) leave room for fewer than one histogram copy per warp
    cat = synth.neyman_scott(600, 20.0, 2.0, 100.0, seed=55)
    e = synth.log_edges(0.05, 12.0, nrp)
    r, c = gpu_rppi(cat, e, 20.0, npi, boxsize=100.0, mode=mode)
    assert np.array_equal(r.npairs, oracle_rppi(c, e, 20.0, npi, periodic=True, box=100.0))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n", [0, 1, 2, 3, 31, 33])
def test_tiny_and_ragged(cuda_device, mode, n):
    cat = synth.uniform_box(n, 10.0, seed=56)
    e = [0.0, 0.5, 1.0, 2.0, 4.5]
    r, c = gpu_rppi(cat, e, 4.0, 4, boxsize=10.0, mode=mode)
    assert np.array_equal(r.npairs, oracle_rppi(c, e, 4.0, 4, periodic=True, box=10.0))


@pytest.mark.parametrize("mode", MODES)
def test_hand_enumerated_edges_and_wraps(cuda_device, mode):
    # rp = 5 exactly (3-4-5 in x, y), dz exactly on pi edges 1, 2, 3, and
    # separations that exist only through a periodic wrap in each axis.
    x = np.array([1.0, 4.0, 0.5, 9.5, 5.0, 5.0, 2.0, 2.0])
    y = np.array([1.0, 5.0, 5.0, 5.0, 0.25, 9.75, 7.0, 7.0])
    z = np.array([2.0, 4.0, 3.0, 3.0, 9.0, 1.0, 0.5, 9.5])
    cat = synth.Catalog(x, y, z, None, 10.0, "hand")
    for box, e, pimax, npi in ((14.0, [1.0, 5.0, 6.0], 4.0, 4), (10.0, [0.0, 1.0, 4.9], 3.0, 3),
                               (10.0, [0.25, 0.5, 1.0, 1.5, 4.0], 4.5, 9)):
        r, c = gpu_rppi(cat, e, pimax, npi, boxsize=box, mode=mode)
        ref = oracle_rppi(c, e, pimax, npi, periodic=True, box=box)
        assert np.array_equal(r.npairs, ref), (box, e)


def test_adversarial_pairs_on_rp_and_pi_edges(cuda_device):
    # Partners at rp equal to an rp edge and dz equal to a pi edge (up to
    # binary64 rounding), so the float32 path must settle many pairs exactly.
    e = synth.log_edges(0.1, 25.0, 14)
    n = 4000
    base = [synth.uniform01(57, s, n) * 340.0 + 40.0 for s in range(3)]
    k = (synth.random_u64(57, 3, n) % np.uint64(15)).astype(int)
    m = (synth.random_u64(57, 4, n) % np.uint64(41)).astype(float)
    sgn = np.where(synth.random_u64(57, 5, n) % np.uint64(2) == 0, 1.0, -1.0)
    d = synth.uniform01(57, 6, n)
    px = np.concatenate([base[0], base[0] + e[k] * d])
    py = np.concatenate([base[1], base[1] + e[k] * np.sqrt(np.maximum(0.0, 1.0 - d * d))])
    pz = np.concatenate([base[2], base[2] + sgn * m])
    cat = synth.Catalog(px, py, pz, None, 420.0, "adversarial")
    r, c = gpu_rppi(cat, e, 40.0, 40, boxsize=420.0, flags=cf.CF_FLAG_VERIFY_BAND)
    assert np.array_equal(r.npairs, oracle_rppi(c, e, 40.0, 40, periodic=True, box=420.0))
    assert r.n_band_violations == 0
    assert r.n_rechecked > 0


def test_verify_band_on_clustered_data(cuda_device):
    cat = synth.neyman_scott(2000, 20.0, 2.0, 200.0, seed=58)
    e = synth.log_edges(0.1, 25.0, 14)
    for dtype in (np.float64, np.float32):
        r, c = gpu_rppi(cat, e, 40.0, 40, dtype, boxsize=200.0, flags=cf.CF_FLAG_VERIFY_BAND)
        assert r.n_band_violations == 0
        assert np.array_equal(r.npairs, oracle_rppi(c, e, 40.0, 40, periodic=True, box=200.0))


def test_properties_symmetry_and_projection(cuda_device):
    cat = synth.neyman_scott(1200, 20.0, 2.0, 180.0, seed=59)
    e = synth.log_edges(0.1, 20.0, 10)
    (x, y, z), _ = dev(cat)
    auto = cf.countpairs_rp_pi(x, y, z, e, 30.0, 30, boxsize=180.0)
    cross = cf.countpairs_rp_pi(x, y, z, e, 30.0, 30, x2=x, y2=y, z2=z, boxsize=180.0)
    coarse = cf.countpairs_rp_pi(x, y, z, e, 30.0, 1, boxsize=180.0)
    f64 = cf.countpairs_rp_pi(x, y, z, e, 30.0, 30, boxsize=180.0, mode="fp64")
    p = np.random.default_rng(5).permutation(cat.n)
    (xp, yp, zp), _ = dev(cat.take(p))
    perm = cf.countpairs_rp_pi(xp, yp, zp, e, 30.0, 30, boxsize=180.0)
    assert np.array_equal(auto.npairs, cross.npairs)  # e_0 > 0: no self pairs in the cross count
    assert np.array_equal(auto.npairs, f64.npairs)
    assert np.array_equal(auto.npairs, perm.npairs)
    # unit-width pi bins summed over pi equal one pi bin of width pimax
    assert np.array_equal(auto.npairs.sum(axis=1), coarse.npairs[:, 0])


def test_count_evals_and_host_inputs(cuda_device):
    cat = synth.neyman_scott(500, 20.0, 2.0, 100.0, seed=60)
    e = synth.log_edges(0.1, 15.0, 10)
    a, _ = gpu_rppi(cat, e, 20.0, 20, boxsize=100.0)
    b, _ = gpu_rppi(cat, e, 20.0, 20, boxsize=100.0, flags=cf.CF_FLAG_COUNT_EVALS)
    h = cf.countpairs_rp_pi(cat.x, cat.y, cat.z, e, 20.0, 20, boxsize=100.0)
    assert np.array_equal(a.npairs, b.npairs) and np.array_equal(a.npairs, h.npairs)
    assert b.n_evaluated >= a.npairs.sum() // 2


def test_float_bit_cells_for_a_narrow_rp_range(cuda_device):
    # rp edges over a narrow range: the rp^2 table keeps cells on float32 bit
    # patterns (the other table shape of the kernels)
    cat = synth.neyman_scott(1500, 20.0, 2.0, 200.0, seed=47)
    e = np.linspace(10.0, 12.0, 5)
    for dtype in (np.float64, np.float32):
        r, c = gpu_rppi(cat, e, 20.0, 20, dtype, boxsize=200.0)
        assert r.table_linear == 0
        assert np.array_equal(r.npairs, oracle_rppi(c, e, 20.0, 20, periodic=True, box=200.0))


@pytest.mark.parametrize("bad", ["pimax_half_box", "pimax_zero", "npibins_zero", "too_many_bins"])
def test_invalid_arguments_rejected(cuda_device, bad):
    cat = synth.uniform_box(100, 10.0, seed=61)
    e, pimax, npi = [0.1, 1.0], 2.0, 4
    if bad == "pimax_half_box":
        pimax = 5.0
    elif bad == "pimax_zero":
        pimax = 0.0
    elif bad == "npibins_zero":
        npi = 0
    else:
        e, npi = synth.log_edges(0.1, 1.0, 10), 500
    (x, y, z), _ = dev(cat)
    with pytest.raises(cf.CfError) as ei:
        cf.countpairs_rp_pi(x, y, z, e, pimax, npi, boxsize=10.0)
    assert ei.value.status == cf.CF_EINVAL
