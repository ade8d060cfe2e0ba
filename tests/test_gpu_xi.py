"""Parity of the CUDA DD(r) path with the CPU oracle (integer counts bit-exact).

Every call goes through the C ABI (cf_countpairs_xi) via the ctypes binding.
Sizes are chosen so the brute-force oracle finishes in seconds while the GPU
path still spans many columns, several z-tiles and ragged chunk tails.
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


def gpu_xi(cat, edges, dtype=np.float64, **kw):
    (x, y, z), c = dev(cat, dtype)
    return cf.countpairs_xi(x, y, z, edges, **kw), c


def oracle_xi(c, edges, **kw):
    return oracle.xi(c.x, c.y, c.z, edges=edges, **kw)[0]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_c1_uniform_20k(cuda_device, mode, dtype):
    cat = synth.c1_uniform20k()
    e = synth.log_edges(0.1, 25.0, 20)
    r, c = gpu_xi(cat, e, dtype, boxsize=synth.BOX, mode=mode)
    ref = oracle_xi(c, e, periodic=True, box=synth.BOX)
    assert np.array_equal(r.npairs, ref)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("refine", [(1, 1, 1), (2, 2, 1), (3, 3, 2), (4, 4, 1), (1, 3, 4)])
def test_clustered_refine_factors(cuda_device, mode, refine):
    cat = synth.neyman_scott(1500, 20.0, 2.0, 200.0, seed=31)
    e = synth.log_edges(0.05, 30.0, 18)
    r, c = gpu_xi(cat, e, boxsize=200.0, mode=mode, refine=refine)
    assert np.array_equal(r.npairs, oracle_xi(c, e, periodic=True, box=200.0))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("periodic", [True, False])
def test_cross_correlation(cuda_device, mode, periodic):
    a = synth.neyman_scott(800, 20.0, 2.0, 150.0, seed=32)
    b = synth.uniform_box(25000, 150.0, seed=33)
    e = synth.log_edges(0.2, 20.0, 15)
    (xa, ya, za), _ = dev(a)
    (xb, yb, zb), _ = dev(b)
    r = cf.countpairs_xi(xa, ya, za, e, x2=xb, y2=yb, z2=zb, periodic=periodic, boxsize=150.0,
                         mode=mode)
    ref = oracle.xi(a.x, a.y, a.z, x2=b.x, y2=b.y, z2=b.z, edges=e, autocorr=False,
                    periodic=periodic, box=150.0)[0]
    assert np.array_equal(r.npairs, ref)


@pytest.mark.parametrize("mode", MODES)
def test_open_box_clustered_auto(cuda_device, mode):
    cat = synth.neyman_scott(1000, 20.0, 3.0, 300.0, seed=34)
    e = synth.log_edges(0.1, 40.0, 20)
    r, c = gpu_xi(cat, e, periodic=False, mode=mode)
    assert np.array_equal(r.npairs, oracle_xi(c, e, periodic=False))


@pytest.mark.parametrize("mode", MODES)
def test_few_columns_per_axis_and_non_cubic_box(cuda_device, mode):
    # box (100, 60, 90), Rmax 28: 3 x 2 base columns, the stencil wraps onto the
    # same column under two different periodic images.
    box = np.array([100.0, 60.0, 90.0])
    u = [synth.uniform01(35, s, 15000) * box[s] for s in range(3)]
    cat = synth.Catalog(u[0], u[1], u[2], None, 100.0, "noncubic")
    e = synth.log_edges(0.5, 28.0, 12)
    for refine in [(1, 1, 1), (2, 2, 1), (4, 4, 1)]:
        (x, y, z), _ = dev(cat)
        r = cf.countpairs_xi(x, y, z, e, boxsize=box, mode=mode, refine=refine)
        assert np.array_equal(r.npairs, oracle.xi(cat.x, cat.y, cat.z, edges=e, box=box)[0])


@pytest.mark.parametrize("mode", MODES)
def test_dense_columns_span_several_tiles(cuda_device, mode):
    # 60k points, box 40, Rmax 19: 2x2 base columns of ~15k points each, so the
    # staged secondary column is split into many shared-memory tiles.
    cat = synth.uniform_box(60000, 40.0, seed=36)
    e = synth.log_edges(0.01, 19.0, 25)
    r, c = gpu_xi(cat, e, boxsize=40.0, mode=mode, refine=(1, 1, 1))
    assert np.array_equal(r.npairs, oracle_xi(c, e, periodic=True, box=40.0))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n", [0, 1, 2, 3, 31, 33])
def test_tiny_and_ragged(cuda_device, mode, n):
    cat = synth.uniform_box(n, 10.0, seed=37)
    e = [0.0, 0.5, 1.0, 2.0, 4.5]
    r, c = gpu_xi(cat, e, boxsize=10.0, mode=mode)
    assert np.array_equal(r.npairs, oracle_xi(c, e, periodic=True, box=10.0))


@pytest.mark.parametrize("mode", MODES)
def test_hand_enumerated_edges_and_wraps(cuda_device, mode):
    # (0,0,0)-(3,4,0) exactly on the squared edge 25; wraps across every face.
    x = np.array([0.5, 3.5, 0.25, 9.75, 5.0, 5.0])
    y = np.array([0.5, 4.5, 5.0, 5.0, 0.125, 9.875])
    z = np.array([5.0, 5.0, 0.25, 0.25, 9.5, 0.5])
    cat = synth.Catalog(x, y, z, None, 10.0, "hand")
    for box, e in ((14.0, [1.0, 5.0, 6.0]), (10.0, [0.25, 0.5, 1.0, 1.5, 4.0]),
                   (10.0, [0.0, 0.75, 1.0, 4.9])):
        r, c = gpu_xi(cat, e, boxsize=box, mode=mode)
        assert np.array_equal(r.npairs, oracle_xi(c, e, periodic=True, box=box)), e


@pytest.mark.parametrize("mode", MODES)
def test_coincident_points(cuda_device, mode):
    x = np.full(500, 3.25)
    cat = synth.Catalog(x, x.copy(), x.copy(), None, 10.0, "same")
    for e in ([0.0, 1.0], [0.125, 1.0]):
        r, c = gpu_xi(cat, e, boxsize=10.0, mode=mode)
        assert np.array_equal(r.npairs, oracle_xi(c, e, periodic=True, box=10.0))


def test_adversarial_pairs_on_squared_edges(cuda_device):
    # Partners placed at separations equal to bin edges (up to binary64 rounding),
    # so the float32 path must re-check many pairs to stay exact.
    e = synth.log_edges(0.1, 25.0, 20)
    n = 4000
    base = [synth.uniform01(38, s, n) * 370.0 + 20.0 for s in range(3)]
    k = (synth.random_u64(38, 3, n) % np.uint64(21)).astype(int)
    d = synth.uniform01(38, 4, n)
    dirs = np.stack([d, np.sqrt(np.maximum(0.0, 1.0 - d * d)), np.zeros(n)])
    px = np.concatenate([base[0], base[0] + e[k] * dirs[0]])
    py = np.concatenate([base[1], base[1] + e[k] * dirs[1]])
    pz = np.concatenate([base[2], base[2] + e[k] * dirs[2]])
    cat = synth.Catalog(px, py, pz, None, 420.0, "adversarial")
    r, c = gpu_xi(cat, e, boxsize=420.0, mode="fp32_recheck", flags=cf.CF_FLAG_VERIFY_BAND)
    assert np.array_equal(r.npairs, oracle_xi(c, e, periodic=True, box=420.0))
    assert r.n_band_violations == 0
    assert r.n_rechecked > 0


def test_verify_band_on_clustered_data(cuda_device):
    cat = synth.neyman_scott(2000, 20.0, 2.0, 200.0, seed=39)
    e = synth.log_edges(0.1, 25.0, 20)
    for dtype in (np.float64, np.float32):
        r, c = gpu_xi(cat, e, dtype, boxsize=200.0, flags=cf.CF_FLAG_VERIFY_BAND)
        assert r.n_band_violations == 0
        assert np.array_equal(r.npairs, oracle_xi(c, e, periodic=True, box=200.0))


def test_host_inputs_equal_device_inputs(cuda_device):
    cat = synth.neyman_scott(500, 20.0, 2.0, 100.0, seed=40)
    e = synth.log_edges(0.1, 20.0, 10)
    rd, _ = gpu_xi(cat, e, boxsize=100.0)
    rh = cf.countpairs_xi(cat.x, cat.y, cat.z, e, boxsize=100.0)
    assert np.array_equal(rd.npairs, rh.npairs)


def test_no_prune_and_count_evals_do_not_change_counts(cuda_device):
    cat = synth.neyman_scott(1000, 20.0, 2.0, 150.0, seed=41)
    e = synth.log_edges(0.1, 25.0, 20)
    # refine 4: columns 7.5 wide, so stencil corners (3 empty columns apart on
    # both axes, gap >= 31.8 > Rmax) are pruned by their bounding boxes.
    kw = dict(boxsize=150.0, refine=(4, 4, 1))
    r0, _ = gpu_xi(cat, e, **kw)
    r1, _ = gpu_xi(cat, e, flags=cf.CF_FLAG_NO_PRUNE | cf.CF_FLAG_COUNT_EVALS, **kw)
    r2, _ = gpu_xi(cat, e, flags=cf.CF_FLAG_COUNT_EVALS, **kw)
    assert np.array_equal(r0.npairs, r1.npairs) and np.array_equal(r0.npairs, r2.npairs)
    assert r1.n_cellpairs > r2.n_cellpairs > 0
    # every counted unordered pair was evaluated at least once
    assert r2.n_evaluated >= r0.npairs.sum() // 2


def test_deterministic_and_permutation_invariant(cuda_device):
    cat = synth.neyman_scott(1500, 20.0, 2.0, 200.0, seed=42)
    e = synth.log_edges(0.1, 25.0, 20)
    a, _ = gpu_xi(cat, e, boxsize=200.0)
    b, _ = gpu_xi(cat, e, boxsize=200.0)
    p = np.random.default_rng(3).permutation(cat.n)
    c, _ = gpu_xi(cat.take(p), e, boxsize=200.0)
    assert np.array_equal(a.npairs, b.npairs) and np.array_equal(a.npairs, c.npairs)


@pytest.mark.parametrize("bad", ["nan", "negative", "at_box", "rmax"])
def test_invalid_inputs_rejected(cuda_device, bad):
    cat = synth.uniform_box(100, 10.0, seed=43)
    x = cat.x.copy()
    e = [0.1, 1.0]
    if bad == "nan":
        x[7] = np.nan
    elif bad == "negative":
        x[7] = -1e-9
    elif bad == "at_box":
        x[7] = 10.0
    else:
        e = [0.1, 5.0]
    import torch
    t = [torch.from_numpy(v).cuda() for v in (x, cat.y, cat.z)]
    with pytest.raises(cf.CfError) as ei:
        cf.countpairs_xi(*t, e, boxsize=10.0)
    assert ei.value.status == cf.CF_EINVAL
    # the library stays usable after a rejected call
    r = cf.countpairs_xi(*[torch.from_numpy(v).cuda() for v in (cat.x, cat.y, cat.z)], [0.1, 1.0],
                         boxsize=10.0)
    assert r.npairs.shape == (1,)


@pytest.mark.parametrize("edges", [synth.log_edges(1e-3, 30.0, 40),  # wide range
                                   synth.linear_edges(0.0, 25.0, 25),  # from 0
                                   synth.log_edges(0.1, 25.0, 20)])
def test_table_shapes_verify_band(cuda_device, edges):
    cat = synth.neyman_scott(1500, 20.0, 2.0, 200.0, seed=44)
    for dtype in (np.float64, np.float32):
        r, c = gpu_xi(cat, edges, dtype, boxsize=200.0, flags=cf.CF_FLAG_VERIFY_BAND)
        assert r.n_band_violations == 0
        assert np.array_equal(r.npairs, oracle_xi(c, edges, periodic=True, box=200.0))
        r2, _ = gpu_xi(cat, edges, dtype, boxsize=200.0, pair_chunk=16, pair_pp=2)
        assert np.array_equal(r2.npairs, r.npairs)


def test_float_bit_cells_for_a_narrow_edge_range(cuda_device):
    # Edges over a narrow range make the host keep the table with cells on
    # float32 bit patterns (finer there than cells linear in d2): the kernels'
    # other table shape, in the verifying sweep and in the production shape.
    cat = synth.neyman_scott(1500, 20.0, 2.0, 200.0, seed=46)
    edges = np.linspace(10.0, 12.0, 9)
    for dtype in (np.float64, np.float32):
        for kw in (dict(flags=cf.CF_FLAG_VERIFY_BAND), dict(pair_chunk=16, pair_pp=2)):
            r, c = gpu_xi(cat, edges, dtype, boxsize=200.0, **kw)
            assert r.table_linear == 0
            assert r.n_band_violations == 0
            assert np.array_equal(r.npairs, oracle_xi(c, edges, periodic=True, box=200.0))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_pinned_host_inputs(cuda_device, dtype):
    # Page-locked host inputs (and views one element into page-locked buffers) are
    # copied inside the call like pageable ones; counts and sums match the oracle.
    import torch
    cat = synth.neyman_scott(700, 20.0, 2.0, 150.0, seed=95)
    w = synth.uniform_weights(cat.n, 0.5, 1.5, seed=96)
    e = synth.log_edges(0.1, 20.0, 12)
    c = cat.astype(dtype) if dtype != np.float64 else cat
    ref_n, ref_w, _ = oracle.xi(c.x, c.y, c.z, w1=w, edges=e, periodic=True, box=150.0)
    pinned = [torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for v in (c.x, c.y, c.z)]
    pw = torch.from_numpy(w).pin_memory()
    r = cf.countpairs_xi(*pinned, e, w=pw, boxsize=150.0)
    assert np.array_equal(r.npairs, ref_n)
    assert np.allclose(r.wsum, ref_w, rtol=1e-5, atol=0.0)
    # views one element into pinned buffers
    big = [torch.cat([torch.zeros(1, dtype=t.dtype), t]).pin_memory() for t in pinned]
    views = [b[1:] for b in big]
    r2 = cf.countpairs_xi(*views, e, boxsize=150.0)
    assert np.array_equal(r2.npairs, ref_n)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("periodic", [True, False])
def test_sparse_catalogues_get_wide_columns(cuda_device, mode, periodic):
    # 100 and 400 points in a box of 1000 with Rmax 40: the planner keeps at
    # least 32 points per column, so the grid shrinks to 1 x 1 and 3 x 3
    # columns, fewer than the stencil's 2 r + 1 per axis (refine 2): the same
    # column then appears under several periodic images
    e = synth.log_edges(1.0, 40.0, 8)
    for n, refine in ((100, (2, 2, 1)), (400, (2, 2, 1)), (400, (0, 0, 0))):
        cat = synth.neyman_scott(n // 10, 10.0, 15.0, 1000.0, seed=44 + n)
        r, c = gpu_xi(cat, e, boxsize=1000.0, mode=mode, periodic=periodic, refine=refine)
        assert np.array_equal(r.npairs, oracle_xi(c, e, periodic=periodic, box=1000.0)), (n, refine)
        u = synth.uniform_box(n, 1000.0, seed=45 + n)
        (ux, uy, uz), _ = dev(u)
        (cx, cy, cz), _ = dev(c)
        rc = cf.countpairs_xi(cx, cy, cz, e, x2=ux, y2=uy, z2=uz, boxsize=1000.0, mode=mode,
                              periodic=periodic, refine=refine)
        want = oracle.xi(c.x, c.y, c.z, edges=e, x2=u.x, y2=u.y, z2=u.z, autocorr=False,
                         periodic=periodic, box=1000.0)[0]
        assert np.array_equal(rc.npairs, want), (n, refine)
