"""Autotuner (cf_config.autotune) and explicit kernel shapes: every choice
counts the same pairs; the first call of a signature tunes, later calls reuse."""
import numpy as np
import pytest

import oracle
import paper_1911_08275_gb300 as cf
from paper_1911_08275_gb300 import synth

pytestmark = pytest.mark.gpu


def dev(cat):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in (cat.x, cat.y, cat.z)]


def test_autotune_counts_equal_and_cache_reused(cuda_device):
    cf.tune_clear()
    cat = synth.neyman_scott(2000, 20.0, 2.0, 200.0, seed=91)
    e = synth.log_edges(0.1, 25.0, 20)
    xyz = dev(cat)
    ref = oracle.xi(cat.x, cat.y, cat.z, edges=e, periodic=True, box=200.0)[0]
    a = cf.countpairs_xi(*xyz, e, boxsize=200.0, autotune=True)
    b = cf.countpairs_xi(*xyz, e, boxsize=200.0, autotune=True)
    assert np.array_equal(a.npairs, ref) and np.array_equal(b.npairs, ref)
    assert a.tuned == 1 and b.tuned == 2 and cf.tune_count() == 1
    assert a.refine_used in ((1, 1, 1), (2, 2, 1), (3, 3, 1), (4, 4, 1)) and a.refine_used == b.refine_used
    assert (a.chunk_used, a.pp_used) in ((16, 2), (8, 2), (16, 1), (32, 1))
    # an explicit refinement is kept
    c = cf.countpairs_xi(*xyz, e, boxsize=200.0, autotune=True, refine=(4, 4, 1))
    assert c.refine_used == (4, 4, 1) and np.array_equal(c.npairs, ref)
    cf.tune_clear()


@pytest.mark.parametrize("kind", ["rppi", "dr_open_weighted"])
def test_autotune_other_kinds(cuda_device, kind):
    cf.tune_clear()
    cat = synth.neyman_scott(800, 20.0, 2.0, 150.0, seed=92)
    e = synth.log_edges(0.1, 20.0, 12)
    xyz = dev(cat)
    if kind == "rppi":
        ref = oracle.rppi(cat.x, cat.y, cat.z, rp_edges=e, pimax=30.0, npibins=30, periodic=True,
                          box=150.0)[0]
        r = cf.countpairs_rp_pi(*xyz, e, 30.0, 30, boxsize=150.0, autotune=True)
    else:
        import torch
        w = synth.uniform_weights(cat.n, 0.5, 1.5, seed=93)
        ref = oracle.xi(cat.x, cat.y, cat.z, w1=w, edges=e, periodic=False)[0]
        r = cf.countpairs_xi(*xyz, e, w=torch.from_numpy(w).cuda(), periodic=False, autotune=True)
    assert np.array_equal(r.npairs, ref) and r.tuned == 1
    cf.tune_clear()


@pytest.mark.parametrize("chunk,pp", [(8, 1), (8, 2), (16, 1), (16, 2), (32, 1)])
def test_explicit_kernel_shapes(cuda_device, chunk, pp):
    cat = synth.neyman_scott(1500, 20.0, 2.0, 200.0, seed=94)
    e = synth.log_edges(0.1, 25.0, 20)
    r = cf.countpairs_xi(*dev(cat), e, boxsize=200.0, pair_chunk=chunk, pair_pp=pp)
    assert (r.chunk_used, r.pp_used) == (chunk, pp)
    assert np.array_equal(r.npairs, oracle.xi(cat.x, cat.y, cat.z, edges=e, periodic=True,
                                              box=200.0)[0])


@pytest.mark.parametrize("chunk,pp", [(12, 0), (0, 3)])
def test_invalid_kernel_shapes_rejected(cuda_device, chunk, pp):
    cat = synth.uniform_box(100, 10.0, seed=95)
    with pytest.raises(cf.CfError) as ei:
        cf.countpairs_xi(*dev(cat), [0.1, 1.0], boxsize=10.0, pair_chunk=chunk, pair_pp=pp)
    assert ei.value.status == cf.CF_EINVAL


def test_default_refinement_follows_the_points_per_column(cuda_device):
    # refine (0, 0, 0): r = round(Rmax / s) in [1, 4], s the column side over
    # which the smaller catalogue holds 1024 points: 200k uniform points in a
    # box of 200 give s = 14.3, so Rmax 5, 30, 60 -> r = 1 (clamped), 2, 4; a
    # cross count against a 20k-point catalogue (s = 45.3) at Rmax 60 -> 1
    big = synth.uniform_box(200000, 200.0, seed=95)
    small = synth.uniform_box(20000, 200.0, seed=96)
    xb, xs = dev(big), dev(small)
    for rmax, want in ((5.0, 1), (30.0, 2), (60.0, 4)):
        e = synth.log_edges(0.5, rmax, 8)
        r = cf.countpairs_xi(*xb, e, boxsize=200.0)
        assert r.refine_used == (want, want, 1), (rmax, r.refine_used)
        fixed = cf.countpairs_xi(*xb, e, boxsize=200.0, refine=(2, 2, 1))
        assert np.array_equal(r.npairs, fixed.npairs)
    e = synth.log_edges(0.5, 60.0, 8)
    rc = cf.countpairs_xi(*xs, e, x2=xb[0], y2=xb[1], z2=xb[2], boxsize=200.0)
    assert rc.refine_used == (1, 1, 1)
    fixed = cf.countpairs_xi(*xs, e, x2=xb[0], y2=xb[1], z2=xb[2], boxsize=200.0, refine=(3, 3, 1))
    assert np.array_equal(rc.npairs, fixed.npairs)
