"""cf_countpairs_xi_noalloc: the allocation-free DD(r) entry point.

It serves callers that cannot allocate device memory while counting (their GPU
memory is owned by another allocator, or they must not wait on cudaMalloc): all
scratch lives in a static device array inside the library.  The tests call it
through the C ABI and require integer counts identical to cf_countpairs_xi (the
tolerance of every count test here is exact equality):

* twice in a row on different catalogues, so the second call must not see the
  first call's leftovers in the shared array;
* cross and open-box counts;
* grids the planner must coarsen: a fine grid whose column count exceeds the
  array's column cap, and a cross-correlation of two 131072-point catalogues
  whose column-pair list alone would not fit the array at the planner's grid
  (box / Rmax = 84).  With at most 131072 points per catalogue a grid of one
  column always fits (about 16 MiB), so the coarsening loop always ends with a
  grid that fits and its "does not fit" error stays a guard; the size limit's
  error is what a caller can meet, and is tested;
* a capturing stream is refused (the call synchronises its stream).

This file is named to be collected last.
"""
import numpy as np
import pytest

import paper_1911_08275_gb300 as cf
from paper_1911_08275_gb300 import synth

pytestmark = pytest.mark.gpu


def _dev(cat):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in (cat.x, cat.y, cat.z)]


@pytest.mark.parametrize("mode", ["fp32_recheck", "fp64"])
def test_noalloc_matches_allocating_entry_point_twice(cuda_device, mode):
    e = synth.log_edges(0.1, 25.0, 20)
    first = synth.neyman_scott(3000, 20.0, 2.0, 200.0, seed=71)   # ~60k points
    second = synth.uniform_box(20000, 150.0, seed=72)
    for cat, box in ((first, 200.0), (second, 150.0)):
        xyz = _dev(cat)
        want = cf.countpairs_xi(*xyz, e, boxsize=box, mode=mode)
        got = cf.countpairs_xi_noalloc(*xyz, e, boxsize=box, mode=mode)
        assert np.array_equal(got.npairs, want.npairs)
        assert got.npairs.sum() > 0


def test_noalloc_cross_and_open_box(cuda_device):
    e = synth.log_edges(0.2, 20.0, 12)
    a = synth.neyman_scott(500, 20.0, 2.0, 120.0, seed=73)
    b = synth.uniform_box(30000, 120.0, seed=74)
    xa, xb = _dev(a), _dev(b)
    for periodic in (True, False):
        kw = dict(x2=xb[0], y2=xb[1], z2=xb[2], periodic=periodic, boxsize=120.0)
        want = cf.countpairs_xi(*xa, e, **kw)
        got = cf.countpairs_xi_noalloc(*xa, e, **kw)
        assert np.array_equal(got.npairs, want.npairs)


def test_noalloc_fine_grid_is_coarsened(cuda_device):
    # box 420, Rmax 2, refine 2: 420 x 420 base columns for 100k points; the
    # planner halves them to at most one column per 32 points, and the halved
    # grid must count the same pairs
    cat = synth.uniform_box(100000, 420.0, seed=77)
    e = synth.log_edges(0.05, 2.0, 8)
    xyz = _dev(cat)
    want = cf.countpairs_xi(*xyz, e, boxsize=420.0, refine=(2, 2, 1))
    got = cf.countpairs_xi_noalloc(*xyz, e, boxsize=420.0, refine=(2, 2, 1))
    assert np.array_equal(got.npairs, want.npairs) and got.npairs.sum() > 0


@pytest.mark.parametrize("periodic", [True, False])
def test_noalloc_cross_at_the_size_limit(cuda_device, periodic):
    # two catalogues of 131072 points, box / Rmax = 84, refine 4: over the
    # 83 x 83 columns the point cap leaves, the 81-offset cross work list and
    # the window records need about 57 MB, so the planner coarsens further to
    # fit the 32 MiB array
    a = synth.uniform_box(131072, 420.0, seed=78)
    b = synth.uniform_box(131072, 420.0, seed=79)
    e = synth.log_edges(0.1, 5.0, 10)
    xa, xb = _dev(a), _dev(b)
    kw = dict(x2=xb[0], y2=xb[1], z2=xb[2], periodic=periodic, boxsize=420.0, refine=(4, 4, 1))
    want = cf.countpairs_xi(*xa, e, **kw)
    got = cf.countpairs_xi_noalloc(*xa, e, **kw)
    assert np.array_equal(got.npairs, want.npairs) and got.npairs.sum() > 0


def test_noalloc_rejects_too_many_points(cuda_device):
    cat = synth.uniform_box(131073, 100.0, seed=75)
    with pytest.raises(cf.CfError, match="131072"):
        cf.countpairs_xi_noalloc(*_dev(cat), [0.1, 1.0], boxsize=100.0)


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")  # nothing may be captured
def test_noalloc_rejects_a_capturing_stream(cuda_device):
    import torch
    cat = synth.uniform_box(2000, 50.0, seed=76)
    xyz = _dev(cat)
    first = cf.countpairs_xi_noalloc(*xyz, [0.5, 2.0], boxsize=50.0)  # set-up outside capture
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with pytest.raises(cf.CfError, match="captured"):
        with torch.cuda.graph(g, stream=s):
            cf.countpairs_xi_noalloc(*xyz, [0.5, 2.0], boxsize=50.0, stream=s.cuda_stream)
    torch.cuda.synchronize()
    again = cf.countpairs_xi_noalloc(*xyz, [0.5, 2.0], boxsize=50.0)  # the context is fine
    assert np.array_equal(again.npairs, first.npairs) and first.npairs.sum() > 0
