"""cf_countpairs_xi_noalloc: the allocation-free DD(r) entry point.

It serves callers that cannot allocate device memory while counting (their GPU
memory is owned by another allocator, or they must not wait on cudaMalloc): all
scratch lives in a static device array inside the library.  The test calls it
through the C ABI twice in a row on different catalogues -- the second call must
not see the first call's leftovers in the shared array -- and requires integer
counts identical to cf_countpairs_xi (the tolerance of every count test here is
exact equality).  This file is named to be collected last.
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


def test_noalloc_rejects_too_many_points(cuda_device):
    cat = synth.uniform_box(131073, 100.0, seed=75)
    with pytest.raises(cf.CfError, match="131072"):
        cf.countpairs_xi_noalloc(*_dev(cat), [0.1, 1.0], boxsize=100.0)
