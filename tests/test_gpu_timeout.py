"""Bounded device waits give up cleanly and leave the context usable.

Every tile-barrier wait of the pair kernels is bounded in time; one that runs
out sets the error word, lets any copy still in flight land, and the kernel
returns, so the call reports CF_ETIMEOUT instead of hanging.  The diagnostic
flag CF_FLAG_DEBUG_STALL arms each CTA's first tile barrier of the float32
DD(r) kernel for a copy that is never issued (nothing can complete that
phase) and shortens the limit to 1 ms.  No fault, trap or endless loop is
involved: the test checks the status, then runs normal counts on the same
context and requires them bit-exact against the oracle.
"""
import time

import numpy as np
import pytest

import oracle
import paper_1911_08275_gb300 as cf
from paper_1911_08275_gb300 import synth

pytestmark = pytest.mark.gpu


def test_wait_that_nothing_completes_times_out_then_counts_are_exact(cuda_device):
    import torch
    cat = synth.neyman_scott(2000, 20.0, 2.0, 150.0, seed=211)
    e = synth.log_edges(0.1, 20.0, 16)
    xyz = [torch.from_numpy(v).cuda() for v in (cat.x, cat.y, cat.z)]
    ref = oracle.xi(cat.x, cat.y, cat.z, edges=e, periodic=True, box=150.0)[0]
    for _ in range(2):
        t0 = time.perf_counter()
        with pytest.raises(cf.CfError) as ei:
            cf.countpairs_xi(*xyz, e, boxsize=150.0, flags=cf.CF_FLAG_DEBUG_STALL)
        assert ei.value.status == cf.CF_ETIMEOUT
        assert time.perf_counter() - t0 < 5.0  # the 1 ms limits, not a hang
        torch.cuda.synchronize()  # the context is healthy
        r = cf.countpairs_xi(*xyz, e, boxsize=150.0)
        assert np.array_equal(r.npairs, ref) and ref.sum() > 0
    r64 = cf.countpairs_xi(*xyz, e, boxsize=150.0, mode="fp64")
    assert np.array_equal(r64.npairs, ref)
