"""Device-side sharding (cf_config.shard_index / shard_count): the shards of
one problem, counted one after another on one GPU, sum to the full result."""
import numpy as np
import pytest

import paper_1911_08275_gb300 as cf
from paper_1911_08275_gb300 import synth

pytestmark = pytest.mark.gpu


def dev(*arrays):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


@pytest.mark.parametrize("n", [2, 3, 7])
@pytest.mark.parametrize("mode", ["fp32_recheck", "fp64"])
def test_shards_sum_to_full(cuda_device, n, mode):
    cat = synth.neyman_scott(1500, 20.0, 2.0, 200.0, seed=511)
    e = synth.log_edges(0.1, 25.0, 20)
    xyz = dev(cat.x, cat.y, cat.z)
    full = cf.countpairs_xi(*xyz, e, boxsize=200.0, mode=mode)
    parts = [cf.countpairs_xi(*xyz, e, boxsize=200.0, mode=mode, shard=(k, n)) for k in range(n)]
    assert np.array_equal(sum(p.npairs for p in parts), full.npairs)
    assert sum(p.n_cellpairs for p in parts) == full.n_cellpairs
    assert all(p.npairs.sum() > 0 for p in parts)  # every shard gets work


def test_shards_rppi_and_weighted(cuda_device):
    cat = synth.neyman_scott(800, 20.0, 2.0, 150.0, seed=512)
    w = synth.uniform_weights(cat.n, 0.5, 1.5, seed=513)
    e = synth.log_edges(0.1, 20.0, 12)
    x, y, z, wd = dev(cat.x, cat.y, cat.z, w)
    full = cf.countpairs_rp_pi(x, y, z, e, 30.0, 30, boxsize=150.0)
    parts = [cf.countpairs_rp_pi(x, y, z, e, 30.0, 30, boxsize=150.0, shard=(k, 3)) for k in range(3)]
    assert np.array_equal(sum(p.npairs for p in parts), full.npairs)
    fw = cf.countpairs_xi(x, y, z, e, w=wd, boxsize=150.0)
    pw = [cf.countpairs_xi(x, y, z, e, w=wd, boxsize=150.0, shard=(k, 2)) for k in range(2)]
    assert np.array_equal(sum(p.npairs for p in pw), fw.npairs)
    assert np.allclose(sum(p.wsum for p in pw), fw.wsum, rtol=1e-5)


def test_invalid_shard_rejected(cuda_device):
    cat = synth.uniform_box(100, 10.0, seed=514)
    with pytest.raises(cf.CfError) as ei:
        cf.countpairs_xi(*dev(cat.x, cat.y, cat.z), [0.1, 1.0], boxsize=10.0, shard=(3, 3))
    assert ei.value.status == cf.CF_EINVAL
