"""Sharded counting over processes (one GPU each) with one host-driven reduction.

Column pairs are independent work units and the result is a sum of histograms
(Sec. 2.1: the paper distributes cell pairs over OpenMP threads and adds the
per-thread histograms), so a problem splits across ranks without exchanging
any data: rank k counts shard k of n (``cf_config.shard_index / shard_count``:
the primary columns whose first point lies in slice k of the gridded points),
then one all-reduce sums the integer counts (exact) and the binary64 sums.

Before the data reduction every rank contributes a status word, so a rank
whose count raised makes every rank raise instead of leaving the others
waiting in the reduction; a rank that never arrives ends the others' next
collective with the process group's timeout.
"""
from __future__ import annotations

from typing import Callable

import numpy as np

from . import Result, countpairs_rp_pi, countpairs_xi


def _device_for(group):
    import torch
    import torch.distributed as dist
    return torch.device("cuda", torch.cuda.current_device()) \
        if dist.get_backend(group) == "nccl" else torch.device("cpu")


def run_sharded(count_fn: Callable[[int, int], Result], group=None) -> Result:
    """Call ``count_fn(k, n)`` for this rank's shard and sum the shards.

    ``count_fn`` returns a Result with npairs and optionally wsum / ravg; every
    rank receives the full Result.  If any rank's count_fn raised, every rank
    raises RuntimeError naming the failed ranks.
    """
    import torch
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    dev = _device_for(group)
    part, err = None, None
    try:
        part = count_fn(rank, world)
    except Exception as e:  # reported to every rank below
        err = e
    failed = torch.zeros(world, dtype=torch.int64, device=dev)
    failed[rank] = 1 if err is not None else 0
    dist.all_reduce(failed, group=group)
    if int(failed.sum()) > 0:
        bad = [int(r) for r in torch.nonzero(failed).flatten().tolist()]
        raise RuntimeError(f"sharded count failed on rank(s) {bad}") from err
    shape = part.npairs.shape
    n = torch.tensor(part.npairs.reshape(-1).astype(np.int64), dtype=torch.int64, device=dev)
    dist.all_reduce(n, group=group)
    npairs = n.cpu().numpy().astype(np.uint64).reshape(shape)
    wsum = ravg = None
    # every collective works on a copy: on the CPU backend the tensor would
    # otherwise share memory with the partial result that is still needed
    if part.wsum is not None:
        w = torch.tensor(part.wsum.reshape(-1), dtype=torch.float64, device=dev)
        dist.all_reduce(w, group=group)
        wsum = w.cpu().numpy().reshape(shape)
    if part.ravg is not None:
        # ravg is a ratio: reduce its numerator and denominator
        den = part.wsum if part.wsum is not None else part.npairs.astype(np.float64)
        num = torch.tensor((part.ravg * den).reshape(-1), dtype=torch.float64, device=dev)
        dist.all_reduce(num, group=group)
        tot = wsum if wsum is not None else npairs.astype(np.float64)
        num = num.cpu().numpy().reshape(shape)
        ravg = np.where(tot != 0, num / np.where(tot != 0, tot, 1.0), 0.0)
    stats = torch.tensor([part.n_cellpairs, part.n_evaluated, part.n_rechecked,
                          part.n_band_violations], dtype=torch.int64, device=dev)
    dist.all_reduce(stats, group=group)
    s = [int(v) for v in stats.cpu().tolist()]
    t = torch.tensor([part.kernel_ms, part.total_ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return Result(npairs, wsum, ravg, s[0], s[1], s[2], s[3], float(t[0]), float(t[1]),
                  part.n_kernels, part.refine_used, part.chunk_used, part.pp_used, part.tuned)


def countpairs_xi_sharded(*args, group=None, **kw) -> Result:
    """``countpairs_xi`` split over the ranks of ``group`` (each on its own GPU)."""
    return run_sharded(lambda k, n: countpairs_xi(*args, shard=(k, n), **kw), group)


def countpairs_rp_pi_sharded(*args, group=None, **kw) -> Result:
    """``countpairs_rp_pi`` split over the ranks of ``group``."""
    return run_sharded(lambda k, n: countpairs_rp_pi(*args, shard=(k, n), **kw), group)
