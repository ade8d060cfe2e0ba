"""Sharded counting across processes (gloo, world size 2, CPU only): the
reduction of per-rank partial histograms, ravg recombination and failure
handling.  Partial counts come from the oracle on disjoint row slices, which
partition the pairs exactly as the GPU shards do (each pair counted once)."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, mode, q):
    try:
        import torch.distributed as dist
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        import datetime
        dist.init_process_group("gloo", rank=rank, world_size=world,
                                timeout=datetime.timedelta(seconds=20))
        import oracle
        from paper_1911_08275_gb300 import Result, parallel, synth
        d = synth.neyman_scott(60, 20.0, 2.0, 60.0, seed=501)
        r = synth.uniform_box(1500, 60.0, seed=502)
        wd = synth.uniform_weights(d.n, 0.5, 1.5, seed=503)
        wr = synth.uniform_weights(r.n, 0.5, 1.5, seed=504)
        e = synth.log_edges(0.2, 12.0, 8)

        if mode == "exit" and rank == 1:
            os._exit(0)  # leaves between steps, before the collective: rank 0 must not hang

        def count(k, n):
            if mode == "fail" and k == 1:
                raise ValueError("injected failure on rank 1")
            lo, hi = d.n * k // n, d.n * (k + 1) // n
            npairs, ws, rs = oracle.xi(d.x[lo:hi], d.y[lo:hi], d.z[lo:hi], w1=wd[lo:hi], x2=r.x,
                                       y2=r.y, z2=r.z, w2=wr, edges=e, autocorr=False,
                                       periodic=True, box=60.0, want_r=True)
            ravg = np.where(ws != 0, rs / np.where(ws != 0, ws, 1.0), 0.0)
            return Result(npairs, ws, ravg, 1, 0, 0, 0, 1.0, 2.0)

        out = parallel.run_sharded(count)
        full_n, full_w, full_r = oracle.xi(d.x, d.y, d.z, w1=wd, x2=r.x, y2=r.y, z2=r.z, w2=wr,
                                           edges=e, autocorr=False, periodic=True, box=60.0,
                                           want_r=True)
        ok = (np.array_equal(out.npairs, full_n) and np.allclose(out.wsum, full_w, rtol=1e-12)
              and np.allclose(out.ravg, np.where(full_w != 0, full_r / np.where(full_w != 0, full_w, 1),
                                                 0), rtol=1e-12) and out.n_cellpairs == world)
        q.put((rank, "ok" if ok else "mismatch"))
    except RuntimeError as ex:
        q.put((rank, "raised: " + str(ex)))
    except Exception as ex:  # noqa: BLE001
        q.put((rank, "error: " + repr(ex)))
    finally:
        try:
            import torch.distributed as dist
            if dist.is_initialized():
                dist.destroy_process_group()
        except Exception:  # noqa: BLE001
            pass


def _run(mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(k, 2, port, mode, q)) for k in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
    for p in ps:
        if p.is_alive():
            p.kill()
            pytest.fail("a rank did not finish")
    out = {}
    while not q.empty():
        k, v = q.get(timeout=5)
        out[k] = v
    return out


def test_shards_sum_to_the_full_histogram():
    out = _run("ok")
    assert out == {0: "ok", 1: "ok"}


def test_a_failing_rank_makes_every_rank_raise():
    out = _run("fail")
    assert all(v.startswith("raised: sharded count failed on rank(s) [1]") for v in out.values()), out


def test_a_rank_that_leaves_ends_the_others_collective_with_an_error():
    out = _run("exit")
    assert 1 not in out and 0 in out and not out[0] == "ok", out
