"""Batched persistent launch (cf_batch_*): every job's counts equal the
single-call path (itself parity-tested against the oracle), with and without
the captured CUDA graph, across job switches, in-place input updates and
re-planning of open boxes."""
import numpy as np
import pytest

import oracle
import paper_1911_08275_gb300 as cf
from paper_1911_08275_gb300 import synth

pytestmark = pytest.mark.gpu


def dev(cat):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in (cat.x, cat.y, cat.z)]


def single(job, xyz, xyz2=None):
    kw = dict(boxsize=job["box"], mode=job["mode"], periodic=job.get("periodic", True))
    if xyz2 is not None:
        kw.update(x2=xyz2[0], y2=xyz2[1], z2=xyz2[2])
    if job["kind"] == "xi":
        return cf.countpairs_xi(*xyz, job["edges"], **kw).npairs
    return cf.countpairs_rp_pi(*xyz, job["edges"], job["pimax"], job["npibins"], **kw).npairs


def add(b, job, xyz, xyz2=None):
    kw = dict(boxsize=job["box"], mode=job["mode"], periodic=job.get("periodic", True))
    if xyz2 is not None:
        kw.update(x2=xyz2[0], y2=xyz2[1], z2=xyz2[2])
    if job["kind"] == "xi":
        return b.add_xi(*xyz, job["edges"], **kw)
    return b.add_rp_pi(*xyz, job["edges"], job["pimax"], job["npibins"], **kw)


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_equals_single_calls(cuda_device, use_graph):
    jobs = [synth.batch_job(j, scale=0.01) for j in range(16)]
    b = cf.Batch()
    xyz = [dev(jb["cat"]) for jb in jobs]
    res = [add(b, jb, x) for jb, x in zip(jobs, xyz)]
    stats = b.run(use_graph=use_graph)
    assert stats["n_jobs"] == 16 and stats["planned"] == 1
    for jb, x, r in zip(jobs, xyz, res):
        assert np.array_equal(r.npairs, single(jb, x)), jb["j"]
    assert stats["pairs"] == sum(int(r.npairs.sum()) for r in res)
    # second run: replay (or re-issue) on the same plan
    stats2 = b.run(use_graph=use_graph)
    assert stats2["planned"] == 0
    for jb, x, r in zip(jobs, xyz, res):
        assert np.array_equal(r.npairs, single(jb, x)), jb["j"]
    b.close()


def test_batch_small_jobs_against_oracle(cuda_device):
    jobs = [synth.batch_job(j, scale=0.002) for j in range(8)]
    b = cf.Batch()
    res = [add(b, jb, dev(jb["cat"])) for jb in jobs]
    b.run()
    for jb, r in zip(jobs, res):
        c = jb["cat"]
        if jb["kind"] == "xi":
            ref = oracle.xi(c.x, c.y, c.z, edges=jb["edges"], periodic=True, box=jb["box"])[0]
        else:
            ref = oracle.rppi(c.x, c.y, c.z, rp_edges=jb["edges"], pimax=jb["pimax"],
                              npibins=jb["npibins"], periodic=True, box=jb["box"])[0]
        assert np.array_equal(r.npairs, ref), jb["j"]
    b.close()


def test_batch_cross_open_and_many_job_switches(cuda_device):
    b = cf.Batch()
    cases = []
    for k in range(40):  # many tiny jobs: every CTA switches job many times
        a = synth.neyman_scott(30 + k, 10.0, 2.0, 120.0, seed=200 + k)
        u = synth.uniform_box(800 + 10 * k, 120.0, seed=300 + k)
        job = dict(kind="xi" if k % 2 == 0 else "rppi", mode="fp64" if k % 3 == 0 else "fp32_recheck",
                   box=120.0, periodic=(k % 4 != 1), edges=synth.log_edges(0.2, 15.0, 10),
                   pimax=12.0, npibins=12)
        xa, xu = dev(a), dev(u)
        cases.append((job, xa, xu, add(b, job, xa, xu)))
    b.run(use_graph=True)
    for job, xa, xu, r in cases:
        assert np.array_equal(r.npairs, single(job, xa, xu))
    b.close()


def test_graph_replay_sees_in_place_updates_and_open_box_replans(cuda_device):
    import torch
    p = synth.neyman_scott(400, 20.0, 2.0, 150.0, seed=401)
    o = synth.uniform_box(20000, 150.0, seed=402)
    e = synth.log_edges(0.1, 20.0, 12)
    xp, xo = dev(p), dev(o)
    b = cf.Batch()
    rp = b.add_xi(*xp, e, boxsize=150.0)
    ro = b.add_rp_pi(*xo, e, 15.0, 15, periodic=False)
    b.run(use_graph=True)
    # periodic job: new positions of the same size, replay without re-planning
    q = synth.neyman_scott(400, 20.0, 2.0, 150.0, seed=403)
    n = min(p.n, q.n)
    for t, v in zip(xp, (q.x, q.y, q.z)):
        t[:n] = torch.from_numpy(v[:n]).cuda()
    s = b.run(use_graph=True)
    assert s["planned"] == 0
    assert np.array_equal(rp.npairs, cf.countpairs_xi(*xp, e, boxsize=150.0).npairs)
    # open job: points moved outside the planned bounding box -> re-plan and recapture
    xo[0].mul_(1.5)
    s = b.run(use_graph=True)
    assert s["planned"] == 1
    assert np.array_equal(ro.npairs, cf.countpairs_rp_pi(*xo, e, 15.0, 15, periodic=False).npairs)
    b.close()


def test_batch_rejects_host_inputs_and_empty_runs(cuda_device):
    c = synth.uniform_box(100, 10.0, seed=404)
    b = cf.Batch()
    with pytest.raises(cf.CfError) as ei:
        b.add_xi(c.x, c.y, c.z, [0.1, 1.0], boxsize=10.0)
    assert ei.value.status == cf.CF_EINVAL
    with pytest.raises(cf.CfError):
        b.run()
    b.close()


def test_batch_autotune_tunes_at_plan_time_and_forced_shapes_are_exact(cuda_device, tmp_path):
    import json
    cf.tune_clear()
    jobs = []
    for k, (n_par, box) in enumerate(((150, 80.0), (600, 120.0), (2400, 200.0), (9000, 300.0))):
        jobs.append(dict(kind="xi", mode="fp32_recheck", box=box,
                         edges=synth.log_edges(0.1, 12.0 + 3 * k, 12),
                         cat=synth.neyman_scott(n_par, 20.0, 2.0, box, seed=420 + k)))
    jobs.append(dict(kind="rppi", mode="fp32_recheck", box=150.0, edges=synth.log_edges(0.2, 10.0, 8),
                     pimax=10.0, npibins=10, cat=synth.uniform_box(20000, 150.0, seed=430)))
    jobs.append(dict(kind="xi", mode="fp64", box=100.0, edges=synth.log_edges(0.2, 10.0, 8),
                     cat=synth.uniform_box(8000, 100.0, seed=431)))
    xyz = [dev(jb["cat"]) for jb in jobs]

    def run_batch():
        b = cf.Batch()
        res = []
        for jb, x in zip(jobs, xyz):
            kw = dict(boxsize=jb["box"], mode=jb["mode"], autotune=True)
            if jb["kind"] == "xi":
                res.append(b.add_xi(*x, jb["edges"], **kw))
            else:
                res.append(b.add_rp_pi(*x, jb["edges"], jb["pimax"], jb["npibins"], **kw))
        b.run(use_graph=True)
        for jb, x, r in zip(jobs, xyz, res):
            assert np.array_equal(r.npairs, single(jb, x))
        b.close()
        return res

    # first batch: every signature is tuned while the batch is planned
    first = run_batch()
    assert cf.tune_count() >= 4
    assert all(r.refine_used[0] in (1, 2, 3, 4) for r in first)
    # force each float32 DD(r) kernel shape through the tuning cache file
    path = str(tmp_path / "tune.json")
    cf.tune_save(path)
    with open(path) as f:
        cache = json.load(f)
    shapes = [(16, 2), (8, 2), (16, 1), (32, 1)]
    forced = {}
    for i, entry in enumerate(e for e in cache["entries"] if e["key"].startswith("k0 m1")):
        entry["chunk"], entry["pp"] = shapes[i % 4]
        forced[entry["key"]] = shapes[i % 4]
    with open(path, "w") as f:
        json.dump(cache, f)
    cf.tune_clear()
    cf.tune_load(path)
    second = run_batch()
    used = {(r.chunk_used, r.pp_used) for jb, r in zip(jobs, second)
            if jb["kind"] == "xi" and jb["mode"] == "fp32_recheck"}
    assert len(used) == min(4, len(forced)) and all(r.tuned == 2 for r in second)
    cf.tune_clear()


def test_batch_mixed_dtypes_empty_catalogues_and_many_segments(cuda_device):
    # 120 jobs gridded together: float32 and float64 inputs side by side, empty
    # catalogues (auto and as the secondary of a cross job), sizes from 0 to
    # 2000, clustered and uniform, DD(r) and DD(rp, pi), both modes
    b = cf.Batch()
    cases = []
    for k in range(120):
        n = [0, 1, 5, 37, 300, 2000][k % 6]
        c = synth.uniform_box(n, 100.0, seed=600 + k)
        if k % 5 == 4:
            c = synth.neyman_scott(max(n // 20, 1), 20.0, 2.0, 100.0, seed=600 + k)
        dtype = np.float32 if k % 3 == 0 else np.float64
        c = c.astype(dtype)
        c2 = None
        if k % 4 == 3:
            c2 = synth.uniform_box([0, 17, 900][k % 3], 100.0, seed=900 + k).astype(dtype)
        job = dict(kind="xi" if k % 2 == 0 else "rppi", mode="fp64" if k % 7 == 0 else "fp32_recheck",
                   box=100.0, periodic=(k % 8 != 5), edges=synth.log_edges(0.3, 12.0, 9),
                   pimax=10.0, npibins=10)
        x = dev(c)
        x2 = dev(c2) if c2 is not None else None
        cases.append((k, job, x, x2, add(b, job, x, x2)))
    for use_graph in (False, True):
        stats = b.run(use_graph=use_graph)
        assert stats["n_jobs"] == 120
        for k, job, x, x2, r in cases:
            assert np.array_equal(r.npairs, single(job, x, x2)), k
    b.close()


def test_batch_reports_a_coordinate_outside_the_box_by_job(cuda_device):
    # the batched gridding checks every segment's coordinates and flags the
    # job that owns a bad one (periodic: x must lie in [0, boxsize))
    good = synth.uniform_box(500, 50.0, seed=501)
    bad = synth.uniform_box(500, 50.0, seed=502)
    bad.x[17] = 50.0
    e = synth.log_edges(0.5, 10.0, 6)
    b = cf.Batch()
    b.add_xi(*dev(good), e, boxsize=50.0)
    b.add_xi(*dev(bad), e, boxsize=50.0)
    with pytest.raises(cf.CfError) as ei:
        b.run(use_graph=False)
    assert ei.value.status == cf.CF_EINVAL and "batch job 1" in str(ei.value)
    b.close()
