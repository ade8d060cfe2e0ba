"""Benchmark: DD(r) Gpairs/s at N = 1.2M, Rmax = 25 on one GB300 per rank.

Workload: the 1.2M-point Neyman-Scott catalogue in a periodic box of side 420
(60,000 parents, Poisson(20) children, sigma 2; a stand-in for the paper's
1.2M-galaxy box of Sec. 3), float64 positions, 20 log bins from 0.1 to 25,
auto-correlation, FP32 distances with binary64 re-check (exact counts).

A step is one cf_countpairs_xi call: gridding, column-pair pruning, the pair
kernel, the histogram merge and its copy to the host.  Gpairs/s counts the
ordered pairs the histogram holds (P_cnt) per second.

  value  device-resident inputs; CUDA events around each call on its stream;
         L2 flushed (a 256 MiB write) between steps, outside the timed region.
  e2e    same call with page-locked HOST inputs: the H2D copy of x, y, z and
         the D2H of the histogram happen inside the timed call.
  roofline  the pair kernel's pair evaluations (diagnostic counter, separate
         run) x 7 FP32 instructions each, over its event-timed duration,
         against SMs x 128 lanes x max SM clock; traffic = DRAM bytes per launch
         from the committed ncu summary while the kernel sources are unchanged.
  other_workloads  a few calls each of DD(r) at Rmax 10 and 50, DD(rp, pi)
         14 x 40, the weighted DR count with ravg (1.2M x 12M, open box), and the
         48-job batched launch (graph replay vs 48 single calls).

cpu_baseline is the plain gridded CPU counter (oracle/gridded.c: cell lists of
Sec. 1.2 / 2.1 / 2.2 with refine (2, 2, 1), scalar canonical binary64, OpenMP
on all host cores, counts equal to the oracle's bit for bit) on the whole
workload; cpu_oracle is the brute-force oracle on a slice of primary points.
--impl reference times the gridded CPU counter on the whole workload each step
(the oracle is the brute-force definition; the gridded counter is the paper's
method on the CPU, pinned to it).

Multi-GPU (torchrun): each rank counts its own replica (independent problems,
no collective on the data path); value = total pairs over the max time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "DD(r) Gpairs/s at N=1.2M, Rmax=25 (FP32+recheck vs FP64, exact counts)"
UNIT = "Gpairs/s"
RMIN, RMAX, NBINS = 0.1, 25.0, 20
INSTR_PER_EVAL = 7  # 3 FADD, FMUL + 2 FFMA, 1 compare per evaluated pair


def workload_config(n):
    return {"workload": "xi_auto_neyman_scott_1.2M_box420_rmax25", "n_points": int(n),
            "box": 420.0, "rmax": RMAX, "nbins": NBINS, "edges": "log 0.1-25", "periodic": True,
            "input_dtype": "float64", "l2": "flushed between steps (256 MiB write)"}


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = []
        for line in open(self.path):
            f = [v.strip() for v in line.split(",")]
            if len(f) >= 9 and f[1].replace(".", "").isdigit():
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None,
                "samples": len(rows), "reasons": reasons}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"sm_max_mhz": 2070.0}, "fallback"


PROFILE = os.path.join(ROOT, "profiles", "k_xi32_xi_auto_1.2M_rmax25.md")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1911_08275_gb300", "csrc", f)
                  for f in ("pairs.cu", "cf_internal.cuh")]


def profile_traffic():
    """DRAM bytes per launch of the pair kernel from the committed ncu summary,
    or None when the kernel sources changed since that capture."""
    import hashlib
    if not os.path.exists(PROFILE):
        return None, "no profile"
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    fields = {}
    for line in open(PROFILE):
        if ":" in line and line.split(":")[0].strip() in ("kernel_source_sha256_16",
                                                          "traffic_bytes_per_launch"):
            k, v = line.split(":", 1)
            fields[k.strip()] = v.split()[0]
    if fields.get("kernel_source_sha256_16") != h.hexdigest()[:16]:
        return None, "kernel changed since the ncu capture"
    return int(fields["traffic_bytes_per_launch"]), "ncu capture " + os.path.basename(PROFILE)


def counts_equal_oracle(name, cat, npairs):
    """Counts against the brute-force oracle's stored histogram of the same
    catalogue (tests/golden/<name>.json, written by tests/golden/make_golden.py,
    which calls only the oracle); None when the file or its catalogue digest
    does not match."""
    path = os.path.join(ROOT, "tests", "golden", name + ".json")
    try:
        with open(path) as f:
            g = json.load(f)
    except OSError:
        return None
    if g.get("catalog_digest") != cat.digest():
        return None
    return bool(np.array_equal(np.asarray(g["npairs"], dtype=np.uint64).ravel(),
                               np.asarray(npairs, dtype=np.uint64).ravel()))


def cpu_baseline_sample(cat, edges, rows, reps=1):
    """Time the oracle on primary rows [0, rows) against the whole catalogue."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    cnt = 0
    for _ in range(reps):
        n, _, _ = oracle.xi(cat.x[:rows], cat.y[:rows], cat.z[:rows], x2=cat.x, y2=cat.y,
                            z2=cat.z, edges=edges, autocorr=False, periodic=True, box=cat.box)
        cnt += int(n.sum())
    dt = time.perf_counter() - t0
    return cnt, dt, oracle.num_threads()


def gridded_run(cat, edges):
    """One gridded CPU count of the whole workload: (pairs, seconds, threads)."""
    import oracle
    oracle.build_gridded()
    t0 = time.perf_counter()
    n = oracle.gridded_xi(cat.x, cat.y, cat.z, edges=edges, periodic=True, box=cat.box)
    dt = time.perf_counter() - t0
    return n, dt, oracle.gridded_num_threads()


GRIDDED_SAMPLE = ("whole workload per step: plain gridded CPU count (oracle/gridded.c: cell "
                  "lists, refine (2,2,1), scalar canonical binary64, OpenMP)")


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1911_08275_gb300 import synth
    cat = synth.c2_clustered()
    edges = synth.log_edges(RMIN, RMAX, NBINS)
    small = cat.take(np.arange(min(cat.n, 100000)))
    for _ in range(args.warmup):
        gridded_run(small, edges)
    times, counts, cores = [], [], 1
    counts_last = None
    for _ in range(args.steps):
        n, dt, cores = gridded_run(cat, edges)
        times.append(dt)
        counts.append(int(n.sum()))
        counts_last = n
    if len(set(counts)) != 1:
        raise RuntimeError("gridded CPU counts changed between steps")
    value = sum(counts) / sum(times) / 1e9
    rows = int(os.environ.get("CF_REF_ROWS", "2000"))
    oc, odt, ocores = cpu_baseline_sample(cat, edges, rows)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": workload_config(cat.n), "p_cnt": counts[0],
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "gridded",
                            "sample": GRIDDED_SAMPLE,
                            "counts_equal_oracle": counts_equal_oracle("c2_xi_r25_f64", cat,
                                                                       counts_last)},
           "cpu_oracle": {"value": oc / odt / 1e9, "unit": UNIT, "cores": ocores, "kind": "oracle",
                          "sample": f"brute force, {rows} primary points x all {cat.n} points "
                                    f"({rows * cat.n:.3g} pair evaluations, {odt:.1f} s)"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def _median_call(fn, flush, reps=3):
    """Median library-reported device time (ms) of reps calls, L2 flushed before each."""
    res = []
    for _ in range(reps):
        flush.zero_()
        res.append(fn())
    ms = statistics.median(r.total_ms for r in res)
    kms = statistics.median(r.kernel_ms for r in res)
    return res[-1], ms, kms


def _timed_row(cf, fn, flush, peak_evals, fp32=True, golden=None):
    """One secondary workload: evaluation count (a separate run with
    CF_FLAG_COUNT_EVALS), then the median of three timed calls; the roofline
    fraction of the pair kernel is evaluations / kernel time / R1 (the same
    7-instructions-per-evaluation roofline as the headline)."""
    diag = fn(cf.CF_FLAG_COUNT_EVALS)
    r, ms, kms = _median_call(lambda: fn(0), flush)
    if not np.array_equal(r.npairs, diag.npairs):
        raise RuntimeError("counts differ between the counting and the timed runs")
    row = {"ms": ms, "kernel_ms": kms, "Gpairs_s": float(r.npairs.sum()) / (ms * 1e-3) / 1e9,
           "evaluations": int(diag.n_evaluated), "refine": list(r.refine_used)}
    if golden is not None:
        row["counts_equal_oracle"] = counts_equal_oracle(golden[0], golden[1], r.npairs)
    if fp32:
        achieved = diag.n_evaluated / (kms * 1e-3) / 1e9
        row["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak_evals,
                           "unit": "Gevals/s", "frac": achieved / peak_evals}
    return row


def other_workloads(cf, synth, torch, cat, xyz, dev, stream, flush, peak_evals):
    """Secondary measurements (a few calls each; not the headline)."""
    out = {}
    st = stream.cuda_stream
    for rmax in (10.0, 50.0):
        e = synth.log_edges(RMIN, rmax, NBINS)
        row = {}
        for mode in ("fp32_recheck", "fp64"):
            row[mode] = _timed_row(cf, lambda fl: cf.countpairs_xi(*xyz, e, boxsize=synth.BOX,
                                                                   mode=mode, flags=fl, stream=st),
                                   flush, peak_evals, mode == "fp32_recheck",
                                   golden=(f"c2_xi_r{rmax:g}_f64", cat))
        out[f"xi_auto_rmax{rmax:g}"] = row
    e = synth.log_edges(RMIN, RMAX, 14)
    row = {}
    for mode in ("fp32_recheck", "fp64"):
        row[mode] = _timed_row(cf, lambda fl: cf.countpairs_rp_pi(*xyz, e, 40.0, 40, boxsize=synth.BOX,
                                                                  mode=mode, flags=fl, stream=st),
                               flush, peak_evals, mode == "fp32_recheck", golden=("c3_rppi_f64", cat))
    out["rppi_auto_14x40_pimax40"] = row
    # weighted DR with ravg: 1.2M clustered data x 12M uniform randoms, open box
    wd = synth.uniform_weights(cat.n, 0.5, 1.5, seed=4)
    rnd = synth.c4_randoms()
    wr = synth.uniform_weights(rnd.n, 0.5, 1.5, seed=5)
    a_w = torch.from_numpy(wd).to(dev)
    b = [torch.from_numpy(v).to(dev) for v in (rnd.x, rnd.y, rnd.z, wr)]
    ed = synth.log_edges(RMIN, RMAX, NBINS)
    out["dr_weighted_ravg_1.2Mx12M_open"] = {"fp32_recheck": _timed_row(
        cf, lambda fl: cf.countpairs_xi(*xyz, ed, w=a_w, x2=b[0], y2=b[1], z2=b[2], w2=b[3],
                                        periodic=False, mode="fp32_recheck", want_ravg=True,
                                        flags=fl, stream=st), flush, peak_evals)}
    out["dr_weighted_1.2Mx12M_open"] = {"fp32_recheck": _timed_row(
        cf, lambda fl: cf.countpairs_xi(*xyz, ed, w=a_w, x2=b[0], y2=b[1], z2=b[2], w2=b[3],
                                        periodic=False, mode="fp32_recheck", flags=fl,
                                        stream=st), flush, peak_evals)}
    del b, a_w
    out["batch_48_jobs"] = batch_workload(cf, synth, torch, dev, flush)
    return out


def _batch(cf, jobs, xyz, autotune):
    b = cf.Batch()
    res = []
    for jb, x in zip(jobs, xyz):
        kw = dict(boxsize=jb["box"], mode=jb["mode"], autotune=autotune)
        if jb["kind"] == "xi":
            res.append(b.add_xi(*x, jb["edges"], **kw))
        else:
            res.append(b.add_rp_pi(*x, jb["edges"], jb["pimax"], jb["npibins"], **kw))
    return b, res


def _time_batch(b, flush, reps=3, use_graph=True):
    runs = []
    for _ in range(reps):
        flush.zero_()
        runs.append(b.run(use_graph=use_graph))
    return statistics.median(r["total_ms"] for r in runs), runs[-1]


def batch_workload(cf, synth, torch, dev, flush):
    """48 independent DD(r) / DD(rp, pi) jobs (synth.batch_job) in one batched
    persistent launch replayed from a CUDA graph, each job with the tuner's
    refinement and float32 DD(r) kernel shape for its signature (tuned while the
    first run plans the batch), against the same jobs as 48 single calls
    (per-job counts must be identical); the float32 and the binary64 jobs as
    batches of their own; and 480 small jobs (launch-bound: every gridding
    stage and the work lists of all jobs run as one launch each) with and
    without the graph, and as 480 single calls."""
    jobs = [synth.batch_job(j) for j in range(48)]
    xyz = [[torch.from_numpy(v).to(dev) for v in (jb["cat"].x, jb["cat"].y, jb["cat"].z)]
           for jb in jobs]
    b, res = _batch(cf, jobs, xyz, autotune=True)
    t0 = time.perf_counter()
    first = b.run(use_graph=True)  # plan (tuning every new signature) + capture
    first_wall_s = time.perf_counter() - t0
    ms, last = _time_batch(b, flush)
    direct_ms, direct = _time_batch(b, flush, reps=2, use_graph=False)
    single_ms, exact = 0.0, 0
    for jb, x, r in zip(jobs, xyz, res):
        flush.zero_()
        kw = dict(boxsize=jb["box"], mode=jb["mode"], autotune=True)
        if jb["kind"] == "xi":
            sc = cf.countpairs_xi(*x, jb["edges"], **kw)
        else:
            sc = cf.countpairs_rp_pi(*x, jb["edges"], jb["pimax"], jb["npibins"], **kw)
        single_ms += sc.total_ms
        exact += int(np.array_equal(sc.npairs, r.npairs))
    pairs = last["pairs"]
    shapes = {}
    for jb, r in zip(jobs, res):
        key = f"{jb['kind']} {jb['mode']} refine {r.refine_used[0]}" + (
            f" shape {r.chunk_used}x{r.pp_used}" if jb["kind"] == "xi" and jb["mode"] == "fp32_recheck"
            else "")
        shapes[key] = shapes.get(key, 0) + 1
    out = {"jobs": 48, "points": int(sum(jb["cat"].n for jb in jobs)), "pairs": int(pairs),
           "ms": ms, "kernel_ms": direct["kernel_ms"], "ms_without_graph": direct_ms,
           "Gpairs_s": pairs / (ms * 1e-3) / 1e9, "graph": True,
           "kernels_per_run": int(last["n_kernels"]), "blocks": int(last["blocks"]),
           "first_run_wall_s_plan_tune_capture": first_wall_s,
           "tuned_choices": shapes,
           "single_calls_ms": single_ms, "single_calls_Gpairs_s": pairs / (single_ms * 1e-3) / 1e9,
           "jobs_exact_vs_single_calls": exact}
    b.close()
    # per mode: the float32 + re-check jobs and the binary64 jobs as batches of their own
    for mode in ("fp32_recheck", "fp64"):
        sel = [k for k, jb in enumerate(jobs) if jb["mode"] == mode]
        bm, rm = _batch(cf, [jobs[k] for k in sel], [xyz[k] for k in sel], autotune=True)
        bm.run(use_graph=True)
        mms, ml = _time_batch(bm, flush)
        out[f"by_mode_{mode}"] = {"jobs": len(sel), "pairs": int(ml["pairs"]), "ms": mms,
                                  "Gpairs_s": ml["pairs"] / (mms * 1e-3) / 1e9}
        bm.close()
    del xyz
    # launch-bound: 480 small jobs (about 2,000-8,000 points each), graph vs direct issue
    small = [synth.batch_job(j % 48, scale=0.004) for j in range(480)]
    sx = [[torch.from_numpy(v).to(dev) for v in (jb["cat"].x, jb["cat"].y, jb["cat"].z)]
          for jb in small]
    bs, sres = _batch(cf, small, sx, autotune=False)
    bs.run(use_graph=True)
    g_ms, gl = _time_batch(bs, flush)
    d_ms, _ = _time_batch(bs, flush, use_graph=False)
    # the same jobs as 480 single calls (each call's own device time, summed)
    s_ms, s_kernels, s_exact = 0.0, 0, 0
    for jb, x, r in zip(small, sx, sres):
        kw = dict(boxsize=jb["box"], mode=jb["mode"])
        if jb["kind"] == "xi":
            sc = cf.countpairs_xi(*x, jb["edges"], **kw)
        else:
            sc = cf.countpairs_rp_pi(*x, jb["edges"], jb["pimax"], jb["npibins"], **kw)
        s_ms += sc.total_ms
        s_kernels += sc.n_kernels
        s_exact += int(np.array_equal(sc.npairs, r.npairs))
    out["small_480_jobs"] = {"jobs": 480, "points": int(sum(jb["cat"].n for jb in small)),
                             "pairs": int(gl["pairs"]), "kernels_per_run": int(gl["n_kernels"]),
                             "ms_graph": g_ms, "ms_without_graph": d_ms,
                             "graph_gain": d_ms / g_ms,
                             "single_calls_ms": s_ms, "single_calls_kernels": s_kernels,
                             "batch_gain_vs_single_calls": s_ms / g_ms,
                             "jobs_exact_vs_single_calls": s_exact}
    bs.close()
    return out


def run_profile_case(args):
    """A few calls of one workload for an ncu capture (no L2 flush, no JSON line):
    xi (C2, Rmax 25), xi64 (the same in binary64), rppi (C2, 14 x 40, pimax 40),
    dr_small (the C2 data, weighted, against the first 1.2M weighted randoms, open
    box, with ravg), batch_small (the 480 small jobs of the batch workload, one run
    per step without the graph, so every launch is visible)."""
    import torch
    import paper_1911_08275_gb300 as cf
    from paper_1911_08275_gb300 import synth
    cf.lib()
    dev = torch.device("cuda", 0)
    if args.profile == "batch_small":
        small = [synth.batch_job(j % 48, scale=0.004) for j in range(480)]
        sx = [[torch.from_numpy(v).to(dev) for v in (jb["cat"].x, jb["cat"].y, jb["cat"].z)]
              for jb in small]
        b, _ = _batch(cf, small, sx, autotune=False)
        runs = [b.run(use_graph=False) for _ in range(args.steps)]
        b.close()
        print(f"profile case batch_small: run ms {[round(r['total_ms'], 3) for r in runs]}, "
              f"pair kernel ms {[round(r['kernel_ms'], 3) for r in runs]}", flush=True)
        return
    cat = synth.c2_clustered()
    xyz = [torch.from_numpy(v).to(dev) for v in (cat.x, cat.y, cat.z)]
    e = synth.log_edges(RMIN, RMAX, NBINS)
    if args.profile == "dr_small":
        wd = torch.from_numpy(synth.uniform_weights(cat.n, 0.5, 1.5, seed=4)).to(dev)
        rnd = synth.c4_randoms().take(np.arange(1200000))
        wr = synth.uniform_weights(12000000, 0.5, 1.5, seed=5)[:1200000]
        b = [torch.from_numpy(np.ascontiguousarray(v)).to(dev) for v in (rnd.x, rnd.y, rnd.z, wr)]
    ms = []
    for _ in range(args.steps):
        if args.profile == "xi":
            r = cf.countpairs_xi(*xyz, e, boxsize=synth.BOX)
        elif args.profile == "xi64":
            r = cf.countpairs_xi(*xyz, e, boxsize=synth.BOX, mode="fp64")
        elif args.profile == "rppi":
            r = cf.countpairs_rp_pi(*xyz, synth.log_edges(RMIN, RMAX, 14), 40.0, 40, boxsize=synth.BOX)
        else:
            r = cf.countpairs_xi(*xyz, e, w=wd, x2=b[0], y2=b[1], z2=b[2], w2=b[3], periodic=False,
                                 want_ravg=True)
        ms.append(round(r.kernel_ms, 4))
    torch.cuda.synchronize()
    print(f"profile case {args.profile}: kernel_ms {ms}, pairs {int(r.npairs.sum())}", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="fp32_recheck", choices=["fp32_recheck", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the secondary workloads (Rmax sweep, DD(rp,pi), weighted DR)")
    ap.add_argument("--profile", choices=["xi", "xi64", "rppi", "dr_small", "batch_small"],
                    help="run --steps calls of one workload for a profiler capture, then exit")
    args = ap.parse_args()
    if args.profile:
        return run_profile_case(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_1911_08275_gb300 as cf
    from paper_1911_08275_gb300 import synth

    cf.lib()
    cat = synth.c2_clustered()
    edges = synth.log_edges(RMIN, RMAX, NBINS)
    dev = torch.device("cuda", local)
    xyz = [torch.from_numpy(v).to(dev) for v in (cat.x, cat.y, cat.z)]
    host = [torch.from_numpy(v).pin_memory() for v in (cat.x, cat.y, cat.z)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def call(inputs, flags=0, mode=args.mode):
        return cf.countpairs_xi(*inputs, edges, boxsize=synth.BOX, mode=mode, flags=flags,
                                stream=stream.cuda_stream)

    diag = call(xyz, flags=cf.CF_FLAG_COUNT_EVALS)  # evaluation count (separate, untimed)
    p_cnt = int(diag.npairs.sum())
    for _ in range(args.warmup):
        call(xyz)
        call(host)

    launches = [0]

    def timed(inputs):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        kms, tms = [], []
        launches[0] = 0
        for s in range(args.steps):
            flush.zero_()
            ev[s][0].record(stream)
            r = call(inputs)
            ev[s][1].record(stream)
            kms.append(r.kernel_ms)
            tms.append(r.total_ms)
            launches[0] += r.n_kernels
            if int(r.npairs.sum()) != p_cnt:
                raise RuntimeError("counts changed between steps")
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev], kms, tms

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        step_ms, kernel_ms, lib_ms = timed(xyz)
    n_launches = launches[0]
    e2e_ms, _, _ = timed(host)
    torch.cuda.synchronize()
    t_mean = statistics.mean(step_ms)
    e_mean = statistics.mean(e2e_ms)
    if dist:
        tt = torch.tensor([t_mean, e_mean], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_mean, e_mean = float(tt[0]), float(tt[1])
        dist.barrier()
    value = world * p_cnt / (t_mean * 1e-3) / 1e9
    e2e_value = world * p_cnt / (e_mean * 1e-3) / 1e9

    peaks, peak_src = load_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fmax = float(peaks.get("sm_max_mhz", 2070.0))
    peak_evals = sms * 128 * fmax * 1e6 / INSTR_PER_EVAL / 1e9  # Gevals/s
    k_mean = statistics.mean(kernel_ms)
    achieved = diag.n_evaluated / (k_mean * 1e-3) / 1e9
    traffic, traffic_src = profile_traffic()
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_evals, "unit": "Gevals/s",
                "frac": achieved / peak_evals, "traffic": traffic, "traffic_source": traffic_src,
                "peak_note": f"{sms} SMs x 128 FP32 lanes x {fmax:.0f} MHz / {INSTR_PER_EVAL} "
                             f"instr per evaluated pair ({peak_src} max SM clock)",
                "kernel_ms": k_mean, "evaluations": diag.n_evaluated,
                "library_call_ms": statistics.mean(lib_ms)}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_mean, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64recheck" if args.mode ==
           "fp32_recheck" else "f64", "data": "synthetic", "config": workload_config(cat.n),
           "p_cnt": p_cnt, "counts_equal_oracle": counts_equal_oracle("c2_xi_r25_f64", cat,
                                                                      diag.npairs),
           "clocks": clk.summary(), "roofline": roofline,
           "e2e": {"value": e2e_value, "unit": UNIT, "ms_per_step": e_mean,
                   "h2d_bytes_per_step": int(3 * 8 * cat.n),
                   "d2h_bytes_per_step": int(8 * NBINS + 8 * 4 + 4)},
           "gpu_launches": n_launches,
           "diag": {"n_cellpairs": diag.n_cellpairs, "n_rechecked": diag.n_rechecked,
                    "useful_fraction": p_cnt / 2 / max(1, diag.n_evaluated)}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        gridded_run(cat.take(np.arange(min(cat.n, 100000))), edges)  # build, warm caches
        gn, gdt, gcores = gridded_run(cat, edges)
        out["cpu_baseline"] = {"value": float(gn.sum()) / gdt / 1e9, "unit": UNIT, "cores": gcores,
                               "kind": "gridded", "sample": GRIDDED_SAMPLE + f" ({gdt:.2f} s)",
                               "counts_equal_gpu": bool(np.array_equal(gn, diag.npairs))}
        rows = int(os.environ.get("CF_CPU_ROWS", "40000"))
        c, dt, cores = cpu_baseline_sample(cat, edges, rows)
        out["cpu_oracle"] = {"value": c / dt / 1e9, "unit": UNIT, "cores": cores,
                             "kind": "oracle",
                             "sample": f"brute force, {rows} primary points x all {cat.n} points "
                                       f"({rows * cat.n:.3g} pair evaluations, {dt:.1f} s)"}
    if args.mode == "fp32_recheck" and rank == 0:
        # the plain binary64 path on the same workload, for the FP32/FP64 ratio
        r64 = [call(xyz, mode="fp64") for _ in range(3)]
        assert all(np.array_equal(r.npairs, diag.npairs) for r in r64)
        out["fp64_path"] = {"ms_per_step": statistics.median(r.total_ms for r in r64),
                            "kernel_ms": statistics.median(r.kernel_ms for r in r64)}
        out["fp64_path"]["value"] = p_cnt / (out["fp64_path"]["ms_per_step"] * 1e-3) / 1e9
        out["fp32_over_fp64"] = out["fp64_path"]["ms_per_step"] / t_mean
    if rank == 0 and world == 1 and not args.no_extra:
        out["other_workloads"] = other_workloads(cf, synth, torch, cat, xyz, dev, stream, flush,
                                                 peak_evals)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
