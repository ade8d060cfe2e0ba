"""Write the stored expected histograms for the full-size parity tests.

Every value in ``tests/golden/*.json`` is produced by this script, which calls
only the CPU oracle (``oracle/``) on catalogues from the seeded generator
(``paper_1911_08275_gb300/synth.py``).  Each file records the catalogue's
digest, so a test can tell a changed input from a wrong count.

Usage:  python tests/golden/make_golden.py [name ...]     (default: all)

The brute-force oracle needs ~7e11 pair evaluations per 1.2M-point
auto-correlation, i.e. minutes per file on a multi-core host.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1911_08275_gb300 import synth  # noqa: E402


def c2(dtype):
    c = synth.c2_clustered()
    return c if dtype == "f64" else c.astype(np.float32)


CASES = {
    # Neyman-Scott stand-in for the paper's 1.2M-galaxy periodic box of side 420
    # (Sec. 3); 20 log bins 0.1 -> Rmax; xi(r) auto-correlation.
    "c2_xi_r25_f64": dict(kind="xi", cat=("c2", "f64"), rmin=0.1, rmax=25.0, nbins=20),
    "c2_xi_r10_f64": dict(kind="xi", cat=("c2", "f64"), rmin=0.1, rmax=10.0, nbins=20),
    "c2_xi_r50_f64": dict(kind="xi", cat=("c2", "f64"), rmin=0.1, rmax=50.0, nbins=20),
    "c2_xi_r25_f32": dict(kind="xi", cat=("c2", "f32"), rmin=0.1, rmax=25.0, nbins=20),
    # DD(rp, pi): 14 log rp bins 0.1 -> 25, pimax 40 in 40 unit bins, LOS = z.
    "c3_rppi_f32": dict(kind="rppi", cat=("c2", "f32"), rmin=0.1, rmax=25.0, nbins=14,
                        pimax=40.0, npibins=40),
    "c3_rppi_f64": dict(kind="rppi", cat=("c2", "f64"), rmin=0.1, rmax=25.0, nbins=14,
                        pimax=40.0, npibins=40),
    # DR with weights and ravg, open box: a slice of the weighted data (the first
    # 8000 points of the clustered catalogue, weights U(0.5,1.5) seed 4) against
    # all 12M weighted randoms (seed 3, weights seed 5); 20 log bins 0.1 -> 25.
    "c4_dr_slice8000_f64": dict(kind="dr", rows=8000, rmin=0.1, rmax=25.0, nbins=20),
}


def c4():
    d = synth.c2_clustered()
    d.w = synth.uniform_weights(d.n, 0.5, 1.5, seed=4)
    r = synth.c4_randoms()
    r.w = synth.uniform_weights(r.n, 0.5, 1.5, seed=5)
    return d, r


def make_dr(name, spec):
    d, r = c4()
    rows = spec["rows"]
    ds = d.take(np.arange(rows))
    edges = synth.log_edges(spec["rmin"], spec["rmax"], spec["nbins"])
    t0 = time.time()
    n, ws, rs = oracle.xi(ds.x, ds.y, ds.z, w1=ds.w, x2=r.x, y2=r.y, z2=r.z, w2=r.w, edges=edges,
                          autocorr=False, periodic=False, want_r=True)
    out = {
        "name": name,
        "source": "tests/golden/make_golden.py -> oracle (brute force, canonical binary64)",
        "workload": spec,
        "catalog": f"{d.name} weights seed 4, first {rows} points",
        "catalog_digest": ds.digest(),
        "randoms": f"{r.name} weights seed 5",
        "randoms_digest": r.digest(),
        "n": ds.n,
        "n_randoms": r.n,
        "edges_hex": [float(e).hex() for e in edges],
        "npairs": [int(v) for v in n],
        "wsum_hex": [float(v).hex() for v in ws],
        "rsum_hex": [float(v).hex() for v in rs],
        "oracle_seconds": round(time.time() - t0, 1),
        "oracle_threads": oracle.num_threads(),
    }
    with open(os.path.join(HERE, name + ".json"), "w") as f:
        json.dump(out, f, indent=1)
    print(name, "done in", out["oracle_seconds"], "s", flush=True)


def make(name):
    spec = CASES[name]
    if spec["kind"] == "dr":
        return make_dr(name, spec)
    cat = c2(spec["cat"][1])
    edges = synth.log_edges(spec["rmin"], spec["rmax"], spec["nbins"])
    t0 = time.time()
    if spec["kind"] == "xi":
        n, _, _ = oracle.xi(cat.x, cat.y, cat.z, edges=edges, periodic=True, box=synth.BOX)
        counts = [int(v) for v in n]
    else:
        n, _, _ = oracle.rppi(cat.x, cat.y, cat.z, rp_edges=edges, pimax=spec["pimax"],
                              npibins=spec["npibins"], periodic=True, box=synth.BOX)
        counts = [[int(v) for v in row] for row in n]
    out = {
        "name": name,
        "source": "tests/golden/make_golden.py -> oracle (brute force, canonical binary64)",
        "workload": spec,
        "catalog": cat.name,
        "catalog_digest": cat.digest(),
        "n": cat.n,
        "box": synth.BOX,
        "edges_hex": [float(e).hex() for e in edges],
        "npairs": counts,
        "oracle_seconds": round(time.time() - t0, 1),
        "oracle_threads": oracle.num_threads(),
    }
    with open(os.path.join(HERE, name + ".json"), "w") as f:
        json.dump(out, f, indent=1)
    print(name, "done in", out["oracle_seconds"], "s", flush=True)


if __name__ == "__main__":
    for nm in (sys.argv[1:] or list(CASES)):
        make(nm)
