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
}


def make(name):
    spec = CASES[name]
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
