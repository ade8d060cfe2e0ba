"""Full-size parity: the 1.2M-point clustered catalogue in the bench's launch
configuration, against stored brute-force oracle histograms.

``tests/golden/*.json`` is written by ``tests/golden/make_golden.py``, which
calls only the CPU oracle; each file records the digest of the catalogue it was
computed on, checked here before comparing counts bin by bin (bit-exact).
Properties that hold at any size complete the check: auto == cross(D, D) for
e_0 > 0, float32+re-check == binary64, invariance under a permutation.
"""
import glob
import json
import os

import numpy as np
import pytest

import paper_1911_08275_gb300 as cf
from paper_1911_08275_gb300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
XI_FILES = sorted(glob.glob(os.path.join(GOLDEN, "c2_xi_*.json")))


@pytest.fixture(scope="module")
def c2():
    return synth.c2_clustered()


def _load(path):
    with open(path) as f:
        return json.load(f)


def _dev(cat):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in (cat.x, cat.y, cat.z)]


def _cat(c2, dtype_tag):
    return c2 if dtype_tag == "f64" else c2.astype(np.float32)


@pytest.mark.parametrize("path", XI_FILES, ids=[os.path.basename(p) for p in XI_FILES])
@pytest.mark.parametrize("mode", ["fp32_recheck", "fp64"])
def test_xi_full_size_matches_stored_oracle(cuda_device, c2, path, mode):
    g = _load(path)
    cat = _cat(c2, g["workload"]["cat"][1])
    assert cat.digest() == g["catalog_digest"], "catalogue differs from the stored one"
    edges = np.array([float.fromhex(h) for h in g["edges_hex"]])
    r = cf.countpairs_xi(*_dev(cat), edges, boxsize=g["box"], mode=mode)
    assert r.npairs.tolist() == g["npairs"]


RPPI_FILES = sorted(glob.glob(os.path.join(GOLDEN, "c3_rppi_*.json")))


@pytest.mark.parametrize("path", RPPI_FILES, ids=[os.path.basename(p) for p in RPPI_FILES])
@pytest.mark.parametrize("mode", ["fp32_recheck", "fp64"])
def test_rppi_full_size_matches_stored_oracle(cuda_device, c2, path, mode):
    g = _load(path)
    cat = _cat(c2, g["workload"]["cat"][1])
    assert cat.digest() == g["catalog_digest"], "catalogue differs from the stored one"
    edges = np.array([float.fromhex(h) for h in g["edges_hex"]])
    w = g["workload"]
    r = cf.countpairs_rp_pi(*_dev(cat), edges, w["pimax"], w["npibins"], boxsize=g["box"], mode=mode)
    assert r.npairs.tolist() == g["npairs"]


def test_full_size_properties(cuda_device, c2):
    edges = synth.log_edges(0.1, 25.0, 20)
    xyz = _dev(c2)
    auto = cf.countpairs_xi(*xyz, edges, boxsize=synth.BOX)
    cross = cf.countpairs_xi(*xyz, edges, x2=xyz[0], y2=xyz[1], z2=xyz[2], boxsize=synth.BOX)
    f64 = cf.countpairs_xi(*xyz, edges, boxsize=synth.BOX, mode="fp64")
    p = np.random.default_rng(7).permutation(c2.n)
    perm = cf.countpairs_xi(*_dev(c2.take(p)), edges, boxsize=synth.BOX)
    assert np.array_equal(auto.npairs, cross.npairs)
    assert np.array_equal(auto.npairs, f64.npairs)
    assert np.array_equal(auto.npairs, perm.npairs)
    # total ordered pairs is even and close to the uniform expectation plus clustering
    n = c2.n
    uniform = n * (n - 1) / synth.BOX ** 3 * 4.0 / 3.0 * np.pi * (25.0 ** 3 - 0.1 ** 3)
    assert auto.npairs.sum() % 2 == 0 and 0.95 * uniform < auto.npairs.sum() < 1.2 * uniform


def test_full_size_float32_refinements_agree(cuda_device, c2):
    edges = synth.log_edges(0.1, 25.0, 20)
    xyz = _dev(c2)
    base = cf.countpairs_xi(*xyz, edges, boxsize=synth.BOX).npairs
    for refine in [(1, 1, 1), (3, 3, 1), (4, 4, 2)]:
        r = cf.countpairs_xi(*xyz, edges, boxsize=synth.BOX, refine=refine)
        assert np.array_equal(r.npairs, base), refine
