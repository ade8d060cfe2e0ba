"""Weighted sums (pair weight w_i * w_j) and mean separations, CUDA vs oracle.

Counts stay bit-exact.  The sums differ from the oracle only by summation
order and, in float32 mode, by float32 arithmetic:
  - binary64 mode: per-pair terms are the oracle's exact binary64 products and
    square roots, so sums agree to 1e-12 relative;
  - float32 mode: weights are rounded to float32 (product error <= 3 u32) and
    each term to a power-of-two fixed-point grid, then summed exactly in
    integers (error <= 2^-22 max|w w| / |w w| per term), so wsum agrees to
    1e-5 relative; r (DD(r)) and rp (DD(rp, pi)) come from the float32 squared
    distance corrected to first order with the coordinates' float32 rounding
    residuals, so ravg agrees to 1e-5 relative as well, for float64 inputs in
    an open box too.
"""
import json
import os

import numpy as np
import pytest

import oracle
import paper_1911_08275_gb300 as cf
from paper_1911_08275_gb300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def tdev(*arrays):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


def close(got, ref, rtol, atol=0.0):
    got, ref = np.asarray(got, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    return np.all(np.abs(got - ref) <= rtol * np.abs(ref) + atol), np.max(
        np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300))


def ravg_of(rsum, den):
    den = np.asarray(den, dtype=np.float64)
    return np.where(den != 0, rsum / np.where(den != 0, den, 1.0), 0.0)


def check(r, n_ref, w_ref, rs_ref, mode, weighted):
    assert np.array_equal(r.npairs, n_ref)
    tol = 1e-12 if mode == "fp64" else 1e-5
    if weighted:
        ok, worst = close(r.wsum, w_ref, tol)
        assert ok, f"wsum rel err {worst}"
    if rs_ref is not None:
        den = w_ref if weighted else n_ref
        ok, worst = close(r.ravg, ravg_of(rs_ref, den), tol)
        assert ok, f"ravg rel err {worst}"


@pytest.mark.parametrize("mode", ["fp32_recheck", "fp64"])
@pytest.mark.parametrize("want_r", [False, True])
def test_xi_weighted_auto_periodic_float32_inputs(cuda_device, mode, want_r):
    cat = synth.neyman_scott(1500, 20.0, 2.0, 200.0, seed=71).astype(np.float32)
    w = synth.uniform_weights(cat.n, 0.5, 1.5, seed=72)
    e = synth.log_edges(0.1, 25.0, 20)
    x, y, z, wd = tdev(cat.x, cat.y, cat.z, w)
    r = cf.countpairs_xi(x, y, z, e, w=wd, boxsize=200.0, mode=mode, want_ravg=want_r)
    n, ws, rs = oracle.xi(cat.x, cat.y, cat.z, w1=w, edges=e, periodic=True, box=200.0,
                          want_r=want_r)
    check(r, n, ws, rs if want_r else None, mode, True)


@pytest.mark.parametrize("mode", ["fp32_recheck", "fp64"])
def test_xi_ravg_unweighted(cuda_device, mode):
    cat = synth.neyman_scott(1200, 20.0, 2.0, 180.0, seed=73).astype(np.float32)
    e = synth.log_edges(0.1, 25.0, 20)
    x, y, z = tdev(cat.x, cat.y, cat.z)
    r = cf.countpairs_xi(x, y, z, e, boxsize=180.0, mode=mode, want_ravg=True)
    assert r.wsum is None
    n, _, rs = oracle.xi(cat.x, cat.y, cat.z, edges=e, periodic=True, box=180.0, want_r=True)
    check(r, n, None, rs, mode, False)
    assert np.all((r.ravg >= e[:-1] * (1 - 1e-6)) | (r.npairs == 0))
    assert np.all(r.ravg <= e[1:] * (1 + 1e-6))


@pytest.mark.parametrize("mode", ["fp32_recheck", "fp64"])
def test_xi_weighted_dr_open_box_float64_inputs(cuda_device, mode):
    # DR: clustered data x uniform randoms, weights U(0.5, 1.5), open box
    d = synth.neyman_scott(600, 20.0, 2.0, 150.0, seed=74)
    rnd = synth.uniform_box(40000, 150.0, seed=75)
    wd = synth.uniform_weights(d.n, 0.5, 1.5, seed=76)
    wr = synth.uniform_weights(rnd.n, 0.5, 1.5, seed=77)
    e = synth.log_edges(0.1, 25.0, 20)
    a = tdev(d.x, d.y, d.z, wd)
    b = tdev(rnd.x, rnd.y, rnd.z, wr)
    r = cf.countpairs_xi(*a[:3], e, w=a[3], x2=b[0], y2=b[1], z2=b[2], w2=b[3], periodic=False,
                         mode=mode, want_ravg=True)
    n, ws, rs = oracle.xi(d.x, d.y, d.z, w1=wd, x2=rnd.x, y2=rnd.y, z2=rnd.z, w2=wr, edges=e,
                          autocorr=False, periodic=False, want_r=True)
    check(r, n, ws, rs, mode, True)


@pytest.mark.parametrize("periodic", [True, False])
def test_xi_ravg_float64_inputs_fp32_mode(cuda_device, periodic):
    # float64 coordinates the float32 path cannot hold exactly: the residual-
    # corrected mean separation agrees to 1e-5 relative in every bin, down to
    # the smallest separations (clusters of sigma 2 fill the bins near 0.1)
    cat = synth.neyman_scott(1500, 20.0, 2.0, 300.0, seed=86)
    e = synth.log_edges(0.1, 25.0, 20)
    x, y, z = tdev(cat.x, cat.y, cat.z)
    r = cf.countpairs_xi(x, y, z, e, boxsize=300.0, periodic=periodic, want_ravg=True)
    n, _, rs = oracle.xi(cat.x, cat.y, cat.z, edges=e, periodic=periodic, box=300.0, want_r=True)
    assert n[0] > 0
    check(r, n, None, rs, "fp32_recheck", False)


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("weighted", [False, True])
def test_rppi_ravg_float64_inputs_fp32_mode(cuda_device, periodic, weighted):
    # the same for DD(rp, pi): rp from residual-corrected rp^2, 1e-5 relative in
    # every (rp, pi) slot down to the 0.1-0.14 rp bin, auto and cross
    cat = synth.neyman_scott(1000, 20.0, 2.0, 300.0, seed=87)
    u = synth.uniform_box(4000, 300.0, seed=88)
    w = synth.uniform_weights(cat.n, 0.5, 1.5, seed=89) if weighted else None
    wu = synth.uniform_weights(u.n, 0.5, 1.5, seed=90) if weighted else None
    e = synth.log_edges(0.1, 20.0, 12)
    x, y, z = tdev(cat.x, cat.y, cat.z)
    kw = dict(boxsize=300.0, periodic=periodic, want_ravg=True)
    if weighted:
        kw["w"] = tdev(w)[0]
    r = cf.countpairs_rp_pi(x, y, z, e, 30.0, 30, **kw)
    n, ws, rs = oracle.rppi(cat.x, cat.y, cat.z, w1=w, rp_edges=e, pimax=30.0, npibins=30,
                            periodic=periodic, box=300.0, want_r=True)
    assert n[0].sum() > 0
    check(r, n, ws, rs, "fp32_recheck", weighted)
    ux, uy, uz = tdev(u.x, u.y, u.z)
    if weighted:
        kw["w2"] = tdev(wu)[0]
    rc = cf.countpairs_rp_pi(x, y, z, e, 30.0, 30, x2=ux, y2=uy, z2=uz, **kw)
    n, ws, rs = oracle.rppi(cat.x, cat.y, cat.z, w1=w, x2=u.x, y2=u.y, z2=u.z, w2=wu, rp_edges=e,
                            pimax=30.0, npibins=30, autocorr=False, periodic=periodic, box=300.0,
                            want_r=True)
    check(rc, n, ws, rs, "fp32_recheck", weighted)


@pytest.mark.parametrize("mode", ["fp32_recheck", "fp64"])
def test_xi_weighted_many_bins_and_ragged(cuda_device, mode):
    # 64 bins: the largest shared layout of the weighted float32 kernel
    for n_pts, seed in ((0, 78), (1, 79), (33, 80), (5000, 81)):
        cat = synth.uniform_box(n_pts, 60.0, seed=seed).astype(np.float32)
        w = synth.uniform_weights(n_pts, 0.5, 1.5, seed=seed + 100)
        e = synth.log_edges(0.05, 20.0, 64)
        x, y, z, wd = tdev(cat.x, cat.y, cat.z, w)
        r = cf.countpairs_xi(x, y, z, e, w=wd, boxsize=60.0, mode=mode, want_ravg=True)
        n, ws, rs = oracle.xi(cat.x, cat.y, cat.z, w1=w, edges=e, periodic=True, box=60.0,
                              want_r=True)
        check(r, n, ws, rs, mode, True)


@pytest.mark.parametrize("mode", ["fp32_recheck", "fp64"])
def test_rppi_weighted_with_ravg(cuda_device, mode):
    cat = synth.neyman_scott(1000, 20.0, 2.0, 160.0, seed=82).astype(np.float32)
    w = synth.uniform_weights(cat.n, 0.5, 1.5, seed=83)
    e = synth.log_edges(0.1, 20.0, 12)
    x, y, z, wd = tdev(cat.x, cat.y, cat.z, w)
    r = cf.countpairs_rp_pi(x, y, z, e, 30.0, 30, w=wd, boxsize=160.0, mode=mode, want_ravg=True)
    n, ws, rs = oracle.rppi(cat.x, cat.y, cat.z, w1=w, rp_edges=e, pimax=30.0, npibins=30,
                            periodic=True, box=160.0, want_r=True)
    check(r, n, ws, rs, mode, True)


def test_weighted_counts_equal_unweighted_counts(cuda_device):
    cat = synth.neyman_scott(800, 20.0, 2.0, 120.0, seed=84)
    w = synth.uniform_weights(cat.n, 0.5, 1.5, seed=85)
    e = synth.log_edges(0.1, 20.0, 16)
    x, y, z, wd = tdev(cat.x, cat.y, cat.z, w)
    plain = cf.countpairs_xi(x, y, z, e, boxsize=120.0)
    unit = cf.countpairs_xi(x, y, z, e, w=tdev(np.ones(cat.n))[0], boxsize=120.0)
    wtd = cf.countpairs_xi(x, y, z, e, w=wd, boxsize=120.0, want_ravg=True)
    assert np.array_equal(plain.npairs, unit.npairs) and np.array_equal(plain.npairs, wtd.npairs)
    # unit weights: the weighted sum is the count itself (float32 partials of
    # integers below 2^24 are exact)
    assert np.array_equal(unit.wsum, plain.npairs.astype(np.float64))


@pytest.mark.parametrize("mode", ["fp32_recheck", "fp64"])
def test_dr_slice_full_randoms_matches_stored_oracle(cuda_device, mode):
    # 8000 weighted clustered points against all 12M weighted randoms, open box,
    # in the launch configuration of the weighted DR workload.
    with open(os.path.join(GOLDEN, "c4_dr_slice8000_f64.json")) as f:
        g = json.load(f)
    d = synth.c2_clustered()
    d.w = synth.uniform_weights(d.n, 0.5, 1.5, seed=4)
    ds = d.take(np.arange(g["n"]))
    rnd = synth.c4_randoms()
    rnd.w = synth.uniform_weights(rnd.n, 0.5, 1.5, seed=5)
    assert ds.digest() == g["catalog_digest"] and rnd.digest() == g["randoms_digest"]
    e = np.array([float.fromhex(h) for h in g["edges_hex"]])
    a = tdev(ds.x, ds.y, ds.z, ds.w)
    b = tdev(rnd.x, rnd.y, rnd.z, rnd.w)
    r = cf.countpairs_xi(*a[:3], e, w=a[3], x2=b[0], y2=b[1], z2=b[2], w2=b[3], periodic=False,
                         mode=mode, want_ravg=True)
    ws = np.array([float.fromhex(h) for h in g["wsum_hex"]])
    rs = np.array([float.fromhex(h) for h in g["rsum_hex"]])
    check(r, np.array(g["npairs"], dtype=np.uint64), ws, rs, mode, True)
