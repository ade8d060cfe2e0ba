"""The gridded CPU counter (the benchmark's CPU baseline) against the oracle.

``oracle/gridded.c`` counts DD(r) by cell lists (Sec. 1.2 / 2.1 / 2.2 of the
paper, scalar, OpenMP) with the oracle's canonical binary64 arithmetic; its
histograms must equal the brute-force oracle's bit for bit, on the C1
configuration (20,000 uniform points, periodic box 420, 20 log bins 0.1-25)
and on a 10^5-point clustered set, auto and cross, periodic and open, for
several refinements, including grids of two cells per axis and pairs placed
across the periodic faces.
"""
import numpy as np
import pytest

import oracle
from paper_1911_08275_gb300 import synth


@pytest.fixture(scope="module")
def clustered():
    c = synth.neyman_scott(5000, 20.0, 2.0, 250.0, seed=201)
    e = synth.log_edges(0.1, 25.0, 20)
    ref = oracle.xi(c.x, c.y, c.z, edges=e, periodic=True, box=250.0)[0]
    return c, e, ref


def test_c1_matches_oracle():
    c = synth.c1_uniform20k()
    e = synth.log_edges(0.1, 25.0, 20)
    ref = oracle.xi(c.x, c.y, c.z, edges=e, periodic=True, box=c.box)[0]
    got = oracle.gridded_xi(c.x, c.y, c.z, edges=e, periodic=True, box=c.box)
    assert np.array_equal(got, ref) and ref.sum() > 0


@pytest.mark.parametrize("refine", [(1, 1, 1), (2, 2, 1), (3, 3, 2), (4, 2, 3)])
def test_clustered_100k_matches_oracle(clustered, refine):
    c, e, ref = clustered
    assert c.n > 90000
    got = oracle.gridded_xi(c.x, c.y, c.z, edges=e, periodic=True, box=250.0, refine=refine)
    assert np.array_equal(got, ref)


def test_cross_open_and_periodic_match_oracle():
    a = synth.neyman_scott(400, 20.0, 2.0, 120.0, seed=202)
    b = synth.uniform_box(12000, 120.0, seed=203)
    e = synth.log_edges(0.2, 30.0, 14)
    for periodic in (True, False):
        ref = oracle.xi(a.x, a.y, a.z, x2=b.x, y2=b.y, z2=b.z, edges=e, autocorr=False,
                        periodic=periodic, box=120.0)[0]
        for refine in ((2, 2, 1), (3, 1, 2)):
            got = oracle.gridded_xi(a.x, a.y, a.z, x2=b.x, y2=b.y, z2=b.z, edges=e, autocorr=False,
                                    periodic=periodic, box=120.0, refine=refine)
            assert np.array_equal(got, ref)


def test_two_cells_per_axis_and_face_pairs():
    # Rmax just below L/2: two cells per axis, so the stencil wraps onto the
    # same cells through different images; points sit at the faces
    rng = np.random.default_rng(204)
    pts = rng.uniform(0.0, 10.0, size=(3000, 3))
    pts[:200] = np.where(rng.random((200, 3)) < 0.5, rng.uniform(0, 0.3, (200, 3)),
                         rng.uniform(9.7, 10.0, (200, 3)))
    x, y, z = (np.ascontiguousarray(pts[:, k]) for k in range(3))
    e = np.array([0.0, 0.5, 1.0, 2.5, 4.99])
    ref = oracle.xi(x, y, z, edges=e, periodic=True, box=10.0)[0]
    for refine in ((1, 1, 1), (2, 2, 2)):
        got = oracle.gridded_xi(x, y, z, edges=e, periodic=True, box=10.0, refine=refine)
        assert np.array_equal(got, ref)


def test_tiny_and_degenerate_inputs():
    e = [0.0, 1.0, 2.0]
    for n in (0, 1, 2):
        x = y = z = np.full(n, 3.0)
        ref = oracle.xi(x, y, z, edges=e, periodic=False)[0]
        got = oracle.gridded_xi(x, y, z, edges=e, periodic=False)
        assert np.array_equal(got, ref)
    # every point in one spot, open box of zero extent
    x = y = z = np.full(50, 1.25)
    assert oracle.gridded_xi(x, y, z, edges=e, periodic=False).tolist() == [50 * 49, 0]
