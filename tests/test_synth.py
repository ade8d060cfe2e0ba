"""The seeded input generator (no GPU).

Stored expected histograms are keyed on the exact bits of the catalogues, so
the generator must reproduce its definition bit for bit on any machine:

* SplitMix64 against its published reference outputs, and the keyed
  counter-based form used here against a sequential pure-Python SplitMix64;
* the series logarithm and exponential (used instead of the platform libm)
  within a few ulps of the libm values;
* the Gaussian and Poisson draws against their moments;
* the full-size catalogues against the digests stored with their expected
  histograms.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1911_08275_gb300 import synth

M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def mix(z):
    """SplitMix64's output function, in Python integers (Steele, Lea & Flood 2014)."""
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def splitmix_sequence(state, n):
    out = []
    for _ in range(n):
        state = (state + GAMMA) & M64
        out.append(mix(state))
    return out


def test_splitmix64_reference_outputs():
    # the first outputs of SplitMix64 from state 0, as published with its
    # reference implementation
    assert splitmix_sequence(0, 3) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    k = np.arange(1, 4, dtype=np.uint64)
    with np.errstate(over="ignore"):
        got = synth._mix64(k * np.uint64(GAMMA))
    assert [int(v) for v in got] == splitmix_sequence(0, 3)


@pytest.mark.parametrize("seed,stream,offset", [(0, 0, 0), (2, 5, 0), (1000, 3, 17), (2**63 + 5, 6, 3)])
def test_random_u64_is_splitmix_from_a_keyed_state(seed, stream, offset):
    key = (seed ^ ((stream * 0xD1B54A32D192ED03) & M64)) & M64
    base = mix(key)
    want = splitmix_sequence(base, offset + 40)[offset:]
    got = synth.random_u64(seed, stream, 40, offset)
    assert [int(v) for v in got] == want


def test_uniform01_has_53_bits_in_unit_interval():
    u = synth.uniform01(3, 1, 100_000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.all(u * 2.0 ** 53 == np.floor(u * 2.0 ** 53))
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / u.size)


def ulps(a, b):
    return np.abs(a - b) / np.spacing(np.abs(b))


def test_series_log_and_exp_track_libm():
    rng = np.random.default_rng(0)
    x = 10.0 ** rng.uniform(-300, 300, 100_000)
    assert ulps(synth._ln(x), np.log(x)).max() <= 4
    # exp serves log-spaced edges: arguments ln(1e-4) .. ln(1e4); its reduction by
    # the rounded ln 2 loses about one ulp per 1.5 units of |x|
    y = rng.uniform(-10.0, 10.0, 100_000)
    assert ulps(synth._exp(y), np.exp(y)).max() <= 8
    assert synth._ln(np.array([1.0]))[0] == 0.0 and synth._exp(np.array([0.0]))[0] == 1.0


def test_gaussian_moments():
    g = synth.gaussian(9, 4, 400_000)
    n = g.size
    assert abs(g.mean()) < 5 / math.sqrt(n)
    assert abs(g.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert abs(np.mean(np.abs(g) < 1.0) - math.erf(1 / math.sqrt(2))) < 5 * math.sqrt(0.25 / n)


@pytest.mark.parametrize("mean", [5.0, 20.0])
def test_poisson_moments(mean):
    c = synth.poisson(11, 3, 100_000, mean)
    n = c.size
    assert abs(c.mean() - mean) < 5 * math.sqrt(mean / n)
    assert abs(c.var() / mean - 1.0) < 0.05
    p0 = math.exp(-mean)
    assert abs(np.mean(c == 0) - p0) < 5 * math.sqrt(p0 * (1 - p0) / n) + 1e-6


def test_log_edges_hit_both_ends_exactly():
    e = synth.log_edges(0.1, 25.0, 20)
    assert e[0] == 0.1 and e[-1] == 25.0 and np.all(np.diff(e) > 0)
    assert np.allclose(np.diff(np.log(e)), math.log(250.0) / 20, rtol=1e-12)


def test_full_size_catalogues_match_the_stored_digests():
    # the expected full-size histograms were computed on exactly these bits
    c2 = synth.c2_clustered()
    for name in ("c2_xi_r25_f64.json", "c2_xi_r25_f32.json", "c3_rppi_f32.json"):
        g = json.load(open(os.path.join(GOLDEN, name)))
        tag = g["workload"]["cat"][1]
        cat = c2 if tag == "f64" else c2.astype(np.float32)
        assert cat.digest() == g["catalog_digest"], name
