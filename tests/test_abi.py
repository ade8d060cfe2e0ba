"""The C-ABI library builds, loads and exports every entry point of include/cf.h.

These tests need no GPU: loading the library does not initialise a device, and
argument errors are reported before any CUDA call.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1911_08275_gb300 as cf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(cf_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_documented_entry_points():
    names = header_functions()
    for required in ("cf_countpairs_xi", "cf_countpairs_rp_pi", "cf_last_error", "cf_version"):
        assert required in names


def test_library_exports_every_header_symbol():
    L = ctypes.CDLL(cf.lib().__getattribute__("_name"))
    for name in header_functions():
        assert hasattr(L, name), f"{name} declared in include/ but not exported"
    assert set(cf.EXPORTS) <= set(header_functions())


def test_version_string():
    assert "sm_103a" in cf.version()


@pytest.mark.parametrize("edges,msg", [
    ([1.0], "at least 2"),
    ([2.0, 1.0], "strictly increasing"),
    ([-1.0, 1.0], "edges[0] >= 0"),
    (list(np.arange(66.0) + 1.0), "at most 64"),
])
def test_bad_edges_rejected_before_any_device_work(edges, msg):
    x = np.zeros(4)
    with pytest.raises(cf.CfError) as ei:
        cf.countpairs_xi(x, x, x, edges, boxsize=10.0)
    assert ei.value.status == cf.CF_EINVAL and msg in str(ei.value)


def test_periodic_rmax_must_be_below_half_box():
    x = np.zeros(4)
    with pytest.raises(cf.CfError, match="boxsize/2"):
        cf.countpairs_xi(x, x, x, [0.1, 5.0], boxsize=10.0)


def test_cross_needs_second_catalogue():
    x = np.zeros(4)
    with pytest.raises(ValueError):
        cf.countpairs_xi(x, x, x, [0.1, 1.0], autocorr=False)


def test_no_cpu_fallback_without_a_gpu():
    # on a host without a usable GPU a counting call reports the CUDA error
    # (status and message) instead of computing anything on the CPU
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    x = np.random.default_rng(0).uniform(0.0, 10.0, 100)
    with pytest.raises(cf.CfError) as ei:
        cf.countpairs_xi(x, x, x, [0.1, 1.0], boxsize=10.0)
    assert ei.value.status == cf.CF_ECUDA and "CUDA" in str(ei.value)
    with pytest.raises(cf.CfError) as ei:
        cf.countpairs_rp_pi(x, x, x, [0.1, 1.0], 2.0, 2, boxsize=10.0)
    assert ei.value.status == cf.CF_ECUDA
