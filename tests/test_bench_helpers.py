"""bench.py's host-side helpers (no GPU): the traffic figure is reported only
while the pair-kernel sources hash to the profiled ones, and the clock record
taken during the timed region is summarised with every throttle reason seen."""
import hashlib
import os

import pytest

import bench


def test_committed_profile_matches_the_kernel_sources():
    # the committed ncu summary names the hash of the sources it was taken on;
    # either it matches (traffic reported) or the bench reports null
    traffic, src = bench.profile_traffic()
    h = hashlib.sha256()
    for f in bench.KERNEL_SOURCES:
        h.update(open(f, "rb").read())
    text = open(bench.PROFILE).read()
    if h.hexdigest()[:16] in text:
        assert isinstance(traffic, int) and traffic > 0 and "ncu capture" in src
    else:
        assert traffic is None


def test_traffic_is_dropped_once_a_kernel_source_changes(tmp_path, monkeypatch):
    srcs = []
    for name, body in (("pairs.cu", b"kernel v1\n"), ("cf_internal.cuh", b"layout\n")):
        p = tmp_path / name
        p.write_bytes(body)
        srcs.append(str(p))
    h = hashlib.sha256(b"kernel v1\n" + b"layout\n").hexdigest()[:16]
    prof = tmp_path / "profile.md"
    prof.write_text(f"# capture\n\nkernel_source_sha256_16: {h}   (note)\n"
                    "traffic_bytes_per_launch: 12345\n")
    monkeypatch.setattr(bench, "KERNEL_SOURCES", srcs)
    monkeypatch.setattr(bench, "PROFILE", str(prof))
    assert bench.profile_traffic() == (12345, "ncu capture profile.md")
    (tmp_path / "pairs.cu").write_bytes(b"kernel v2\n")
    traffic, why = bench.profile_traffic()
    assert traffic is None and "changed" in why
    monkeypatch.setattr(bench, "PROFILE", str(tmp_path / "missing.md"))
    assert bench.profile_traffic()[0] is None


def clock_rows(rows):
    return "".join(", ".join(r) + "\n" for r in rows)


@pytest.mark.parametrize("active,want", [
    ((), []),
    (("sw_power_cap",), ["sw_power_cap"]),
    (("hw_slowdown", "sw_thermal_slowdown"), ["hw_slowdown", "sw_thermal_slowdown"]),
])
def test_clock_summary_reports_median_and_reasons(tmp_path, active, want):
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    rows = []
    for k, mhz in enumerate(("2070", "2070", "1980", "2070", "2070")):
        flags = ["Active" if (n in active and k == 2) else "Not Active" for n in names]
        rows.append(["0", mhz, "2070", "812.5", "0x0", *flags])
    rows.append(["0", "[N/A]", "2070", "[N/A]", "0x0", *["Not Active"] * 4])  # unparsable: skipped
    p = tmp_path / "clocks.csv"
    p.write_text(clock_rows(rows))
    s = bench.ClockSampler(0)
    s.path = str(p)
    out = s.summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["samples"] == 5 and out["power_w_max"] == 812.5
    assert out["reasons"] == want
    assert not os.path.exists(p)


def test_clock_summary_without_samples(tmp_path):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "none.csv")
    assert s.summary()["reasons"] == ["unsampled"]


def test_counts_equal_oracle_checks_the_stored_histogram_and_its_catalogue():
    import json

    import numpy as np

    from paper_1911_08275_gb300 import synth
    path = os.path.join(bench.ROOT, "tests", "golden", "c2_xi_r10_f64.json")
    with open(path) as f:
        g = json.load(f)
    cat = synth.c2_clustered()
    ref = np.asarray(g["npairs"], dtype=np.uint64)
    assert bench.counts_equal_oracle("c2_xi_r10_f64", cat, ref) is True
    bad = ref.copy()
    bad[-1] += 2
    assert bench.counts_equal_oracle("c2_xi_r10_f64", cat, bad) is False
    # another catalogue, or no stored histogram: no claim either way
    other = synth.uniform_box(1000, 420.0, seed=1)
    assert bench.counts_equal_oracle("c2_xi_r10_f64", other, ref) is None
    assert bench.counts_equal_oracle("no_such_golden", cat, ref) is None
