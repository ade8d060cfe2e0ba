"""Autotuner cache (include/cf.h, cf_tune_*): JSON round trip and rejection of
malformed files, through the C ABI without a GPU."""
import json

import pytest

import paper_1911_08275_gb300 as cf

ENTRY = ('{"key": "k0 m1 d1 a1 p1 w0 n40 n40 r12 b20", "refine": [2, 2, 1], "chunk": 16, '
         '"pp": 2, "ms": 1.7}')


@pytest.fixture(autouse=True)
def empty_cache():
    cf.tune_clear()
    yield
    cf.tune_clear()


def write(tmp_path, name, text):
    p = tmp_path / name
    p.write_text(text)
    return str(p)


def test_round_trip(tmp_path):
    src = write(tmp_path, "a.json", '{"version": 1, "entries": [\n ' + ENTRY + ',\n ' +
                ENTRY.replace("r12", "r14").replace("[2, 2, 1]", "[3, 3, 1]").replace(
                    '"pp": 2', '"pp": 1') + '\n]}\n')
    cf.tune_load(src)
    assert cf.tune_count() == 2
    out = str(tmp_path / "b.json")
    cf.tune_save(out)
    doc = json.loads(open(out).read())
    assert doc["version"] == 1
    by_key = {e["key"]: e for e in doc["entries"]}
    assert by_key["k0 m1 d1 a1 p1 w0 n40 n40 r14 b20"]["refine"] == [3, 3, 1]
    assert by_key["k0 m1 d1 a1 p1 w0 n40 n40 r14 b20"]["pp"] == 1
    cf.tune_clear()
    assert cf.tune_count() == 0
    cf.tune_load(out)
    assert cf.tune_count() == 2


@pytest.mark.parametrize("text", [
    "garbage",
    '{"version": 2, "entries": []}',
    '{"version": 1, "entries": [{"key": "x", "refine": [2, 2], "chunk": 16, "pp": 2, "ms": 1}]}',
    '{"version": 1, "entries": [' + ENTRY.replace('"chunk": 16', '"chunk": 12') + ']}',
    '{"version": 1, "entries": [' + ENTRY.replace("[2, 2, 1]", "[9, 2, 1]") + ']}',
])
def test_malformed_files_are_rejected_and_leave_the_cache_alone(tmp_path, text):
    cf.tune_load(write(tmp_path, "ok.json", '{"version": 1, "entries": [' + ENTRY + ']}'))
    with pytest.raises(cf.CfError) as ei:
        cf.tune_load(write(tmp_path, "bad.json", text))
    assert ei.value.status == cf.CF_EINVAL
    assert cf.tune_count() == 1


def test_missing_file_is_an_error(tmp_path):
    with pytest.raises(cf.CfError):
        cf.tune_load(str(tmp_path / "nope.json"))
