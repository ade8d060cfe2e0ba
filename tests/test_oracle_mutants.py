"""The oracle's pins are strong enough to catch plausible mistakes.

Each mutant is a one-line change to a copy of ``oracle/oracle.c`` (a dropped
term, a wrong sign or index, an off-by-one edge test, a missing factor of two),
compiled on the CPU into a temporary library.  The pins of
``test_oracle_pins.py`` are run against it and at least one must fail.  The
real oracle is never modified.

Two one-line changes are equivalent (they cannot change any output) and are
not listed: wrapping at |d| >= L/2 instead of > L/2 (both images then have
|d| = L/2), and making the [Rmin^2, Rmax^2) pre-check in bin_of inclusive (the
per-bin half-open test that follows still rejects r^2 = Rmax^2).
"""
import os

import pytest

import oracle
from tests import test_oracle_pins as pins

MUTANTS = {
    "drop_dz_term": ("const double r2 = rp2 + dz * dz;", "const double r2 = rp2;"),
    "rp2_uses_dz": ("const double rp2 = dx * dx + dy * dy;", "const double rp2 = dx * dx + dz * dz;"),
    "wrap_sign": ("return d + (double)s * L;", "return d - (double)s * L;"),
    "wrong_axis_box": ("component(yi, by[j], periodic, Ly)", "component(yi, by[j], periodic, Lx)"),
    "bin_closed_upper": ("if (E2[k] <= s && s < E2[k + 1])", "if (E2[k] < s && s <= E2[k + 1])"),
    "no_auto_doubling": ("const uint64_t mult = jb->autocorr ? 2u : 1u;",
                         "const uint64_t mult = 1u;"),
    "self_pairs_counted": ("const int64_t j0 = jb->autocorr ? i + 1 : 0;",
                           "const int64_t j0 = jb->autocorr ? i : 0;"),
    "weight_wrong_index": ("pw = a->w[i] * b->w[j];", "pw = a->w[i] * b->w[i];"),
    "weight_sum_not_product": ("pw = a->w[i] * b->w[j];", "pw = a->w[i] + b->w[j];"),
    "ravg_unsquared": ("const double rv = sqrt(s) * pw;", "const double rv = s * pw;"),
    "rppi_ravg_uses_r": ("s = rp2;", "s = rp2 + dz * dz;"),
    "pi_without_abs": ("pibin_of(fabs(dz), jb->P", "pibin_of(dz, jb->P"),
    "pi_edges_shifted": ("P[m] = (pimax * (double)m) / (double)npibins;",
                         "P[m] = (pimax * (double)(m + 1)) / (double)npibins;"),
    "edges_not_squared": ("E2[k] = edges[k] * edges[k];", "E2[k] = edges[k];"),
    "pi_bin_uses_rp_edges": ("slot = k * jb->npibins + m;", "slot = m * jb->npibins + k;"),
}


@pytest.fixture(scope="module")
def source():
    with open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")) as f:
        return f.read()


def _fails(orc) -> str | None:
    for fn, kw in pins.pin_cases():
        try:
            fn(orc, **kw)
        except Exception as exc:  # any failed pin (assertion or error) kills the mutant
            return f"{fn.__name__}{kw}: {type(exc).__name__}"
    return None


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, source, tmp_path):
    old, new = MUTANTS[name]
    assert source.count(old) == 1, f"mutation site for {name} not found exactly once"
    src = tmp_path / "oracle_mutant.c"
    src.write_text(source.replace(old, new))
    lib = oracle.build(force=True, src=str(src), out=str(tmp_path / "liboracle_mutant.so"))
    killed_by = _fails(oracle.load_variant(lib))
    assert killed_by is not None, f"mutant {name} survived every pin"


def test_unmodified_oracle_passes_every_pin():
    assert _fails(oracle.Oracle(oracle._load())) is None
