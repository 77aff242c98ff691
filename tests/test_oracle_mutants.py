"""The pins must catch plausible mistakes in the oracle: each mutant below is a copy of
oracle/corr_oracle.c with one deliberate error, compiled with gcc into a temporary library (the
committed oracle is untouched). With the mutant in place of the oracle, the pins of
test_oracle_pins.py are run again; every mutant must fail at least two of them."""
import ctypes
import os
import subprocess

import pytest

import tests.test_oracle_pins as pins
from oracle import oracle

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "corr_oracle.c")

MUTANTS = {
    "conjugate on the wrong side": (
        "acc_im += (int64_t)xi[t] * yr[t] - (int64_t)xr[t] * yi[t];",
        "acc_im += (int64_t)xr[t] * yi[t] - (int64_t)xi[t] * yr[t];"),
    "dropped Im x Im term": (
        "acc_re += (int64_t)xr[t] * yr[t] + (int64_t)xi[t] * yi[t];",
        "acc_re += (int64_t)xr[t] * yr[t];"),
    "swapped polarisation order": (
        "(size_t)(p * np + q)) * 2",
        "(size_t)(q * np + p)) * 2"),
    "missing sign extension": (
        "return (v & 0x8u) ? (int)v - 16 : (int)v;",
        "return (int)v;"),
    "transposed triangle index": (
        "const int64_t b = (int64_t)a * (a + 1) / 2 + c;",
        "const int64_t b = (int64_t)c * (c + 1) / 2 + a;"),
}

PIN_CALLS = [
    ("brute force n_pol=1", lambda: pins.test_brute_force_every_cell(1, (7, 3, 4))),
    ("brute force n_pol=2", lambda: pins.test_brute_force_every_cell(2, (33, 4, 6))),
    ("rank-1 closed form", pins.test_rank1_common_signal_closed_form),
    ("Walsh-Hadamard closed form", pins.test_walsh_hadamard_codes_closed_form),
    ("extreme -8-8i", lambda: pins.test_constant_extremes(-8, -8, 128)),
    ("extreme -8+7i", lambda: pins.test_constant_extremes(-8, 7, 113)),
    ("alternating signs", pins.test_alternating_signs_cancel),
    ("invariants", pins.test_invariants_random),
    ("permutation", pins.test_permutation_of_inputs),
    ("golden fixtures", pins.test_golden_fixtures),
]


def _mutant_lib(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, "mutation site not found: " + name
    path_c = tmp_path / "mutant.c"
    path_c.write_text(src.replace(old, new))
    path_so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-pthread", str(path_c), "-o", str(path_so)])
    lib = ctypes.CDLL(str(path_so))
    ref = oracle._load()
    for fn in ("oracle_correlate", "oracle_cells", "oracle_autos"):
        getattr(lib, fn).argtypes = getattr(ref, fn).argtypes
        getattr(lib, fn).restype = getattr(ref, fn).restype
    return lib


def test_unmutated_oracle_passes_every_pin():
    for label, call in PIN_CALLS:
        call()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_the_mutant(tmp_path, monkeypatch, name):
    old, new = MUTANTS[name]
    monkeypatch.setattr(oracle, "_lib", _mutant_lib(tmp_path, name, old, new))
    caught = []
    for label, call in PIN_CALLS:
        try:
            call()
        except AssertionError:
            caught.append(label)
    assert len(caught) >= 2, "mutant '%s' caught only by %s" % (name, caught)
