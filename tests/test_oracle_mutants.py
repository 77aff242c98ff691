"""The pins must catch plausible mistakes in the oracle.

* C mutants: a copy of oracle/corr_oracle.c with one deliberate error, compiled with gcc into a
  temporary library; every mutant must fail at least two of the correlation pins (one for the 32-bit
  accumulator, which only the int64 overflow pin can see).
* numpy mutants: a copy of oracle/oracle.py with one deliberate error in the requantiser, the PFB,
  the station selection, the dump formats or the sample unpacking, executed as a separate module
  whose functions replace the oracle's; every mutant must fail at least one pin (an assertion or an
  error).

The committed oracle is never modified; the mutants exist only for the duration of a test."""
import ctypes
import os
import subprocess
import types

import pytest

import tests.test_oracle_pins as pins
from oracle import oracle

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "corr_oracle.c")
PY_SRC = os.path.join(os.path.dirname(SRC), "oracle.py")

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
    "last sample dropped from the cross sums": (
        "for (int t = 0; t < T; ++t) {\n              /* x_i * conj(x_j)",
        "for (int t = 0; t < T - 1; ++t) {\n              /* x_i * conj(x_j)"),
    "32-bit cross accumulators": (
        "int64_t acc_re = 0, acc_im = 0;",
        "int32_t acc_re = 0, acc_im = 0;"),
    "Im x Im dropped from the autos": (
        "acc += (int64_t)xr[t] * xr[t] + (int64_t)xi[t] * xi[t];",
        "acc += (int64_t)xr[t] * xr[t];"),
    "every channel read from channel 0": (
        "const uint8_t* row = jb->in + ((size_t)t * C + f) * N;",
        "const uint8_t* row = jb->in + ((size_t)t * C + 0) * N;"),
    "c-side input takes the a-side polarisation": (
        "const int i = a * np + p, j = c * np + q;",
        "const int i = a * np + p, j = c * np + p;"),
}

# pins each mutant must fail at least (default 2); only the int64 overflow pin can see a 32-bit
# accumulator, since every other pin stays far below 2^31
MIN_CAUGHT = {"32-bit cross accumulators": 1}

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
    ("int64 overflow", pins.test_int64_overflow_pin),
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
    assert len(caught) >= MIN_CAUGHT.get(name, 2), "mutant '%s' caught only by %s" % (name, caught)


NP_MUTANTS = {
    "requantize: ties rounded away from zero": (
        "r = np.rint(xf)",
        "r = np.trunc(xf + np.copysign(np.float32(0.5), xf))"),
    "requantize: gain product in double precision": (
        "xf = (sel.astype(np.float32) * g).astype(np.float32)",
        "xf = sel.astype(np.float64) * np.asarray(g, dtype=np.float64)"),
    "requantize: Re and Im nibbles swapped": (
        "(((r[..., 0] & 0xF) << 4) | (r[..., 1] & 0xF))",
        "(((r[..., 1] & 0xF) << 4) | (r[..., 0] & 0xF))"),
    "requantize: clipped at +8": (
        "np.clip(r, lo, 7.0)",
        "np.clip(r, lo, 8.0)"),
    "requantize: corner turn to [C][T][N]": (
        "packed.transpose(1, 2, 0)",
        "packed.transpose(2, 1, 0)"),
    "pfb_coeffs: Hann instead of Hamming window": (
        "0.54 - 0.46 * np.cos",
        "0.5 - 0.5 * np.cos"),
    "pfb_coeffs: sinc twice as wide": (
        "np.sinc((j - 0.5 * (L - 1)) / n_fft)",
        "np.sinc((j - 0.5 * (L - 1)) / (2 * n_fft))"),
    "pfb_fir: taps in reverse order": (
        "h[p * n_fft:(p + 1) * n_fft]",
        "h[(n_taps - 1 - p) * n_fft:(n_taps - p) * n_fft]"),
    "pfb: conjugated DFT": (
        "np.fft.rfft(y.astype(np.float64), axis=-1)",
        "np.conj(np.fft.rfft(y.astype(np.float64), axis=-1))"),
    "pfb: 1 / M scale dropped": (
        "[..., :n_fft // 2] / n_fft",
        "[..., :n_fft // 2]"),
    "station_cross: pair transposed": (
        "cl.append((f, st[k] * n_pol + p, st[l] * n_pol + q))",
        "cl.append((f, st[l] * n_pol + q, st[k] * n_pol + p))"),
    "to_format: normalised by n - 1": (
        "/ float(n_samples)",
        "/ float(max(n_samples - 1, 1))"),
    "unpack: sign extension off by one": (
        "re = np.where(re >= 8, re - 16, re)",
        "re = np.where(re > 8, re - 16, re)"),
}

NP_FUNCS = ("requantize", "pfb_coeffs", "pfb_fir", "pfb", "station_cross", "station_autos", "to_format", "unpack",
            "pack")

NP_PIN_CALLS = [
    ("brute force n_pol=2", lambda: pins.test_brute_force_every_cell(2, (33, 4, 6))),
    ("pack / unpack", pins.test_pack_unpack_roundtrip_and_range),
    ("dump formats", pins.test_dump_formats),
    ("station subset n_pol=1", lambda: pins.test_station_subset_brute_force(1)),
    ("station subset n_pol=2", lambda: pins.test_station_subset_brute_force(2)),
    ("station subset of all", pins.test_station_subset_of_all_stations_is_the_full_dump),
    ("requantize power-of-two gain", pins.test_requantize_power_of_two_gain_matches_integer_rounding),
    ("requantize clip and specials", pins.test_requantize_identity_clip_and_specials),
    ("requantize single-precision gain", pins.test_requantize_gain_product_is_single_precision),
    ("requantize corner turn", pins.test_requantize_corner_turn_and_per_channel_gains),
    ("pfb coefficients", pins.test_pfb_coeffs_shape_symmetry_and_peak),
    ("pfb brute force", pins.test_pfb_fir_and_dft_brute_force),
    ("pfb tone response", pins.test_pfb_channel_response_of_a_tone),
    ("pfb linearity", pins.test_pfb_linearity),
]


def _mutant_module(old, new):
    src = open(PY_SRC).read()
    assert src.count(old) == 1, "mutation site not found or ambiguous: " + old
    mod = types.ModuleType("oracle_mutant")
    mod.__file__ = PY_SRC
    exec(compile(src.replace(old, new), PY_SRC, "exec"), mod.__dict__)
    return mod


def test_unmutated_oracle_passes_every_numpy_pin():
    for label, call in NP_PIN_CALLS:
        call()


@pytest.mark.parametrize("name", sorted(NP_MUTANTS))
def test_pins_catch_the_numpy_mutant(monkeypatch, name):
    mod = _mutant_module(*NP_MUTANTS[name])
    for fn in NP_FUNCS:
        monkeypatch.setattr(oracle, fn, getattr(mod, fn))
    caught = []
    for label, call in NP_PIN_CALLS:
        try:
            call()
        except Exception:  # an assertion, or an error from a wrong shape or type
            caught.append(label)
    assert caught, "numpy mutant '%s' caught by no pin" % name
