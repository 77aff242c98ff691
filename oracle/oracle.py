"""CPU oracle for the X-engine: Python wrapper around ``corr_oracle.c`` plus the dump-format rules.

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module. The product library never imports, links or calls it, and it
shares no code with the CUDA path.

Definitions it follows (paper: Sec. 1, the O(N^2) stage on GPUs; Sec. 2.5, pairwise products of the
spectra integrated over groups of spectra; Table 1 note (a), the four polarisation products;
Sec. 2.6, the auto-correlation cells; Sec. 2.2, samples requantised to 4+4 bits):

* sample byte = (Re nibble << 4) | Im nibble, each nibble a 4-bit two's-complement integer;
* ``cross[f, b(a, c), p * n_pol + q] = sum_t x_{a p}(t) conj(x_{c q}(t))`` for stations a >= c,
  ``b(a, c) = a (a + 1) / 2 + c``, stored as int64 (re, im);
* ``autos[f, m] = sum_t |x_m(t)|^2``;
* selected stations (Sec. 2.6, cells of chosen antennas dumped and zeroed on their own cadence), for
  a station list st: ``station_cross[f, k (k + 1) / 2 + l, p * n_pol + q] =
  sum_t x_{st[k] p}(t) conj(x_{st[l] q}(t))`` for list positions k >= l, and
  ``station_autos[f, k, p] = autos[f, st[k] n_pol + p]``.

Requantiser (the F-engine tail, Sec. 2.2: a digital gain across the band, requantisation from 18+18
to 4+4 bits, channel selection, corner turn; the rounding rule is not stated, the reading taken is
round to nearest, ties to even, in IEEE single precision):

* per component v: ``x = fl32(gain * fl32(v))``, ``q = clip(rint(x), lo, 7)``, lo = -8 (or -7 when
  symmetric), NaN -> 0;
* ``out[t, c, n] = (q_re << 4) | (q_im & 0xF)`` for PFB channel chan0 + c of input n at time t.

PFB F-engine (Sec. 2.2: a 4-tap, 8192-point polyphase filterbank, FIR then FFT, Hamming window,
18-bit coefficients, a halving at each FFT stage; window centring and coefficient rounding are the
readings taken):

* ``h[j] = floor(s w[j] sinc((j - (L - 1) / 2) / M) + 1/2)``, ``L = P M``, Hamming
  ``w[j] = 0.54 - 0.46 cos(2 pi j / (L - 1))``, s such that max |h| = 2^17 - 1;
* ``y_t[m] = sum_p h[p M + m] x[(t + p) M + m]`` (exact integers for 8-bit samples);
* ``X_t[k] = M^-1 sum_m y_t[m] exp(-2 pi i k m / M)`` for k < M / 2 (the per-stage halving of a
  radix-2 FFT over log2 M stages is a factor 1 / M in all).

Dump formats (the paper stores visibilities as 32-bit floats after averaging, Sec. 2.5; the
integer sum is the exact product, so two float views are defined on top of it):

* CI64: the int64 sums themselves;
* CF32: each int64 rounded to the nearest float32;
* CF32_NORM: each int64 divided by the sample count in float64, then rounded to float32.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "corr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

FMT_CI64, FMT_CF32, FMT_CF32_NORM = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc into ``oracle/_build/liboracle.so``; returns the path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            p_u8 = ctypes.POINTER(ctypes.c_uint8)
            p_i64 = ctypes.POINTER(ctypes.c_int64)
            p_i32 = ctypes.POINTER(ctypes.c_int32)
            lib.oracle_correlate.argtypes = [p_u8, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             p_i64, p_i64, ctypes.c_int]
            lib.oracle_correlate.restype = ctypes.c_int
            lib.oracle_cells.argtypes = [p_u8, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, p_i32, p_i64]
            lib.oracle_cells.restype = ctypes.c_int
            lib.oracle_autos.argtypes = [p_u8, ctypes.c_int, ctypes.c_int, ctypes.c_int, p_i64]
            lib.oracle_autos.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _check_samples(samples: np.ndarray) -> np.ndarray:
    if samples.dtype != np.uint8 or samples.ndim != 3:
        raise ValueError("samples must be a uint8 array of shape [T][C][N]")
    return np.ascontiguousarray(samples)


def n_baselines(n_inputs: int, n_pol: int) -> int:
    s = n_inputs // n_pol
    return s * (s + 1) // 2


def correlate(samples: np.ndarray, n_pol: int, threads: int = 1):
    """Full X-engine result for ``samples[T][C][N]``: ``(cross[C][B_s][n_pol^2][2], autos[C][N])``."""
    samples = _check_samples(samples)
    T, C, N = samples.shape
    if n_pol not in (1, 2) or N % n_pol:
        raise ValueError("bad n_pol")
    bs = n_baselines(N, n_pol)
    cross = np.zeros((C, bs, n_pol * n_pol, 2), dtype=np.int64)
    autos = np.zeros((C, N), dtype=np.int64)
    rc = _load().oracle_correlate(_ptr(samples, ctypes.c_uint8), N, C, T, n_pol, _ptr(cross, ctypes.c_int64),
                                  _ptr(autos, ctypes.c_int64), int(threads))
    if rc != 0:
        raise RuntimeError("oracle_correlate failed: %d" % rc)
    return cross, autos


def cells(samples: np.ndarray, cell_list) -> np.ndarray:
    """Visibility cells ``(f, i, j) -> sum_t x_{f,i}(t) conj(x_{f,j}(t))`` as int64 ``[k][2]``."""
    samples = _check_samples(samples)
    T, C, N = samples.shape
    cl = np.ascontiguousarray(np.asarray(cell_list, dtype=np.int32).reshape(-1, 3))
    out = np.zeros((cl.shape[0], 2), dtype=np.int64)
    rc = _load().oracle_cells(_ptr(samples, ctypes.c_uint8), N, C, T, cl.shape[0], _ptr(cl, ctypes.c_int32),
                              _ptr(out, ctypes.c_int64))
    if rc != 0:
        raise RuntimeError("oracle_cells failed: %d" % rc)
    return out


def autos(samples: np.ndarray) -> np.ndarray:
    """Autocorrelations (total power) ``[C][N]`` int64."""
    samples = _check_samples(samples)
    T, C, N = samples.shape
    out = np.zeros((C, N), dtype=np.int64)
    rc = _load().oracle_autos(_ptr(samples, ctypes.c_uint8), N, C, T, _ptr(out, ctypes.c_int64))
    if rc != 0:
        raise RuntimeError("oracle_autos failed: %d" % rc)
    return out


def station_cross(samples: np.ndarray, stations, n_pol: int) -> np.ndarray:
    """Cross cells among a station list, ``[C][n (n + 1) / 2][n_pol^2][2]`` int64, by the cell definition."""
    samples = _check_samples(samples)
    C = samples.shape[1]
    st = [int(v) for v in stations]
    cl = []
    for f in range(C):
        for k in range(len(st)):
            for l in range(k + 1):
                for p in range(n_pol):
                    for q in range(n_pol):
                        cl.append((f, st[k] * n_pol + p, st[l] * n_pol + q))
    npairs = len(st) * (len(st) + 1) // 2
    return cells(samples, cl).reshape(C, npairs, n_pol * n_pol, 2)


def station_autos(samples: np.ndarray, stations, n_pol: int) -> np.ndarray:
    """Autocorrelations of the inputs of a station list, ``[C][n][n_pol]`` int64."""
    a = autos(samples)
    idx = [int(s) * n_pol + p for s in stations for p in range(n_pol)]
    return a[:, idx].reshape(a.shape[0], len(stations), n_pol)


def requantize(x: np.ndarray, chan0: int, n_chans: int, gain: float = 1.0, gains=None,
               symmetric: bool = False) -> np.ndarray:
    """PFB output ``x[N][T][F][2]`` (int32 or float32) -> packed 4+4-bit ``uint8[T][n_chans][N]``."""
    x = np.asarray(x)
    if x.ndim != 4 or x.shape[3] != 2 or x.dtype not in (np.int32, np.float32):
        raise ValueError("x must be [N][T][F][2] int32 or float32")
    # 1) channel selection
    sel = x[:, :, chan0:chan0 + n_chans, :]
    if sel.shape[2] != n_chans:
        raise ValueError("channel range outside the PFB")
    # 2) digital gain: one IEEE single-precision product per component
    g = np.float32(gain) if gains is None else np.asarray(gains, dtype=np.float32)[None, None, :, None]
    with np.errstate(invalid="ignore", over="ignore"):
        xf = (sel.astype(np.float32) * g).astype(np.float32)
    # 3) round to nearest, ties to even; 4) clip; NaN -> 0
    r = np.rint(xf)
    lo = -7.0 if symmetric else -8.0
    r = np.where(np.isnan(r), 0.0, np.clip(r, lo, 7.0)).astype(np.int64)
    # 5) pack Re in the high nibble; 6) corner turn [N][T][C] -> [T][C][N]
    packed = (((r[..., 0] & 0xF) << 4) | (r[..., 1] & 0xF)).astype(np.uint8)
    return np.ascontiguousarray(packed.transpose(1, 2, 0))


def pfb_coeffs(n_fft: int, n_taps: int) -> np.ndarray:
    """Prototype filter ``h[n_taps * n_fft]`` (int64 values of 18-bit range)."""
    L = n_fft * n_taps
    j = np.arange(L, dtype=np.float64)
    w = 0.54 - 0.46 * np.cos(2.0 * np.pi * j / (L - 1)) if L > 1 else np.ones(1)
    h = w * np.sinc((j - 0.5 * (L - 1)) / n_fft)
    s = 131071.0 / np.abs(h).max()
    return np.floor(h * s + 0.5).astype(np.int64)


def pfb_fir(adc: np.ndarray, n_fft: int, n_taps: int, coeffs=None) -> np.ndarray:
    """FIR stage ``y[N][T][n_fft]`` of real samples ``adc[N][S]`` (int64 for integer input, else float64)."""
    adc = np.asarray(adc)
    h = pfb_coeffs(n_fft, n_taps) if coeffs is None else np.asarray(coeffs, dtype=np.int64)
    N, S = adc.shape
    T = S // n_fft - n_taps + 1
    if T < 1:
        raise ValueError("need at least n_taps frames")
    integer = np.issubdtype(adc.dtype, np.integer)
    frames = adc[:, :(T + n_taps - 1) * n_fft].reshape(N, T + n_taps - 1, n_fft)
    frames = frames.astype(np.int64 if integer else np.float64)
    y = np.zeros((N, T, n_fft), dtype=frames.dtype)
    for p in range(n_taps):
        y += frames[:, p:p + T, :] * h[p * n_fft:(p + 1) * n_fft][None, None, :]
    return y


def pfb(adc: np.ndarray, n_fft: int = 8192, n_taps: int = 4, coeffs=None) -> np.ndarray:
    """PFB output ``X[N][T][n_fft / 2]`` complex128: FIR, then the real DFT scaled by 1 / n_fft."""
    y = pfb_fir(adc, n_fft, n_taps, coeffs)
    return np.fft.rfft(y.astype(np.float64), axis=-1)[..., :n_fft // 2] / n_fft


def to_format(values: np.ndarray, fmt: int, n_samples: int) -> np.ndarray:
    """Convert int64 sums to a dump format (CI64 / CF32 / CF32_NORM), element by element."""
    values = np.asarray(values, dtype=np.int64)
    if fmt == FMT_CI64:
        return values.copy()
    if fmt == FMT_CF32:
        return values.astype(np.float32)
    if fmt == FMT_CF32_NORM:
        if n_samples <= 0:
            return np.zeros(values.shape, dtype=np.float32)
        return (values.astype(np.float64) / float(n_samples)).astype(np.float32)
    raise ValueError("unknown format")


def unpack(samples: np.ndarray):
    """Packed bytes -> (re, im) int64 arrays of the same shape (sign-extended nibbles)."""
    s = np.asarray(samples, dtype=np.uint8)
    re = (s >> 4).astype(np.int64)
    im = (s & 0xF).astype(np.int64)
    re = np.where(re >= 8, re - 16, re)
    im = np.where(im >= 8, im - 16, im)
    return re, im


def pack(re, im) -> np.ndarray:
    """(re, im) integers in [-8, 7] -> packed bytes (Re in the high nibble)."""
    re = np.asarray(re, dtype=np.int64)
    im = np.asarray(im, dtype=np.int64)
    if re.min(initial=0) < -8 or re.max(initial=0) > 7 or im.min(initial=0) < -8 or im.max(initial=0) > 7:
        raise ValueError("components must lie in [-8, 7]")
    return (((re & 0xF) << 4) | (im & 0xF)).astype(np.uint8)
