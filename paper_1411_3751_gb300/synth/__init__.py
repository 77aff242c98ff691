"""Seeded synthetic 4+4-bit inputs shaped like the paper's workloads (test and benchmark input only).

The generator is defined in ``synth.h`` and implemented twice: a CUDA kernel (fills device buffers
for the benchmark and the GPU tests) and a plain C function (produces the same bytes on the host for
the oracle). Neither side reads the other's output; ``tests/test_synth.py`` checks they agree.

Workload recipes (the paper's sky data are not available; these take its shapes):

* ``uniform``    each component i.i.d. uniform over [-8, 7];
* ``gauss_tone`` Gaussian-like noise of standard deviation sigma (Irwin-Hall of four 16-bit uniforms)
  plus a common tone A exp(i 2 pi (t + k_n) / 1024) with a seeded per-input phase k_n, quantised by
  rounding and clipped to [-8, 7] (the 4+4-bit requantisation of Sec. 2.2), A^2 = rho 2 sigma^2 / (1 - rho)
  so that the tone's correlation coefficient between inputs is rho;
* ``saturate``   as ``gauss_tone`` but alternating 4096-sample segments use sigma_hi (heavy clipping),
  and one segment is all -8-8i.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_BUILD = os.path.join(_PKG, "_build")

UNIFORM, GAUSS_TONE = 0, 1
NOISE_STD_FIELDS = 65536.0 / math.sqrt(3.0)  # std of the sum of four 16-bit uniform fields


class SynthParams(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("profile", ctypes.c_int32),
        ("unit_lo", ctypes.c_int32),
        ("unit_hi", ctypes.c_int32),
        ("sat_period", ctypes.c_int32),
        ("seg_len", ctypes.c_int32),
        ("m8_segment", ctypes.c_int32),
    ]


@dataclass
class Spec:
    kind: str = "uniform"  # uniform | gauss_tone | saturate
    seed: int = 0x14113751
    sigma: float = 2.5
    sigma_hi: float = 6.0
    rho: float = 0.1
    seg_len: int = 4096
    m8_segment: int = -1

    def params(self) -> SynthParams:
        p = SynthParams()
        p.seed = self.seed & 0xFFFFFFFFFFFFFFFF
        p.profile = UNIFORM if self.kind == "uniform" else GAUSS_TONE
        p.unit_lo = int(round(NOISE_STD_FIELDS / self.sigma))
        p.unit_hi = int(round(NOISE_STD_FIELDS / self.sigma_hi))
        p.sat_period = 2 if self.kind == "saturate" else 0
        p.seg_len = int(self.seg_len)
        p.m8_segment = int(self.m8_segment) if self.kind == "saturate" else -1
        return p

    def tone_amplitude(self) -> float:
        return math.sqrt(self.rho * 2.0 * self.sigma ** 2 / (1.0 - self.rho))

    def tables(self):
        """Tone tables round(A u cos(2 pi p / 1024)) for the low and high units (int32[1024] each)."""
        p = self.params()
        A = self.tone_amplitude()
        ph = np.arange(1024) * (2.0 * np.pi / 1024.0)
        lo = np.round(A * p.unit_lo * np.cos(ph)).astype(np.int32)
        hi = np.round(A * p.unit_hi * np.cos(ph)).astype(np.int32)
        return lo, hi

    def phases(self, n_inputs: int) -> np.ndarray:
        """Per-input tone phase offsets k_n in [0, 1024), from a SplitMix64 draw of (seed ^ salt, n)."""
        return _phase_offsets(self.seed, n_inputs)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(0xBF58476D1CE4E5B9)
        z ^= z >> np.uint64(27)
        z *= np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
    return z


def _phase_offsets(seed: int, n: int) -> np.ndarray:
    s = np.uint64((seed ^ 0x5EED5EED5EED5EED) & 0xFFFFFFFFFFFFFFFF)
    k = np.arange(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = s + (k + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
    return (_mix64(z) >> np.uint64(54)).astype(np.int32)


_host_lib = None
_cuda_lib = None


def _lib_host():
    global _host_lib
    if _host_lib is None:
        path = os.path.join(_BUILD, "libcorrsynth_host.so")
        if not os.path.exists(path):
            from .. import _build

            _build.build()
        lib = ctypes.CDLL(path)
        lib.synth_generate_host.restype = ctypes.c_int
        lib.synth_generate_host.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, ctypes.c_longlong, ctypes.POINTER(SynthParams),
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        _host_lib = lib
    return _host_lib


def _lib_cuda():
    global _cuda_lib
    if _cuda_lib is None:
        path = os.path.join(_BUILD, "libcorrsynth_cuda.so")
        if not os.path.exists(path):
            raise OSError("generator library not built (%s missing)" % path)
        lib = ctypes.CDLL(path)
        lib.synth_generate_device.restype = ctypes.c_int
        lib.synth_generate_device.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_longlong, ctypes.POINTER(SynthParams), ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.synth_generate_device_range.restype = ctypes.c_int
        lib.synth_generate_device_range.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                    ctypes.c_int, ctypes.c_int, ctypes.c_longlong,
                                                    ctypes.POINTER(SynthParams), ctypes.c_void_p, ctypes.c_void_p,
                                                    ctypes.c_void_p, ctypes.c_void_p]
        _cuda_lib = lib
    return _cuda_lib


def generate_host(spec: Spec, T: int, C: int, N: int, t0: int = 0, t_range=None, c_range=None) -> np.ndarray:
    """uint8 [t][c][N] for times t0 + t_range and channels c_range of a C-channel array."""
    tb, tn = (0, T) if t_range is None else (t_range[0], t_range[1] - t_range[0])
    cb, cn = (0, C) if c_range is None else (c_range[0], c_range[1] - c_range[0])
    out = np.zeros((tn, cn, N), dtype=np.uint8)
    lo, hi = spec.tables()
    k = spec.phases(N)
    p = spec.params()
    rc = _lib_host().synth_generate_host(out.ctypes.data, tb, tn, cb, cn, C, N, t0, ctypes.byref(p),
                                         lo.ctypes.data, hi.ctypes.data, k.ctypes.data)
    if rc != 0:
        raise ValueError("synth_generate_host rejected the parameters")
    return out


_device_tables = {}


def _tables_on_device(spec: Spec, N: int):
    """Tone tables and phase offsets on the device, cached per (spec, N) so launches need no sync."""
    import torch

    key = (spec.kind, spec.seed, spec.sigma, spec.sigma_hi, spec.rho, N, torch.cuda.current_device())
    t = _device_tables.get(key)
    if t is None:
        lo, hi = spec.tables()
        k = spec.phases(N)
        t = (torch.from_numpy(lo).cuda(), torch.from_numpy(hi).cuda(), torch.from_numpy(k).cuda())
        torch.cuda.synchronize()
        _device_tables[key] = t
    return t


def generate_device(spec: Spec, T: int, C: int, N: int, t0: int = 0, out=None, stream=None, sync: bool = True,
                    c_range=None):
    """torch.uint8 cuda tensor [T][C][N], or [T][c1 - c0][N] holding channels c_range = (c0, c1) of a
    C-channel array (written on the given or current stream; sync=False returns without waiting for
    the kernel)."""
    import torch

    cb, cn = (0, C) if c_range is None else (c_range[0], c_range[1] - c_range[0])
    if out is None:
        out = torch.empty((T, cn, N), dtype=torch.uint8, device="cuda")
    d_lo, d_hi, d_k = _tables_on_device(spec, N)
    s = stream if stream is not None else torch.cuda.current_stream()
    p = spec.params()
    rc = _lib_cuda().synth_generate_device_range(out.data_ptr(), T, cb, cn, C, N, t0, ctypes.byref(p), d_lo.data_ptr(),
                                                 d_hi.data_ptr(), d_k.data_ptr(), int(s.cuda_stream))
    if rc != 0:
        raise RuntimeError("synth_generate_device failed: %d" % rc)
    if sync:
        s.synchronize()
    return out


def phases_radians(spec: Spec, n_inputs: int) -> np.ndarray:
    return spec.phases(n_inputs).astype(np.float64) * (2.0 * np.pi / 1024.0)
