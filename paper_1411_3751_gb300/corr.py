"""Python binding of libcorr's C ABI (include/corr.h): argument marshalling only.

Every function here has the name of the C entry point it calls and takes plain integers and
pointers. :class:`Correlator` adds torch-tensor marshalling on top (data pointers, the current CUDA
stream); all work runs in the library's CUDA kernels. There is no fallback: if the library cannot
be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libcorr.so")

CORR_OK = 0
CORR_ERR_ARG, CORR_ERR_CUDA, CORR_ERR_OOM, CORR_ERR_STATE, CORR_ERR_TIMEOUT, CORR_ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -6
CORR_PATH_AUTO, CORR_PATH_FP32, CORR_PATH_I8MMA, CORR_PATH_FP8TC, CORR_PATH_FP8TC_FUSED = 0, 1, 2, 3, 4
CORR_WHAT_CROSS, CORR_WHAT_AUTO = 1, 2
CORR_FMT_CI64, CORR_FMT_CF32, CORR_FMT_CF32_NORM = 0, 1, 2
CORR_KERNEL_XENG, CORR_KERNEL_UNPACK, CORR_KERNEL_AUTOS, CORR_KERNEL_DUMP = 0, 1, 2, 3

PATHS = {"auto": CORR_PATH_AUTO, "fp32": CORR_PATH_FP32, "i8mma": CORR_PATH_I8MMA, "fp8tc": CORR_PATH_FP8TC,
         "fp8tc_fused": CORR_PATH_FP8TC_FUSED}

# (name, restype, argtypes) of every symbol include/corr.h declares
_c_int, _c_ll, _c_sz, _c_vp, _c_cp = ctypes.c_int, ctypes.c_longlong, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_char_p
SIGNATURES = [
    ("corr_create", _c_vp, [_c_int, _c_int, _c_int, _c_int]),
    ("corr_set_path", _c_int, [_c_vp, _c_int]),
    ("corr_get_path", _c_int, [_c_vp]),
    ("corr_set_tile_plan", _c_int, [_c_vp, _c_int]),
    ("corr_get_tile_plan", _c_int, [_c_vp]),
    ("corr_tile_plan", _c_int, [_c_int, _c_int, _c_vp, _c_int]),
    ("corr_channel_group", _c_int, [_c_int, _c_int]),
    ("corr_set_prep_sms", _c_int, [_c_vp, _c_int]),
    ("corr_get_prep_sms", _c_int, [_c_vp]),
    ("corr_set_batch_blocks", _c_int, [_c_vp, _c_int]),
    ("corr_get_batch_blocks", _c_int, [_c_vp]),
    ("corr_autotune", _c_int, [_c_vp, ctypes.POINTER(ctypes.c_void_p), _c_int, _c_int, _c_vp, _c_vp]),
    ("corr_set_flush_period", _c_int, [_c_vp, _c_int]),
    ("corr_accumulate", _c_int, [_c_vp, _c_vp, _c_vp]),
    ("corr_accumulate_batch", _c_int, [_c_vp, ctypes.POINTER(ctypes.c_void_p), _c_int, _c_vp]),
    ("corr_accumulate_host", _c_int, [_c_vp, _c_vp, _c_vp]),
    ("corr_accumulate_autos", _c_int, [_c_vp, _c_vp, _c_vp]),
    ("corr_dump", _c_int, [_c_vp, _c_vp, _c_int, _c_int, _c_int, _c_int, _c_vp]),
    ("corr_dump_stations", _c_int, [_c_vp, _c_vp, _c_int, _c_vp, _c_int, _c_int, _c_int, _c_int, _c_vp]),
    ("corr_pfb_coeffs", _c_int, [_c_int, _c_int, _c_vp]),
    ("corr_pfb", _c_int, [_c_vp, _c_int, ctypes.c_longlong, ctypes.c_longlong, _c_int, _c_vp, _c_int, _c_vp, _c_vp]),
    ("corr_requantize", _c_int, [_c_vp, _c_int, _c_int, _c_int, _c_int, _c_int, _c_int, ctypes.c_float, _c_vp,
                                 _c_int, _c_vp, _c_vp]),
    ("corr_corner_turn_pack", _c_int, [_c_vp, _c_int, _c_int, _c_int, ctypes.POINTER(ctypes.c_int), _c_int, _c_vp,
                                       _c_vp]),
    ("corr_corner_turn_unpack", _c_int, [_c_vp, _c_int, _c_int, _c_int, ctypes.POINTER(ctypes.c_int), _c_int, _c_vp,
                                         _c_vp]),
    ("corr_samples_accumulated", _c_ll, [_c_vp, _c_int]),
    ("corr_reset", _c_int, [_c_vp, _c_int, _c_vp]),
    ("corr_sync", _c_int, [_c_vp, _c_vp]),
    ("corr_selftest_wait", _c_int, [_c_vp, _c_int, _c_vp]),
    ("corr_footprint_bytes", _c_sz, [_c_int, _c_int, _c_int, _c_int, _c_int]),
    ("corr_n_baselines", _c_ll, [_c_int, _c_int]),
    ("corr_batch_blocks", _c_int, [_c_int, _c_int, _c_int, _c_int]),
    ("corr_profile_enable", _c_int, [_c_vp, _c_int]),
    ("corr_profile_read", _c_int, [_c_vp, _c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]),
    ("corr_group_create", _c_vp, [_c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _c_int, _c_int]),
    ("corr_group_member", _c_vp, [_c_vp, _c_int]),
    ("corr_group_accumulate", _c_int, [_c_vp, ctypes.POINTER(ctypes.c_void_p), _c_int, _c_vp]),
    ("corr_group_autotune", _c_int, [_c_vp, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int), _c_vp]),
    ("corr_group_capture", _c_int, [_c_vp, ctypes.POINTER(ctypes.c_void_p), _c_vp]),
    ("corr_group_launch", _c_int, [_c_vp, _c_vp]),
    ("corr_group_destroy", _c_int, [_c_vp]),
    ("corr_xengine_static", _c_int, [_c_vp, _c_int, _c_int, _c_int, _c_int, _c_vp, _c_vp, _c_vp]),
    ("corr_xengine_static_status", _c_int, [ctypes.POINTER(ctypes.c_int), _c_vp]),
    ("corr_xengine_static_selftest_wait", _c_int, [_c_int, _c_vp]),
    ("corr_probe_mma_rate", _c_int, [_c_int, _c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                     _c_vp]),
    ("corr_destroy", _c_int, [_c_vp]),
    ("corr_last_error", _c_cp, []),
    ("corr_version", _c_cp, []),
]


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libcorr and attach the C signatures. Raises OSError if it is missing."""
    if not os.path.exists(path):
        raise OSError("libcorr is not built (%s missing): run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = load()


class CorrError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = corr_last_error()
        super().__init__("%s failed (%d): %s" % (where, code, msg))
        self.code = code


def _check(rc: int, where: str) -> int:
    if rc < 0:
        raise CorrError(rc, where)
    return rc


# ---- C entry points, same names ---------------------------------------------------------------
def corr_create(n_inputs: int, n_chans: int, n_time_per_block: int, n_pol: int) -> int:
    h = _lib.corr_create(n_inputs, n_chans, n_time_per_block, n_pol)
    if not h:
        raise CorrError(CORR_ERR_ARG, "corr_create")
    return h


def corr_set_path(ctx: int, path: int) -> int:
    return _check(_lib.corr_set_path(ctx, path), "corr_set_path")


def corr_get_path(ctx: int) -> int:
    return _check(_lib.corr_get_path(ctx), "corr_get_path")


def corr_set_tile_plan(ctx: int, plan: int) -> int:
    return _check(_lib.corr_set_tile_plan(ctx, plan), "corr_set_tile_plan")


def corr_get_tile_plan(ctx: int) -> int:
    return _check(_lib.corr_get_tile_plan(ctx), "corr_get_tile_plan")


def corr_tile_plan(n_inputs: int, plan: int):
    """Work items of one channel as a list of (c0, a0, nb, extra) (host only)."""
    n = _check(_lib.corr_tile_plan(n_inputs, plan, None, 0), "corr_tile_plan")
    buf = (ctypes.c_int * (4 * max(n, 1)))()
    _check(_lib.corr_tile_plan(n_inputs, plan, buf, n), "corr_tile_plan")
    return [tuple(buf[4 * i:4 * i + 4]) for i in range(n)]


def corr_channel_group(n_inputs: int, plan: int) -> int:
    """Channels per work item of the two-pass tensor path (host only): 4, 2 or 1."""
    return _check(_lib.corr_channel_group(n_inputs, plan), "corr_channel_group")


def corr_set_prep_sms(ctx: int, sms: int) -> int:
    return _check(_lib.corr_set_prep_sms(ctx, sms), "corr_set_prep_sms")


def corr_get_prep_sms(ctx: int) -> int:
    return _check(_lib.corr_get_prep_sms(ctx), "corr_get_prep_sms")


def corr_set_batch_blocks(ctx: int, blocks: int) -> int:
    return _check(_lib.corr_set_batch_blocks(ctx, blocks), "corr_set_batch_blocks")


def corr_get_batch_blocks(ctx: int) -> int:
    return _check(_lib.corr_get_batch_blocks(ctx), "corr_get_batch_blocks")


class CorrTuning(ctypes.Structure):
    _fields_ = [("tile_plan", ctypes.c_int), ("batch_blocks", ctypes.c_int), ("prep_sms", ctypes.c_int),
                ("n_tried", ctypes.c_int), ("ms_per_block", ctypes.c_double)]


def corr_autotune(ctx: int, d_blocks, reps: int, stream: int) -> dict:
    """Time the batch schedules on the given device blocks, keep the fastest; returns the choice."""
    arr = (ctypes.c_void_p * len(d_blocks))(*[int(p) for p in d_blocks])
    t = CorrTuning()
    _check(_lib.corr_autotune(ctx, arr, len(d_blocks), reps, ctypes.byref(t), stream), "corr_autotune")
    return {"tile_plan": t.tile_plan, "batch_blocks": t.batch_blocks, "prep_sms": t.prep_sms, "n_tried": t.n_tried,
            "ms_per_block": t.ms_per_block}


def corr_set_flush_period(ctx: int, n_samples: int) -> int:
    return _check(_lib.corr_set_flush_period(ctx, n_samples), "corr_set_flush_period")


def corr_accumulate(ctx: int, d_samples: int, stream: int) -> int:
    return _check(_lib.corr_accumulate(ctx, d_samples, stream), "corr_accumulate")


def corr_accumulate_batch(ctx: int, d_blocks, stream: int) -> int:
    arr = (ctypes.c_void_p * len(d_blocks))(*[int(p) for p in d_blocks])
    return _check(_lib.corr_accumulate_batch(ctx, arr, len(d_blocks), stream), "corr_accumulate_batch")


def corr_accumulate_host(ctx: int, h_samples: int, stream: int) -> int:
    return _check(_lib.corr_accumulate_host(ctx, h_samples, stream), "corr_accumulate_host")


def corr_accumulate_autos(ctx: int, d_samples: int, stream: int) -> int:
    return _check(_lib.corr_accumulate_autos(ctx, d_samples, stream), "corr_accumulate_autos")


def corr_dump(ctx: int, out: int, is_device_ptr: int, what: int, fmt: int, reset: int, stream: int) -> int:
    return _check(_lib.corr_dump(ctx, out, is_device_ptr, what, fmt, reset, stream), "corr_dump")


CORR_IN_CI32, CORR_IN_CF32 = 0, 1


def corr_requantize(d_in: int, in_type: int, n_inputs: int, n_time: int, n_pfb_chans: int, chan0: int, n_chans: int,
                    gain: float, d_gains: int, symmetric: int, d_out: int, stream: int) -> int:
    return _check(_lib.corr_requantize(d_in, in_type, n_inputs, n_time, n_pfb_chans, chan0, n_chans, gain, d_gains,
                                       symmetric, d_out, stream), "corr_requantize")


def requantize(x, chan0: int, n_chans: int, gain: float = 1.0, gains=None, symmetric: bool = False, out=None,
               stream=None):
    """torch wrapper: x is a cuda tensor [N][T][F][2] of int32 or float32; returns uint8 [T][n_chans][N]."""
    import torch

    if not x.is_cuda or x.dim() != 4 or x.shape[3] != 2 or not x.is_contiguous():
        raise ValueError("x must be a contiguous cuda tensor [N][T][F][2]")
    if x.dtype == torch.int32:
        in_type = CORR_IN_CI32
    elif x.dtype == torch.float32:
        in_type = CORR_IN_CF32
    else:
        raise ValueError("x must be int32 or float32")
    N, T, F = x.shape[0], x.shape[1], x.shape[2]
    if out is None:
        out = torch.empty((T, n_chans, N), dtype=torch.uint8, device=x.device)
    if gains is not None and (not gains.is_cuda or gains.dtype != torch.float32 or gains.numel() != n_chans):
        raise ValueError("gains must be a cuda float32 tensor of n_chans values")
    corr_requantize(x.data_ptr(), in_type, N, T, F, chan0, n_chans, float(gain),
                    gains.data_ptr() if gains is not None else None, 1 if symmetric else 0, out.data_ptr(),
                    _stream_handle(stream))
    return out


def corr_pfb_coeffs(n_fft: int, n_taps: int):
    """Prototype filter of the PFB as a numpy int32 array [n_taps * n_fft] (computed by the library)."""
    import numpy as np

    h = np.zeros(n_fft * n_taps, dtype=np.int32)
    _check(_lib.corr_pfb_coeffs(n_fft, n_taps, h.ctypes.data), "corr_pfb_coeffs")
    return h


def corr_pfb(d_adc: int, n_inputs: int, input_stride: int, n_samples: int, n_taps: int, d_coeffs: int,
             n_spectra: int, d_out: int, stream: int) -> int:
    return _check(_lib.corr_pfb(d_adc, n_inputs, input_stride, n_samples, n_taps, d_coeffs, n_spectra, d_out, stream),
                  "corr_pfb")


PFB_FFT = 8192
_pfb_coeff_cache = {}


def pfb(adc, n_taps: int = 4, coeffs=None, out=None, stream=None):
    """torch wrapper: adc is a cuda int8 tensor [N][S] of real samples; returns float32 [N][T][4096][2]
    with T = S // 8192 - n_taps + 1 spectra (corr_pfb)."""
    import torch

    if not adc.is_cuda or adc.dtype != torch.int8 or adc.dim() != 2 or adc.stride(1) != 1:
        raise ValueError("adc must be a cuda int8 tensor [N][S] with contiguous rows")
    N, S = adc.shape
    T = S // PFB_FFT - n_taps + 1
    if T < 1:
        raise ValueError("need at least n_taps frames of 8192 samples")
    if coeffs is None:
        key = (n_taps, adc.device.index)
        coeffs = _pfb_coeff_cache.get(key)
        if coeffs is None:
            coeffs = torch.from_numpy(corr_pfb_coeffs(PFB_FFT, n_taps)).to(adc.device)
            _pfb_coeff_cache[key] = coeffs
    if out is None:
        out = torch.empty((N, T, PFB_FFT // 2, 2), dtype=torch.float32, device=adc.device)
    stride = adc.stride(0) if N > 1 else S  # a single row may carry any stride (e.g. a broadcast view)
    corr_pfb(adc.data_ptr(), N, stride, S, n_taps, coeffs.data_ptr(), T, out.data_ptr(), _stream_handle(stream))
    return out


def corr_dump_stations(ctx: int, stations, n_stations: int, out: int, is_device_ptr: int, what: int, fmt: int,
                       reset: int, stream: int) -> int:
    """`stations`: a host int32 buffer address (or a sequence of ints, marshalled here)."""
    if not isinstance(stations, int):
        arr = (ctypes.c_int * len(stations))(*[int(v) for v in stations])
        stations = ctypes.addressof(arr)
    return _check(_lib.corr_dump_stations(ctx, stations, n_stations, out, is_device_ptr, what, fmt, reset, stream),
                  "corr_dump_stations")


def corr_corner_turn_pack(d_in: int, n_time: int, n_chans: int, n_local: int, chan_bounds, d_out: int,
                          stream: int) -> int:
    b = (ctypes.c_int * len(chan_bounds))(*[int(v) for v in chan_bounds])
    return _check(_lib.corr_corner_turn_pack(d_in, n_time, n_chans, n_local, b, len(chan_bounds) - 1, d_out, stream),
                  "corr_corner_turn_pack")


def corr_corner_turn_unpack(d_in: int, n_time: int, n_chans: int, n_inputs: int, input_bounds, d_out: int,
                            stream: int) -> int:
    b = (ctypes.c_int * len(input_bounds))(*[int(v) for v in input_bounds])
    return _check(_lib.corr_corner_turn_unpack(d_in, n_time, n_chans, n_inputs, b, len(input_bounds) - 1, d_out,
                                               stream), "corr_corner_turn_unpack")


def corr_samples_accumulated(ctx: int, what: int) -> int:
    return _check(_lib.corr_samples_accumulated(ctx, what), "corr_samples_accumulated")


def corr_reset(ctx: int, what: int, stream: int) -> int:
    return _check(_lib.corr_reset(ctx, what, stream), "corr_reset")


def corr_sync(ctx: int, stream: int) -> int:
    return _check(_lib.corr_sync(ctx, stream), "corr_sync")


def corr_selftest_wait(ctx: int, limit_ms: int, stream: int) -> int:
    return _check(_lib.corr_selftest_wait(ctx, limit_ms, stream), "corr_selftest_wait")


def corr_footprint_bytes(n_inputs: int, n_chans: int, n_time_per_block: int, n_pol: int, path: int) -> int:
    return int(_lib.corr_footprint_bytes(n_inputs, n_chans, n_time_per_block, n_pol, path))


def corr_n_baselines(n_inputs: int, n_pol: int) -> int:
    return int(_lib.corr_n_baselines(n_inputs, n_pol))


def corr_batch_blocks(n_inputs: int, n_chans: int, n_time_per_block: int, n_pol: int) -> int:
    """Blocks per tensor-core launch of corr_accumulate_batch for this shape (0 if invalid)."""
    return int(_lib.corr_batch_blocks(n_inputs, n_chans, n_time_per_block, n_pol))


def corr_profile_enable(ctx: int, on: int) -> int:
    return _check(_lib.corr_profile_enable(ctx, on), "corr_profile_enable")


def corr_profile_read(ctx: int, kernel: int):
    """Returns (total_ms, launches) recorded for `kernel` since the last read."""
    ms = ctypes.c_double(0.0)
    n = ctypes.c_longlong(0)
    _check(_lib.corr_profile_read(ctx, kernel, ctypes.byref(ms), ctypes.byref(n)), "corr_profile_read")
    return ms.value, n.value


def corr_xengine_static(d_samples: int, n_inputs: int, n_chans: int, n_time: int, n_pol: int, d_cross: int,
                        d_autos: int, stream: int) -> int:
    """Allocation-free tensor-path X-engine for one block (adds into d_cross / d_autos)."""
    return _check(_lib.corr_xengine_static(d_samples, n_inputs, n_chans, n_time, n_pol, d_cross, d_autos, stream),
                  "corr_xengine_static")


def corr_probe_mma_rate(n_mma: int, n_cols: int, stream: int):
    """Issue rate of the X-engine's tcgen05 MMA with no operand traffic: (TFLOP/s, cycles per MMA)."""
    tf = ctypes.c_double(0.0)
    cyc = ctypes.c_double(0.0)
    _check(_lib.corr_probe_mma_rate(n_mma, n_cols, ctypes.byref(tf), ctypes.byref(cyc), stream), "corr_probe_mma_rate")
    return tf.value, cyc.value


def corr_xengine_static_status(stream: int) -> int:
    """The error word the last corr_xengine_static call left (0 if none; a bounded-wait timeout code
    otherwise), cleared by the call; raises CorrError on a CUDA error."""
    code = ctypes.c_int(0)
    rc = _lib.corr_xengine_static_status(ctypes.byref(code), stream)
    if rc < 0 and rc != CORR_ERR_TIMEOUT:
        raise CorrError(rc, "corr_xengine_static_status")
    return code.value


def corr_xengine_static_selftest_wait(limit_ms: int, stream: int) -> int:
    return _check(_lib.corr_xengine_static_selftest_wait(limit_ms, stream), "corr_xengine_static_selftest_wait")


def _ptr_array(ptrs):
    return (ctypes.c_void_p * len(ptrs))(*[int(p) for p in ptrs])


def corr_group_create(n_inputs, n_chans, n_time_per_block: int, n_pol: int) -> int:
    n = len(n_inputs)
    h = _lib.corr_group_create(n, (ctypes.c_int * n)(*n_inputs), (ctypes.c_int * n)(*n_chans), n_time_per_block, n_pol)
    if not h:
        raise CorrError(CORR_ERR_ARG, "corr_group_create")
    return h


def corr_group_member(group: int, i: int) -> int:
    h = _lib.corr_group_member(group, i)
    if not h:
        raise CorrError(CORR_ERR_ARG, "corr_group_member")
    return h


def corr_group_accumulate(group: int, d_samples, mode: int, stream: int) -> int:
    return _check(_lib.corr_group_accumulate(group, _ptr_array(d_samples), mode, stream), "corr_group_accumulate")


def corr_group_autotune(group: int, d_samples, stream: int):
    plans = (ctypes.c_int * len(d_samples))()
    _check(_lib.corr_group_autotune(group, _ptr_array(d_samples), plans, stream), "corr_group_autotune")
    return list(plans)


def corr_group_capture(group: int, d_samples, stream: int) -> int:
    return _check(_lib.corr_group_capture(group, _ptr_array(d_samples), stream), "corr_group_capture")


def corr_group_launch(group: int, stream: int) -> int:
    return _check(_lib.corr_group_launch(group, stream), "corr_group_launch")


def corr_group_destroy(group: int) -> int:
    return _check(_lib.corr_group_destroy(group), "corr_group_destroy")


def corr_destroy(ctx: int) -> int:
    return _check(_lib.corr_destroy(ctx), "corr_destroy")


def corr_last_error() -> str:
    return (_lib.corr_last_error() or b"").decode()


def corr_version() -> str:
    return (_lib.corr_version() or b"").decode()


# ---- torch marshalling ---------------------------------------------------------------------
def _stream_handle(stream) -> int:
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Correlator:
    """Owns one libcorr context (or wraps a group member); passes torch tensors' pointers and the
    current stream."""

    def __init__(self, n_inputs: int, n_chans: int, n_time_per_block: int, n_pol: int = 2, path: str = "auto",
                 _handle: int = 0):
        self.n_inputs, self.n_chans, self.n_time, self.n_pol = n_inputs, n_chans, n_time_per_block, n_pol
        self.n_baselines = corr_n_baselines(n_inputs, n_pol)
        self._owned = not _handle
        self.ctx = _handle or corr_create(n_inputs, n_chans, n_time_per_block, n_pol)
        if self._owned:
            self.set_path(path)

    def set_path(self, path: str):
        corr_set_path(self.ctx, PATHS[path])

    def set_flush_period(self, n: int):
        corr_set_flush_period(self.ctx, n)

    def set_prep_sms(self, sms: int):
        """SMs that build the next launch's operand beside the X-engine in batches (-1 auto, 0 none)."""
        corr_set_prep_sms(self.ctx, sms)

    @property
    def prep_sms(self) -> int:
        return corr_get_prep_sms(self.ctx)

    def set_batch_blocks(self, blocks: int):
        """Blocks per tensor-core launch of batches (0: the default)."""
        corr_set_batch_blocks(self.ctx, blocks)

    @property
    def batch_blocks(self) -> int:
        return corr_get_batch_blocks(self.ctx)

    def autotune(self, blocks, reps: int = 2, stream=None) -> dict:
        """Time the batch schedules on these device blocks and keep the fastest (accumulators end at zero)."""
        for b in blocks:
            self._check_samples(b, True)
        return corr_autotune(self.ctx, [b.data_ptr() for b in blocks], reps, _stream_handle(stream))

    def set_tile_plan(self, plan: int):
        """Work-item plan of the two-pass tensor path (0: 64 x 128-input tiles, 1: 64 x 64, 2: c-block
        pairs, 3: 128 x 128-input tiles on SM pairs; a new context starts on 3 from 512 inputs, else 0)."""
        corr_set_tile_plan(self.ctx, plan)

    @property
    def tile_plan(self) -> int:
        return corr_get_tile_plan(self.ctx)

    @property
    def path(self) -> int:
        return corr_get_path(self.ctx)

    def _check_samples(self, x, device: bool):
        import torch

        if x.dtype != torch.uint8 or tuple(x.shape) != (self.n_time, self.n_chans, self.n_inputs):
            raise ValueError("samples must be uint8 [T][C][N] = %s" % ((self.n_time, self.n_chans, self.n_inputs),))
        if not x.is_contiguous():
            raise ValueError("samples must be contiguous")
        if x.is_cuda != device:
            raise ValueError("samples must be on the %s" % ("device" if device else "host"))

    def accumulate(self, samples, stream=None):
        self._check_samples(samples, True)
        corr_accumulate(self.ctx, samples.data_ptr(), _stream_handle(stream))

    def accumulate_batch(self, blocks, stream=None):
        for b in blocks:
            self._check_samples(b, True)
        corr_accumulate_batch(self.ctx, [b.data_ptr() for b in blocks], _stream_handle(stream))

    def accumulate_host(self, samples, stream=None):
        self._check_samples(samples, False)
        corr_accumulate_host(self.ctx, samples.data_ptr(), _stream_handle(stream))

    def accumulate_autos(self, samples, stream=None):
        self._check_samples(samples, True)
        corr_accumulate_autos(self.ctx, samples.data_ptr(), _stream_handle(stream))

    def out_shape(self, what: int):
        if what == CORR_WHAT_CROSS:
            return (self.n_chans, self.n_baselines, self.n_pol * self.n_pol, 2)
        return (self.n_chans, self.n_inputs)

    def dump(self, what: int = CORR_WHAT_CROSS, fmt: int = CORR_FMT_CI64, reset: bool = False, out=None,
             device: bool = True, stream=None):
        """Snapshot the accumulators into a new (or given) tensor on the device or the host."""
        import torch

        dtype = torch.int64 if fmt == CORR_FMT_CI64 else torch.float32
        shape = self.out_shape(what)
        if out is None:
            out = torch.empty(shape, dtype=dtype, device="cuda" if device else "cpu",
                              pin_memory=(not device))
        if out.dtype != dtype or tuple(out.shape) != shape or not out.is_contiguous():
            raise ValueError("bad output tensor")
        corr_dump(self.ctx, out.data_ptr(), 1 if out.is_cuda else 0, what, fmt, 1 if reset else 0,
                  _stream_handle(stream))
        return out

    def station_out_shape(self, what: int, n_stations: int):
        if what == CORR_WHAT_CROSS:
            return (self.n_chans, n_stations * (n_stations + 1) // 2, self.n_pol * self.n_pol, 2)
        return (self.n_chans, n_stations, self.n_pol)

    def dump_stations(self, stations, what: int = CORR_WHAT_AUTO, fmt: int = CORR_FMT_CI64, reset: bool = False,
                      out=None, device: bool = True, stream=None):
        """Snapshot (and with reset, zero) only the cells among `stations` (a list of station indices)."""
        import torch

        stations = [int(v) for v in stations]
        dtype = torch.int64 if fmt == CORR_FMT_CI64 else torch.float32
        shape = self.station_out_shape(what, len(stations))
        if out is None:
            out = torch.empty(shape, dtype=dtype, device="cuda" if device else "cpu", pin_memory=(not device))
        if out.dtype != dtype or tuple(out.shape) != shape or not out.is_contiguous():
            raise ValueError("bad output tensor")
        corr_dump_stations(self.ctx, stations, len(stations), out.data_ptr(), 1 if out.is_cuda else 0, what, fmt,
                           1 if reset else 0, _stream_handle(stream))
        return out

    def reset(self, what: int = CORR_WHAT_CROSS | CORR_WHAT_AUTO, stream=None):
        corr_reset(self.ctx, what, _stream_handle(stream))

    def samples(self, what: int = CORR_WHAT_CROSS) -> int:
        return corr_samples_accumulated(self.ctx, what)

    def sync(self, stream=None):
        corr_sync(self.ctx, _stream_handle(stream))

    def profile(self, on: bool = True):
        corr_profile_enable(self.ctx, 1 if on else 0)

    def profile_read(self, kernel: int):
        return corr_profile_read(self.ctx, kernel)

    def close(self):
        if self.ctx and self._owned:
            corr_destroy(self.ctx)
        self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Group:
    """A group of sub-arrays correlated with one persistent tensor-core launch (corr_group_*)."""

    def __init__(self, shapes, n_time_per_block: int, n_pol: int = 2):
        self.shapes = [(int(n), int(c)) for n, c in shapes]
        self.n_time, self.n_pol = n_time_per_block, n_pol
        self.handle = corr_group_create([n for n, _ in self.shapes], [c for _, c in self.shapes], n_time_per_block, n_pol)
        self.members = [Correlator(n, c, n_time_per_block, n_pol, _handle=corr_group_member(self.handle, i))
                        for i, (n, c) in enumerate(self.shapes)]

    def _ptrs(self, blocks):
        assert len(blocks) == len(self.shapes)
        for m, b in zip(self.members, blocks):
            m._check_samples(b, True)
        return [b.data_ptr() for b in blocks]

    def accumulate(self, blocks, separate: bool = False, stream=None):
        corr_group_accumulate(self.handle, self._ptrs(blocks), 1 if separate else 0, _stream_handle(stream))

    def autotune(self, blocks, stream=None):
        return corr_group_autotune(self.handle, self._ptrs(blocks), _stream_handle(stream))

    def capture(self, blocks, stream):
        corr_group_capture(self.handle, self._ptrs(blocks), _stream_handle(stream))

    def launch(self, stream=None):
        corr_group_launch(self.handle, _stream_handle(stream))

    def close(self):
        if self.handle:
            for m in self.members:
                m.ctx = None
            corr_group_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
