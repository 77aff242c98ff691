"""corr_xengine_static: the allocation-free entry point, for callers that cannot call cudaMalloc while
they correlate (code running inside another runtime's memory pool or arena, or a real-time pipeline
that forbids allocation once it has started). Its scratch is a fixed device array inside the library.

Checked on two calls in a row into the same output buffers (the second call adds the second block):
against the CPU oracle and against the context entry points (corr_create / corr_accumulate /
corr_dump), with the device's free memory unchanged across the second call; at the largest shape its
fixed array admits, and past it; its error word through the status call and the bounded-wait
self-test; and in a second CUDA context, where the array lives at another address.

Collected last on purpose (file name), so a stop-at-first-failure run has already run every other
test before this one.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import oracle

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1411_3751_gb300 import corr, synth

    assert torch.cuda.is_available()
    return corr, synth, torch


# (N, C, T, n_pol); 512 x 7 x 8192 is the largest 512-input block the 64 MiB array admits
SHAPES = [(64, 4, 1000, 2), (200, 3, 300, 1), (512, 7, 8192, 2)]


@pytest.mark.parametrize("shape", SHAPES)
def test_static_matches_oracle_and_context_path_on_two_calls(env, shape):
    corr, synth, torch = env
    N, C, T, npol = shape
    spec = synth.Spec(kind="gauss_tone", seed=N + C + T)
    h1 = synth.generate_host(spec, T, C, N, t0=0)
    h2 = synth.generate_host(spec, T, C, N, t0=T)
    b1, b2 = torch.from_numpy(h1).cuda(), torch.from_numpy(h2).cuda()
    with corr.Correlator(N, C, T, npol) as xc:
        xc.accumulate(b1)
        ctx_c1, ctx_a1 = xc.dump(corr.CORR_WHAT_CROSS), xc.dump(corr.CORR_WHAT_AUTO)
        xc.accumulate(b2)
        ctx_c2, ctx_a2 = xc.dump(corr.CORR_WHAT_CROSS), xc.dump(corr.CORR_WHAT_AUTO)
        xc.sync()
    cross = torch.zeros_like(ctx_c1)
    autos = torch.zeros_like(ctx_a1)
    stream = torch.cuda.current_stream().cuda_stream
    corr.corr_xengine_static(b1.data_ptr(), N, C, T, npol, cross.data_ptr(), autos.data_ptr(), stream)
    torch.cuda.synchronize()
    got_c1, got_a1 = cross.cpu().numpy(), autos.cpu().numpy()
    free_before = torch.cuda.mem_get_info()[0]
    corr.corr_xengine_static(b2.data_ptr(), N, C, T, npol, cross.data_ptr(), autos.data_ptr(), stream)
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    assert free_after == free_before, "device memory changed across a call: %d -> %d" % (free_before, free_after)
    assert corr.corr_xengine_static_status(stream) == 0
    got_c2, got_a2 = cross.cpu().numpy(), autos.cpu().numpy()
    # the existing entry points, cell by cell
    assert np.array_equal(got_c1, ctx_c1.cpu().numpy()) and np.array_equal(got_a1, ctx_a1.cpu().numpy())
    assert np.array_equal(got_c2, ctx_c2.cpu().numpy()) and np.array_equal(got_a2, ctx_a2.cpu().numpy())
    # the oracle: the first block, then both blocks
    want_c1, want_a1 = oracle.correlate(h1, npol, threads=8)
    assert np.array_equal(got_c1, want_c1) and np.array_equal(got_a1, want_a1)
    want_c2, want_a2 = oracle.correlate(np.concatenate([h1, h2]), npol, threads=8)
    assert np.array_equal(got_c2, want_c2) and np.array_equal(got_a2, want_a2)


def test_static_rejects_sizes_beyond_its_scratch(env):
    corr, _, torch = env
    x = torch.zeros(8, dtype=torch.uint8, device="cuda")
    out = torch.zeros(8, dtype=torch.int64, device="cuda")
    for shape in ((512, 8, 8192, 2), (512, 128, 8192, 2), (4096, 1, 8192, 2)):
        with pytest.raises(corr.CorrError) as ei:
            corr.corr_xengine_static(x.data_ptr(), shape[0], shape[1], shape[2], shape[3], out.data_ptr(),
                                     out.data_ptr(), 0)
        assert "fixed maximum" in str(ei.value)


def test_static_error_word_status_and_selftest(env):
    """The bounded-wait self-test pointed at the fixed array's error word: the status call reports the
    timeout once (code 90) and clears it; the next call then runs clean."""
    corr, synth, torch = env
    stream = torch.cuda.current_stream().cuda_stream
    assert corr.corr_xengine_static_status(stream) == 0
    corr.corr_xengine_static_selftest_wait(100, stream)
    assert corr.corr_xengine_static_status(stream) == 90
    assert corr.corr_xengine_static_status(stream) == 0
    with pytest.raises(corr.CorrError):
        corr.corr_xengine_static_selftest_wait(0, stream)
    N, C, T, npol = 64, 2, 256, 2
    h = synth.generate_host(synth.Spec(kind="uniform", seed=5), T, C, N)
    d = torch.from_numpy(h).cuda()
    cross = torch.zeros((C, corr.corr_n_baselines(N, npol), npol * npol, 2), dtype=torch.int64, device="cuda")
    autos = torch.zeros((C, N), dtype=torch.int64, device="cuda")
    corr.corr_xengine_static(d.data_ptr(), N, C, T, npol, cross.data_ptr(), autos.data_ptr(), stream)
    assert corr.corr_xengine_static_status(stream) == 0
    want_c, want_a = oracle.correlate(h, npol)
    assert np.array_equal(cross.cpu().numpy(), want_c) and np.array_equal(autos.cpu().numpy(), want_a)


_CHILD = r'''
import ctypes, json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1411_3751_gb300 import corr
N, C, T, npol = int(sys.argv[2]), int(sys.argv[3]), int(sys.argv[4]), int(sys.argv[5])
x = np.load(sys.argv[6])
cu = ctypes.CDLL("libcuda.so.1")
def ck(r, what):
    if r != 0:
        raise SystemExit("%s failed: %d" % (what, r))
ck(cu.cuInit(0), "cuInit")
dev = ctypes.c_int(0)
ck(cu.cuDeviceGet(ctypes.byref(dev), 0), "cuDeviceGet")
prim = ctypes.c_void_p()
ck(cu.cuDevicePrimaryCtxRetain(ctypes.byref(prim), dev), "cuDevicePrimaryCtxRetain")
ck(cu.cuCtxSetCurrent(prim), "cuCtxSetCurrent")
second = ctypes.c_void_p()
if hasattr(cu, "cuCtxCreate_v2"):
    ck(cu.cuCtxCreate_v2(ctypes.byref(second), 0, dev), "cuCtxCreate_v2")
else:
    ck(cu.cuCtxCreate_v4(ctypes.byref(second), None, 0, dev), "cuCtxCreate_v4")
nc = C * corr.corr_n_baselines(N, npol) * npol * npol * 2
na = C * N
def run(ctx):
    ck(cu.cuCtxSetCurrent(ctx), "cuCtxSetCurrent")
    d_in, d_c, d_a = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    ck(cu.cuMemAlloc_v2(ctypes.byref(d_in), ctypes.c_size_t(x.nbytes)), "cuMemAlloc")
    ck(cu.cuMemAlloc_v2(ctypes.byref(d_c), ctypes.c_size_t(nc * 8)), "cuMemAlloc")
    ck(cu.cuMemAlloc_v2(ctypes.byref(d_a), ctypes.c_size_t(na * 8)), "cuMemAlloc")
    ck(cu.cuMemcpyHtoD_v2(d_in, ctypes.c_void_p(x.ctypes.data), ctypes.c_size_t(x.nbytes)), "cuMemcpyHtoD")
    ck(cu.cuMemsetD8_v2(d_c, ctypes.c_ubyte(0), ctypes.c_size_t(nc * 8)), "cuMemsetD8")
    ck(cu.cuMemsetD8_v2(d_a, ctypes.c_ubyte(0), ctypes.c_size_t(na * 8)), "cuMemsetD8")
    corr.corr_xengine_static(d_in.value, N, C, T, npol, d_c.value, d_a.value, 0)
    ck(cu.cuCtxSynchronize(), "cuCtxSynchronize")
    status = corr.corr_xengine_static_status(0)
    c = np.zeros(nc, dtype=np.int64)
    a = np.zeros(na, dtype=np.int64)
    ck(cu.cuMemcpyDtoH_v2(ctypes.c_void_p(c.ctypes.data), d_c, ctypes.c_size_t(nc * 8)), "cuMemcpyDtoH")
    ck(cu.cuMemcpyDtoH_v2(ctypes.c_void_p(a.ctypes.data), d_a, ctypes.c_size_t(na * 8)), "cuMemcpyDtoH")
    for p in (d_in, d_c, d_a):
        ck(cu.cuMemFree_v2(p), "cuMemFree")
    return c, a, status
res = {}
for k, ctx in enumerate((prim, second, prim, second)):
    c, a, status = run(ctx)
    np.save(sys.argv[7] + "_c%d.npy" % k, c)
    np.save(sys.argv[7] + "_a%d.npy" % k, a)
    res[k] = status
ck(cu.cuCtxDestroy_v2(second), "cuCtxDestroy")
print(json.dumps(res))
'''


def test_static_in_a_second_cuda_context(env, tmp_path):
    """A child process calls the entry point alternately in the device's primary context and in a second
    context made with the driver API (buffers allocated by the driver in each): the array is loaded
    into each context at its own address, and every call matches the oracle."""
    corr, synth, _ = env
    N, C, T, npol = 96, 3, 640, 2
    h = synth.generate_host(synth.Spec(kind="gauss_tone", seed=9), T, C, N)
    np.save(tmp_path / "x.npy", h)
    out = subprocess.run([sys.executable, "-c", _CHILD, ROOT, str(N), str(C), str(T), str(npol),
                          str(tmp_path / "x.npy"), str(tmp_path / "r")], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-2000:]
    status = json.loads(out.stdout.strip().splitlines()[-1])
    assert all(v == 0 for v in status.values()), status
    want_c, want_a = oracle.correlate(h, npol)
    for k in range(4):
        got_c = np.load(tmp_path / ("r_c%d.npy" % k)).reshape(want_c.shape)
        got_a = np.load(tmp_path / ("r_a%d.npy" % k)).reshape(want_a.shape)
        assert np.array_equal(got_c, want_c) and np.array_equal(got_a, want_a), k
