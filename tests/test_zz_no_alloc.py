"""corr_xengine_static: the allocation-free entry point, for callers that cannot call cudaMalloc
(code running inside another runtime's memory pool, or a real-time pipeline that forbids
allocation after start-up). Its scratch is a fixed device array inside the library. Checked
against the context entry points (corr_create / corr_accumulate / corr_dump) on two calls in a
row, which must also show that the shared scratch carries nothing over from one call to the next.

Collected last on purpose (file name), so a stop-at-first-failure run has already run every other
test before this one.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1411_3751_gb300 import corr, synth

    assert torch.cuda.is_available()
    return corr, synth, torch


@pytest.mark.parametrize("shape", [(64, 4, 1000, 2), (512, 4, 8192, 2), (200, 3, 300, 1)])
def test_static_matches_context_path_on_two_calls(env, shape):
    corr, synth, torch = env
    N, C, T, npol = shape
    spec = synth.Spec(kind="gauss_tone", seed=N + C + T)
    b1 = synth.generate_device(spec, T, C, N, t0=0)
    b2 = synth.generate_device(spec, T, C, N, t0=T)
    with corr.Correlator(N, C, T, npol) as xc:
        xc.accumulate(b1)
        want_c1 = xc.dump(corr.CORR_WHAT_CROSS)
        want_a1 = xc.dump(corr.CORR_WHAT_AUTO)
        xc.accumulate(b2)
        want_c2 = xc.dump(corr.CORR_WHAT_CROSS)
        want_a2 = xc.dump(corr.CORR_WHAT_AUTO)
        xc.sync()
    cross = torch.zeros_like(want_c1)
    autos = torch.zeros_like(want_a1)
    stream = torch.cuda.current_stream().cuda_stream
    corr.corr_xengine_static(b1.data_ptr(), N, C, T, npol, cross.data_ptr(), autos.data_ptr(), stream)
    torch.cuda.synchronize()
    assert torch.equal(cross, want_c1) and torch.equal(autos, want_a1)
    corr.corr_xengine_static(b2.data_ptr(), N, C, T, npol, cross.data_ptr(), autos.data_ptr(), stream)
    torch.cuda.synchronize()
    assert torch.equal(cross, want_c2) and torch.equal(autos, want_a2)


def test_static_rejects_sizes_beyond_its_scratch(env):
    corr, _, torch = env
    x = torch.zeros(8, dtype=torch.uint8, device="cuda")
    out = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(corr.CorrError) as ei:
        corr.corr_xengine_static(x.data_ptr(), 512, 128, 8192, 2, out.data_ptr(), out.data_ptr(), 0)
    assert "fixed maximum" in str(ei.value)
