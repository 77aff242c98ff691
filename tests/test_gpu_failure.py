"""Failure detection on the GPU without a fault: a bounded device-side wait that runs out.

corr_selftest_wait enqueues a one-thread kernel whose bounded mbarrier wait (the same helper every
pipeline handoff of the tensor-core kernels uses) targets a barrier phase that nothing completes.
The wait must give up after its limit, the next corr_sync must report CORR_ERR_TIMEOUT once, and the
same context must then correlate bit-exactly again.
"""
import time

import numpy as np
import pytest

from oracle import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1411_3751_gb300 import corr, synth

    assert torch.cuda.is_available()
    return corr, synth, torch


def test_bounded_wait_gives_up_and_the_context_stays_usable(env):
    corr, synth, torch = env
    N, C, T = 96, 3, 640
    host = synth.generate_host(synth.Spec(kind="gauss_tone", seed=1411), T, C, N)
    want_c, want_a = oracle.correlate(host, 2)
    stream = torch.cuda.current_stream().cuda_stream
    with corr.Correlator(N, C, T, 2, path="fp8tc") as xc:
        xc.sync()
        t0 = time.perf_counter()
        corr.corr_selftest_wait(xc.ctx, 200, stream)
        with pytest.raises(corr.CorrError) as info:
            xc.sync()
        elapsed = time.perf_counter() - t0
        assert info.value.code == corr.CORR_ERR_TIMEOUT
        assert 0.15 < elapsed < 10.0, elapsed  # the wait ran to its limit, then returned
        xc.sync()  # reported once, then cleared
        for bad in (0, 2001):
            with pytest.raises(corr.CorrError):
                corr.corr_selftest_wait(xc.ctx, bad, stream)
        xc.accumulate(torch.from_numpy(host).cuda())
        c = xc.dump(corr.CORR_WHAT_CROSS).cpu().numpy()
        a = xc.dump(corr.CORR_WHAT_AUTO).cpu().numpy()
        xc.sync()
    assert np.array_equal(c, want_c) and np.array_equal(a, want_a)
