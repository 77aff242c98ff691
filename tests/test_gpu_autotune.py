"""The batch schedule knobs and their autotuner: every launch length gives the oracle's sums, and
corr_autotune leaves zeroed accumulators, a valid schedule that then correlates bit-exactly, and a
cached choice for the next context of the same shape."""
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


def _blocks(env, N, C, T, n, seed):
    _, synth, torch = env
    host = synth.generate_host(synth.Spec(kind="gauss_tone", seed=seed), n * T, C, N)
    return host, [torch.from_numpy(np.ascontiguousarray(host[b * T:(b + 1) * T])).cuda() for b in range(n)]


def test_every_launch_length_matches_the_oracle(env):
    corr, _, torch = env
    N, C, T, npol, n = 144, 3, 1000, 2, 7
    host, blocks = _blocks(env, N, C, T, n, 41)
    want_c, want_a = oracle.correlate(host, npol, threads=8)
    with corr.Correlator(N, C, T, npol) as xc:
        default = xc.batch_blocks
        assert default == corr.corr_batch_blocks(N, C, T, npol)
        for K in (1, 2, 3, 7, 0):
            xc.set_batch_blocks(K)
            assert xc.batch_blocks == (K or default)
            xc.accumulate_batch(blocks)
            c = xc.dump(corr.CORR_WHAT_CROSS, reset=True).cpu().numpy()
            a = xc.dump(corr.CORR_WHAT_AUTO, reset=True).cpu().numpy()
            xc.sync()
            assert np.array_equal(c, want_c) and np.array_equal(a, want_a), K
        for bad in (-1, 1 << 20):
            with pytest.raises(corr.CorrError):
                xc.set_batch_blocks(bad)


def test_autotune_then_correlate(env):
    corr, _, torch = env
    N, C, T, npol, n = 256, 3, 4096, 2, 12
    host, blocks = _blocks(env, N, C, T, n, 43)
    want_c, want_a = oracle.correlate(host, npol, threads=8)
    with corr.Correlator(N, C, T, npol) as xc:
        choice = xc.autotune(blocks, reps=1)
        assert choice["tile_plan"] in (0, 1, 2, 3) and choice["batch_blocks"] >= 1 and choice["n_tried"] >= 6
        assert choice["ms_per_block"] > 0
        assert (xc.tile_plan, xc.batch_blocks, xc.prep_sms) == (choice["tile_plan"], choice["batch_blocks"],
                                                                choice["prep_sms"])
        assert xc.samples(corr.CORR_WHAT_CROSS) == 0 and xc.samples(corr.CORR_WHAT_AUTO) == 0
        assert not torch.any(xc.dump(corr.CORR_WHAT_CROSS) != 0).item()
        xc.accumulate_batch(blocks)
        c = xc.dump(corr.CORR_WHAT_CROSS).cpu().numpy()
        a = xc.dump(corr.CORR_WHAT_AUTO).cpu().numpy()
        xc.sync()
    assert np.array_equal(c, want_c) and np.array_equal(a, want_a)
    # the same shape again: the cached choice, applied without timing
    with corr.Correlator(N, C, T, npol) as xc:
        again = xc.autotune(blocks, reps=1)
        assert again["n_tried"] == 0
        assert (again["tile_plan"], again["batch_blocks"], again["prep_sms"]) == (
            choice["tile_plan"], choice["batch_blocks"], choice["prep_sms"])


def test_autotune_needs_the_tensor_path(env):
    corr, _, torch = env
    _, blocks = _blocks(env, 64, 1, 256, 2, 5)
    with corr.Correlator(64, 1, 256, 2, path="fp32") as xc:
        with pytest.raises(corr.CorrError):
            xc.autotune(blocks)
