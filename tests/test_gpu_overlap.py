"""Overlapped batches: the TMA-fed operand build of launch j + 1 on a few SMs beside the X-engine's
multiply of launch j (corr_set_prep_sms). Bit-exact against the oracle and against the sequential
schedule, for several SM splits, input counts that are not multiples of the 128-input build unit,
block lengths that are not multiples of the 128-sample tile, and a last launch shorter than the
others; total power through both cadences."""
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


def _batch(env, host_blocks, N, C, T, npol, prep_sms, plan=0):
    corr, _, torch = env
    with corr.Correlator(N, C, T, npol, path="fp8tc") as xc:
        xc.set_tile_plan(plan)  # the overlapped schedule runs plans 0, 1 and 3
        xc.set_prep_sms(prep_sms)
        assert xc.prep_sms == prep_sms
        blocks = [torch.from_numpy(b).cuda() for b in host_blocks]
        xc.accumulate_batch(blocks)
        c = xc.dump(corr.CORR_WHAT_CROSS).cpu().numpy()
        a = xc.dump(corr.CORR_WHAT_AUTO).cpu().numpy()
        xc.sync()
        k = corr.corr_batch_blocks(N, C, T, npol)
    return c, a, k


@pytest.mark.parametrize("plan", [0, 3])
@pytest.mark.parametrize("shape", [(144, 3, 1000, 2), (256, 2, 4096, 2), (128, 4, 2048, 1)])
def test_overlapped_batch_matches_oracle_and_sequential(env, shape, plan):
    """Tile plan 0 (one SM per item) and plan 3 (SM pairs: the X-engine on S - k SMs is a grid of
    (S - k) / 2 clusters; with k = S the build has no room beside the pair CTAs and runs between them)."""
    corr, synth, torch = env
    N, C, T, npol = shape
    k = corr.corr_batch_blocks(N, C, T, npol)
    n_blocks = 2 * k + 1  # three launches, the last one block long
    spec = synth.Spec(kind="saturate", seed=N + 31 * T, seg_len=512, m8_segment=3)
    host = synth.generate_host(spec, n_blocks * T, C, N)
    blocks = [np.ascontiguousarray(host[b * T:(b + 1) * T]) for b in range(n_blocks)]
    want_c, want_a = oracle.correlate(host, npol, threads=8)
    seq_c, seq_a, _ = _batch(env, blocks, N, C, T, npol, 0, plan)
    assert np.array_equal(seq_c, want_c) and np.array_equal(seq_a, want_a)
    n_sms = torch.cuda.get_device_properties(0).multi_processor_count
    for sms in (1, 8, 30, 43, 76, n_sms - 1, n_sms):  # n_sms: a small build CTA beside the X-engine on every SM
        c, a, _ = _batch(env, blocks, N, C, T, npol, sms, plan)
        bad = np.argwhere(c != want_c)
        assert bad.size == 0, (sms, bad[:3].tolist())
        assert np.array_equal(a, want_a), sms


@pytest.mark.parametrize("plan", [0, 3])
def test_overlapped_batch_512_inputs(env, plan):
    """The benchmark's shape per launch (512 inputs, 8192-sample blocks, 4 blocks per launch) on two
    channels, nine blocks: launches of 4, 4 and 1 blocks, the build on 43 SMs (about 2/7 of them)."""
    corr, synth, torch = env
    N, C, T, npol = 512, 2, 8192, 2
    assert corr.corr_batch_blocks(N, C, T, npol) == 4
    spec = synth.Spec(kind="gauss_tone", seed=0x14113751 + 21)
    host = synth.generate_host(spec, 9 * T, C, N)
    blocks = [np.ascontiguousarray(host[b * T:(b + 1) * T]) for b in range(9)]
    want_c, want_a = oracle.correlate(host, npol, threads=8)
    c, a, _ = _batch(env, blocks, N, C, T, npol, 43, plan)
    assert np.array_equal(c, want_c) and np.array_equal(a, want_a)


def test_overlap_then_single_blocks_and_dumps_in_order(env):
    """An overlapped batch, then corr_accumulate and a total-power dump with reset on the same stream,
    then another batch: every dump sees exactly the work enqueued before it."""
    corr, synth, torch = env
    N, C, T, npol = 256, 3, 4096, 2
    k = corr.corr_batch_blocks(N, C, T, npol)
    spec = synth.Spec(kind="gauss_tone", seed=5)
    nb = 2 * k
    host = synth.generate_host(spec, (2 * nb + 1) * T, C, N)
    blk = [torch.from_numpy(np.ascontiguousarray(host[b * T:(b + 1) * T])).cuda() for b in range(2 * nb + 1)]
    with corr.Correlator(N, C, T, npol, path="fp8tc") as xc:
        xc.set_tile_plan(0)
        xc.set_prep_sms(24)
        xc.accumulate_batch(blk[:nb])
        xc.accumulate(blk[nb])
        a1 = xc.dump(corr.CORR_WHAT_AUTO, reset=True).cpu().numpy()
        xc.accumulate_batch(blk[nb + 1:])
        a2 = xc.dump(corr.CORR_WHAT_AUTO).cpu().numpy()
        c = xc.dump(corr.CORR_WHAT_CROSS).cpu().numpy()
        xc.sync()
    assert np.array_equal(a1, oracle.autos(host[:(nb + 1) * T]))
    assert np.array_equal(a2, oracle.autos(host[(nb + 1) * T:]))
    want_c, _ = oracle.correlate(host, npol, threads=8)
    assert np.array_equal(c, want_c)


def test_prep_sms_bounds(env):
    corr, _, torch = env
    with corr.Correlator(128, 1, 256, 2) as xc:
        assert xc.prep_sms == 0  # automatic: sequential
        assert xc.set_prep_sms(torch.cuda.get_device_properties(0).multi_processor_count) is None
        for bad in (-2, 100000):
            with pytest.raises(corr.CorrError):
                xc.set_prep_sms(bad)
        xc.set_prep_sms(0)
        assert xc.prep_sms == 0
