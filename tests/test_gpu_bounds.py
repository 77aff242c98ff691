"""GPU parity at the top of each path's exactness bound, and int64 sums past 2^31.

Every path is exact because its in-chip partial sums stay exact integers until they are flushed to
int64. These tests drive each partial sum to the largest value its path allows in one flush:

* FP8 tensor paths (offset operand u = v + 8 in [0, 15], FP32 sums in TMEM): components 7 (u = 15)
  or 6 (u = 14) put every real product sum G[r, s] = sum_t u_r u_s of a 65 536-sample flush in
  [2^23, 2^24), the binade where an FP32 accumulator has no fractional bit left, so an adder that
  dropped or rounded addend bits would be off by whole units;
* FP32 CUDA-core path (signed samples): components -8 / -7 give |Re V| up to 128 * 65 536 = 2^23
  per flush;
* int8 mma.sync path (int32 partial sums): flushed every 16 384 and every 65 536 samples.

The expected values are the closed forms of constant inputs (V = |x|^2 T, A = |x|^2 T) and the CPU
oracle for seeded inputs drawn from the high-magnitude values. The last test is the GPU twin of the
oracle's overflow pin: 2^25 samples of -8-8i give Re V = 2^32 exactly, so an accumulator that kept
32 bits anywhere on the way would wrap.
"""
import numpy as np
import pytest

from oracle import oracle

pytestmark = pytest.mark.gpu

T_FLUSH = 65536


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1411_3751_gb300 import corr, synth

    assert torch.cuda.is_available()
    return corr, synth, torch


def _byte(re, im):
    return ((np.asarray(re, dtype=np.int64) & 0xF) << 4) | (np.asarray(im, dtype=np.int64) & 0xF)


def _correlate(env, x_host, npol, path, flush, blocks=1, block_t=None):
    corr, _, torch = env
    T, C, N = x_host.shape
    bt = T if block_t is None else block_t
    d = torch.from_numpy(x_host).cuda()
    path, _, plan = path.partition("/plan")  # "fp8tc/plan3": the tensor path on SM pairs
    with corr.Correlator(N, C, bt, npol, path=path) as xc:
        if plan:
            xc.set_tile_plan(int(plan))
        xc.set_flush_period(flush)
        for b in range(blocks):
            for t0 in range(0, T, bt):
                xc.accumulate(d[t0:t0 + bt])
        cross = xc.dump(corr.CORR_WHAT_CROSS).cpu().numpy()
        autos = xc.dump(corr.CORR_WHAT_AUTO).cpu().numpy()
        xc.sync()
        assert xc.samples(corr.CORR_WHAT_CROSS) == T * blocks
    return cross, autos


CASES = [("fp8tc", T_FLUSH), ("fp8tc/plan3", T_FLUSH), ("fp8tc_fused", T_FLUSH), ("fp32", T_FLUSH), ("i8mma", 16384),
         ("i8mma", T_FLUSH)]


@pytest.mark.parametrize("path,flush", CASES)
@pytest.mark.parametrize("value", [(7, 7), (-8, -8)])
def test_constant_input_one_full_flush(env, path, flush, value):
    """128 inputs x 2 channels x 65 536 samples in ONE block, all equal to 7+7i (u = 15: every tensor
    partial sum 225 * 65536, the top binade of FP32) or -8-8i (Re V = 128 * 65536 = 2^23 on the FP32
    path): every cross cell is |x|^2 T + 0i, every auto |x|^2 T."""
    N, C, T, npol = 128, 2, T_FLUSH, 2
    host = np.full((T, C, N), _byte(*value), dtype=np.uint8)
    cross, autos = _correlate(env, host, npol, path, flush)
    p = value[0] ** 2 + value[1] ** 2
    assert np.all(cross[..., 0] == p * T), (path, np.unique(cross[..., 0])[:4])
    assert np.all(cross[..., 1] == 0)
    assert np.all(autos == p * T)


def _high_magnitude(seed, T, C, N):
    """Seeded components: inputs n % 3 != 0 draw each component from {6, 7} (offset u in {14, 15}: the
    tensor partial sums of such pairs land in [2^23, 2^24) over 65 536 samples with varying low bits);
    inputs n % 3 == 0 draw from {-8, -7} (large signed products for the FP32 path; their cross terms
    with the first group are large and negative)."""
    rng = np.random.default_rng(seed)
    re = rng.integers(0, 2, size=(T, C, N)).astype(np.int64)
    im = rng.integers(0, 2, size=(T, C, N)).astype(np.int64)
    low = (np.arange(N) % 3) == 0
    re = np.where(low, -8 + re, 6 + re)
    im = np.where(low, -8 + im, 6 + im)
    return _byte(re, im).astype(np.uint8)


@pytest.mark.parametrize("path,flush", CASES)
def test_high_magnitude_one_full_flush(env, path, flush):
    """Seeded high-magnitude samples (see _high_magnitude), 128 inputs x 2 channels x 65 536 samples in
    one block and one flush: bit-exact against the oracle, cell by cell."""
    N, C, T, npol = 128, 2, T_FLUSH, 2
    host = _high_magnitude(0x14113751 + 17, T, C, N)
    want_c, want_a = oracle.correlate(host, npol, threads=8)
    # the case does reach the top binade in the offset domain: a pair of high inputs sums to >= 2^23
    u = ((host[:, 0, 1] >> 4) & 0xF).astype(np.int64) ^ 8
    w = ((host[:, 0, 2] >> 4) & 0xF).astype(np.int64) ^ 8
    assert int(np.dot(u, w)) >= 1 << 23
    got_c, got_a = _correlate(env, host, npol, path, flush)
    bad = np.argwhere(got_c != want_c)
    assert bad.size == 0, "%s: %d cells differ, first %s got %s want %s" % (
        path, len(bad), bad[0].tolist(), got_c[tuple(bad[0])], want_c[tuple(bad[0])])
    assert np.array_equal(got_a, want_a)


@pytest.mark.parametrize("path", ["fp8tc", "fp8tc/plan3", "fp8tc_fused", "fp32", "i8mma"])
@pytest.mark.parametrize("n_inputs", [2, 64])
@pytest.mark.parametrize("value", [(-8, -8), (7, 7)])
def test_int64_sums_past_2_31(env, path, n_inputs, value):
    """2^25 samples (512 blocks of 65 536) of a constant sample on one channel: every cross cell is
    |x|^2 2^25 (2^32 for -8-8i; 98 * 2^25 > 2^31 for 7+7i, whose offset-domain sums reach
    450 * 2^25 > 2^33 in the int64 accumulators) and every auto the same; the GPU twin of the oracle's
    int64 overflow pin. 64 inputs also run the fused tensor kernel (it needs at least 64)."""
    corr, _, torch = env
    N, C, T, npol, blocks = n_inputs, 1, T_FLUSH, 2, 512
    d = torch.full((T, C, N), int(_byte(*value)), dtype=torch.uint8, device="cuda")
    path, _, plan = path.partition("/plan")
    with corr.Correlator(N, C, T, npol, path=path) as xc:
        if plan:
            xc.set_tile_plan(int(plan))
        for _ in range(blocks):
            xc.accumulate(d)
        cross = xc.dump(corr.CORR_WHAT_CROSS).cpu().numpy()
        autos = xc.dump(corr.CORR_WHAT_AUTO).cpu().numpy()
        xc.sync()
    p = value[0] ** 2 + value[1] ** 2
    total = p * T * blocks
    assert total > (1 << 31)
    assert np.all(cross[..., 0] == total), (path, np.unique(cross[..., 0])[:4])
    assert np.all(cross[..., 1] == 0)
    assert np.all(autos == total)
