"""Precision variants at 512 inputs x 256 channels x 65536 samples with saturation-heavy segments
(alternating 4096-sample segments at sigma = 6 and one all -8-8i segment): the FP8 tensor path with
in-chip partial sums flushed to int64 every 4096 samples and once per 65536 samples, and the int8
mma.sync path flushed every 16384 samples, all bit-exact (sampled oracle cells on host-regenerated
channels, oracle autos, and agreement between the three)."""
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


def test_flush_periods_saturating_input(env):
    corr, synth, torch = env
    N, C, T, npol = 512, 256, 65536, 2
    spec = synth.Spec(kind="saturate", seed=0x14113751 + 3, seg_len=4096, m8_segment=5)
    x = synth.generate_device(spec, T, C, N)
    results = {}
    for path, flush in (("fp8tc", 4096), ("fp8tc", 65536), ("i8mma", 16384)):
        with corr.Correlator(N, C, T, npol, path=path) as xc:
            xc.set_flush_period(flush)
            xc.accumulate(x)
            results[path, flush] = (xc.dump(corr.CORR_WHAT_CROSS).cpu().numpy(),
                                    xc.dump(corr.CORR_WHAT_AUTO).cpu().numpy())
            xc.sync()
    for key in (("fp8tc", 65536), ("i8mma", 16384)):
        assert np.array_equal(results["fp8tc", 4096][0], results[key][0]), key
        assert np.array_equal(results["fp8tc", 4096][1], results[key][1]), key
    cross, autos = results["fp8tc", 4096]
    rng = np.random.default_rng(33)
    for f in (0, 200):
        hf = synth.generate_host(spec, T, C, N, c_range=(f, f + 1))
        assert np.array_equal(autos[f], oracle.autos(hf)[0])
        cells, idx = [], []
        for _ in range(48):
            sa = int(rng.integers(0, N // 2))
            sc = int(rng.integers(0, sa + 1))
            p, q = int(rng.integers(0, 2)), int(rng.integers(0, 2))
            cells.append((0, 2 * sa + p, 2 * sc + q))
            idx.append((sa * (sa + 1) // 2 + sc, 2 * p + q))
        got = oracle.cells(hf, cells)
        for k, (b, pq) in enumerate(idx):
            assert tuple(cross[f, b, pq]) == tuple(got[k]), (f, b, pq)
    # the all -8-8i segment and the clipped segments saturate: autos stay exact integers >= 0
    assert autos.min() >= 0
