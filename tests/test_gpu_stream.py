"""Streaming serving loop (paper_1411_3751_gb300.stream) on the GPU, against the oracle.

One full-band 512-input x 2400-channel stream and three 64-input x 2400-channel streams in 10 ms
blocks (240 samples); cross-power dumps every 900 blocks (9 s), total-power dumps every 100 blocks
(1 s). Checks admission by footprint, the dump cadences and counts, and the first dumps of each kind
against the oracle on sampled channels regenerated on the host (cells, autos, Freivalds).
"""
import numpy as np
import pytest

from oracle import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1411_3751_gb300 import corr, stream, synth

    assert torch.cuda.is_available()
    return corr, stream, synth, torch


def test_stream_loop_512_plus_three_64(env):
    corr, stream, synth, torch = env
    specs = [stream.StreamSpec("leda512", 512, 2400, gulp_blocks=25, seed=0x14113751 + 5)]
    specs += [stream.StreamSpec("lwa64_%d" % k, 64, 2400, gulp_blocks=25, seed=0x14113751 + 50 + k) for k in range(3)]
    total_fp = sum(s.footprint() for s in specs)
    srv = stream.Server(hbm_budget_bytes=total_fp + (1 << 30), keep_dumps=1)
    try:
        for s in specs:
            assert srv.admit(s), s.name
        # a second full-band stream does not fit the budget and is rejected
        assert not srv.admit(stream.StreamSpec("extra512", 512, 2400, gulp_blocks=25))
        out = srv.run(1800)  # 18 s-equivalent: 2 cross and 18 total-power dumps per stream
        assert out["rejected"] == ["extra512"]
        for name, st in out["streams"].items():
            assert st["cross_dumps"] == 2 and st["auto_dumps"] == 18, name
            assert st["cross_latency_ms"]["p99"] > 0
        assert out["real_time_factor"] > 1.0 and out["real_time_factor_correlator"] >= out["real_time_factor"]
        print("stream loop: RTF %.1f (correlator alone %.1f) over %.0f s-equivalent, wall %.2f s" %
              (out["real_time_factor"], out["real_time_factor_correlator"], out["simulated_s"], out["wall_s"]))
        rng = np.random.default_rng(55)
        for live in srv.streams:
            sp = live.spec
            gen = synth.Spec(kind=sp.kind, seed=sp.seed)
            (c0, cross), (a0, autos) = live.cross_dumps[0], live.auto_dumps[0]
            assert c0 == 0 and a0 == 0
            n_cross = sp.cross_every * sp.block_samples
            n_auto = sp.auto_every * sp.block_samples
            for f in (7, 1999):
                hf = synth.generate_host(gen, n_cross, sp.n_chans, sp.n_inputs, c_range=(f, f + 1))
                assert np.array_equal(autos[f], oracle.autos(np.ascontiguousarray(hf[:n_auto]))[0])
                if sp.n_inputs <= 64:
                    want, _ = oracle.correlate(hf, sp.n_pol, threads=8)
                    assert np.array_equal(cross[f], want[0]), (sp.name, f)
                else:
                    cells, idx = [], []
                    for _ in range(64):
                        sa = int(rng.integers(0, sp.n_inputs // 2))
                        sc = int(rng.integers(0, sa + 1))
                        p, q = int(rng.integers(0, 2)), int(rng.integers(0, 2))
                        cells.append((0, 2 * sa + p, 2 * sc + q))
                        idx.append((sa * (sa + 1) // 2 + sc, 2 * p + q))
                    got = oracle.cells(hf, cells)
                    for k, (b, pq) in enumerate(idx):
                        assert tuple(cross[f, b, pq]) == tuple(got[k]), (sp.name, f, b, pq)
    finally:
        srv.close()


def test_fast_dump_mode_with_outriggers(env):
    """The paper's minimum dump time (0.33 s = one 8000-sample group, Table 1) with float32 visibilities
    (exact at this length) and 1 s total power of ten outrigger stations by selective dumps (Sec. 2.6)."""
    corr, stream, synth, torch = env
    outr = (251, 252, 253, 254, 255, 3, 77, 128, 200, 9)
    sp = stream.StreamSpec("fast512", 512, 240, block_samples=8000, gulp_blocks=1, cross_every=1, auto_every=3,
                           seed=0x14113751 + 6, outriggers=outr, cross_fmt=corr.CORR_FMT_CF32)
    srv = stream.Server(hbm_budget_bytes=sp.footprint() + (1 << 30), keep_dumps=2)
    try:
        assert srv.admit(sp)
        out = srv.run(6)
        st = out["streams"]["fast512"]
        assert st["cross_dumps"] == 6 and st["auto_dumps"] == 2
        live = srv.streams[0]
        gen = synth.Spec(kind=sp.kind, seed=sp.seed)
        rng = np.random.default_rng(66)
        for (b0, cross) in live.cross_dumps:
            assert cross.dtype == np.float32
            for f in (5, 239):
                hf = synth.generate_host(gen, 8000, sp.n_chans, sp.n_inputs, t0=b0 * 8000, c_range=(f, f + 1))
                cells, idx = [], []
                for _ in range(32):
                    sa = int(rng.integers(0, 256))
                    sc = int(rng.integers(0, sa + 1))
                    p, q = int(rng.integers(0, 2)), int(rng.integers(0, 2))
                    cells.append((0, 2 * sa + p, 2 * sc + q))
                    idx.append((sa * (sa + 1) // 2 + sc, 2 * p + q))
                got = oracle.cells(hf, cells).astype(np.float32)
                for k, (b, pq) in enumerate(idx):
                    assert tuple(cross[f, b, pq]) == tuple(got[k]), (b0, f, b, pq)
        for (b0, autos) in live.auto_dumps:
            hf = synth.generate_host(gen, 3 * 8000, sp.n_chans, sp.n_inputs, t0=b0 * 8000)
            assert np.array_equal(autos, oracle.station_autos(hf, outr, 2)), b0
    finally:
        srv.close()
