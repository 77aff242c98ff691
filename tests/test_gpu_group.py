"""Groups of uneven sub-arrays in one persistent tensor-core launch (corr_group_*), against the oracle.

Checks the grouped launch, the separate-launch comparison mode, the autotuner (plans and its reset)
and CUDA-graph capture / replay, first on a small group (full oracle), then on the 5-array workload
with 32, 64, 200, 256 and 512 inputs and 2400, 600, 300, 150 and 109 channels of 4096 samples
(sampled oracle cells on host-regenerated channels, oracle autos and a Freivalds projection on
every channel).
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
    from paper_1411_3751_gb300 import corr, synth

    assert torch.cuda.is_available()
    return corr, synth, torch


def _dump(member, corr):
    c = member.dump(corr.CORR_WHAT_CROSS)
    a = member.dump(corr.CORR_WHAT_AUTO)
    member.sync()
    return c.cpu().numpy(), a.cpu().numpy()


def test_small_group_all_modes(env):
    corr, synth, torch = env
    shapes = [(32, 24), (64, 12), (200, 6), (256, 5), (512, 3)]
    T, npol = 4096, 2
    specs = [synth.Spec(kind="gauss_tone", seed=4000 + i) for i in range(len(shapes))]
    blk = [[synth.generate_device(sp, T, c, n, t0=k * T) for sp, (n, c) in zip(specs, shapes)] for k in range(2)]
    want = [oracle.correlate(np.concatenate([blk[0][i].cpu().numpy(), blk[1][i].cpu().numpy()]), npol, threads=8)
            for i in range(len(shapes))]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        # grouped launch, two blocks
        with corr.Group(shapes, T, npol) as g:
            g.accumulate(blk[0])
            g.accumulate(blk[1])
            for i, m in enumerate(g.members):
                c, a = _dump(m, corr)
                assert np.array_equal(c, want[i][0]) and np.array_equal(a, want[i][1]), "grouped, array %d" % i
                assert m.samples(corr.CORR_WHAT_CROSS) == 2 * T
        # separate launches
        with corr.Group(shapes, T, npol) as g:
            g.accumulate(blk[0], separate=True)
            g.accumulate(blk[1], separate=True)
            for i, m in enumerate(g.members):
                c, a = _dump(m, corr)
                assert np.array_equal(c, want[i][0]) and np.array_equal(a, want[i][1]), "separate, array %d" % i
        # autotune (must leave the accumulators empty), then graph capture + two replays
        with corr.Group(shapes, T, npol) as g:
            plans = g.autotune(blk[0])
            assert len(plans) == len(shapes) and all(p in (0, 1) for p in plans)
            for m in g.members:
                c, a = _dump(m, corr)
                assert not c.any() and not a.any() and m.samples(corr.CORR_WHAT_CROSS) == 0
            bufs = [torch.empty_like(b) for b in blk[0]]
            g.capture(bufs, stream)
            for k in range(2):
                for dst, src in zip(bufs, blk[k]):
                    dst.copy_(src)
                g.launch(stream)
            for i, m in enumerate(g.members):
                c, a = _dump(m, corr)
                assert np.array_equal(c, want[i][0]) and np.array_equal(a, want[i][1]), "graph, array %d" % i
                assert m.samples(corr.CORR_WHAT_CROSS) == 2 * T
    stream.synchronize()


def _freivalds(x_bytes, V_cross, npol, rng, chunk=16384):
    T, N = x_bytes.shape
    S = N // npol
    Vf = np.zeros((N, N), dtype=np.complex128)
    for sa in range(S):
        for sc in range(sa + 1):
            b = sa * (sa + 1) // 2 + sc
            for p in range(npol):
                for q in range(npol):
                    i, j = sa * npol + p, sc * npol + q
                    if i < j:
                        continue
                    v = V_cross[b, p * npol + q]
                    Vf[i, j] = v[0] + 1j * v[1]
                    Vf[j, i] = v[0] - 1j * v[1]
    w = rng.integers(-2, 3, size=N) + 1j * rng.integers(-2, 3, size=N)
    re, im = oracle.unpack(x_bytes)
    re, im = re.astype(np.float64), im.astype(np.float64)
    yr = re @ np.real(w) + im @ np.imag(w)
    yi = re @ np.imag(w) - im @ np.real(w)
    zr = re.T @ yr - im.T @ yi
    zi = re.T @ yi + im.T @ yr
    Vw = Vf @ w
    return np.array_equal(Vw.real, zr) and np.array_equal(Vw.imag, zi)


def test_five_uneven_subarrays_graph(env):
    """N in {32, 64, 200, 256, 512} with {2400, 600, 300, 150, 109} channels, 4096 samples each."""
    corr, synth, torch = env
    shapes = [(32, 2400), (64, 600), (200, 300), (256, 150), (512, 109)]
    T, npol = 4096, 2
    specs = [synth.Spec(kind="gauss_tone", seed=0x14113751 + 4 + 100 * i) for i in range(len(shapes))]
    blocks = [synth.generate_device(sp, T, c, n) for sp, (n, c) in zip(specs, shapes)]
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(44)
    with torch.cuda.stream(stream), corr.Group(shapes, T, npol) as g:
        plans = g.autotune(blocks)
        g.capture(blocks, stream)
        g.launch(stream)
        stream.synchronize()
        for i, ((n, c), m) in enumerate(zip(shapes, g.members)):
            cross, autos = _dump(m, corr)
            x = blocks[i].cpu().numpy()
            for f in (0, c // 2, c - 1):
                hf = synth.generate_host(specs[i], T, c, n, c_range=(f, f + 1))
                assert np.array_equal(hf[:, 0], x[:, f])
                cells, idx = [], []
                for _ in range(40):
                    sa = int(rng.integers(0, n // 2))
                    sc = int(rng.integers(0, sa + 1))
                    p, q = int(rng.integers(0, 2)), int(rng.integers(0, 2))
                    cells.append((0, 2 * sa + p, 2 * sc + q))
                    idx.append((sa * (sa + 1) // 2 + sc, 2 * p + q))
                got = oracle.cells(hf, cells)
                for k, (b, pq) in enumerate(idx):
                    assert tuple(cross[f, b, pq]) == tuple(got[k]), (i, f, b, pq)
            for f in range(c):
                xf = np.ascontiguousarray(x[:, f])
                assert np.array_equal(autos[f], oracle.autos(xf[:, None, :])[0]), (i, f)
                assert _freivalds(xf, cross[f], npol, rng), (i, f)
    print("five-array group: tile plans %s" % plans)


def test_group_channel_pairs_and_build_load_widths(env):
    """Members of at most 32 inputs (channel groups of 2 or 4, full and partial last groups) beside
    larger ones, with input counts whose rows allow 16-, 8-, 4- and 1-byte loads in the one-launch
    operand build (6, 16, 17, 20, 24, 32, 100, 130 inputs), a ragged block length and one
    polarisation: grouped, separate and graph replay all equal the oracle."""
    corr, synth, torch = env
    shapes = [(17, 5), (20, 3), (24, 4), (32, 7), (100, 2), (130, 3), (16, 6), (6, 5)]
    T, npol = 1000, 1
    specs = [synth.Spec(kind="saturate", seed=700 + i, seg_len=128, m8_segment=1) for i in range(len(shapes))]
    blk = [[synth.generate_device(sp, T, c, n, t0=k * T) for sp, (n, c) in zip(specs, shapes)] for k in range(2)]
    want = [oracle.correlate(np.concatenate([blk[0][i].cpu().numpy(), blk[1][i].cpu().numpy()]), npol, threads=8)
            for i in range(len(shapes))]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for mode in ("grouped", "separate", "graph"):
            with corr.Group(shapes, T, npol) as g:
                if mode == "graph":
                    bufs = [torch.empty_like(b) for b in blk[0]]
                    g.capture(bufs, stream)
                for k in range(2):
                    if mode == "graph":
                        for dst, src in zip(bufs, blk[k]):
                            dst.copy_(src)
                        g.launch(stream)
                    else:
                        g.accumulate(blk[k], separate=(mode == "separate"))
                for i, m in enumerate(g.members):
                    c, a = _dump(m, corr)
                    assert np.array_equal(c, want[i][0]) and np.array_equal(a, want[i][1]), (mode, shapes[i])
    stream.synchronize()


def test_member_path_switch_releases_scratch_and_group_rejects_it(env):
    """Setting a member to the FP32 path releases its operand scratch; the grouped launch then refuses
    with an error (no launch on a missing buffer) and works again once a tensor path is set."""
    corr, synth, torch = env
    shapes = [(64, 8), (512, 16)]
    T, npol = 1024, 2
    blocks = [synth.generate_device(synth.Spec(kind="gauss_tone", seed=90 + i), T, c, n) for i, (n, c) in enumerate(shapes)]
    with corr.Group(shapes, T, npol) as g:
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        g.members[1].set_path("fp32")
        free1 = torch.cuda.mem_get_info()[0]
        assert free1 - free0 >= 100 << 20  # 16 ch x 1024 samples x 1024 rows x 8 blocks per launch
        with pytest.raises(corr.CorrError):
            g.accumulate(blocks)
        g.members[1].set_path("fp8tc")
        g.accumulate(blocks)
        for i, m in enumerate(g.members):
            c, a = _dump(m, corr)
            want_c, want_a = oracle.correlate(blocks[i].cpu().numpy(), npol, threads=8)
            assert np.array_equal(c, want_c) and np.array_equal(a, want_a), i
