"""Selective dumps (corr_dump_stations): the cells among a station list are dumped and zeroed on their
own cadence while every other cell keeps integrating (Sec. 2.6), on every arithmetic path, against the
oracle over the matching time windows."""
import numpy as np
import pytest

from oracle import oracle

pytestmark = pytest.mark.gpu

PATHS = ["fp32", "i8mma", "fp8tc", "fp8tc_fused"]


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1411_3751_gb300 import corr, synth

    assert torch.cuda.is_available()
    return corr, synth, torch


def _selected_pairs(stations):
    out = set()
    for k in range(len(stations)):
        for l in range(k + 1):
            a, c = max(stations[k], stations[l]), min(stations[k], stations[l])
            out.add(a * (a + 1) // 2 + c)
    return sorted(out)


@pytest.mark.parametrize("path", PATHS)
def test_selective_dump_and_reset(env, path):
    corr, synth, torch = env
    N, C, T, npol = 40, 3, 640, 2
    st = [13, 2, 7, 19, 0]
    host = synth.generate_host(synth.Spec(kind="gauss_tone", seed=515), 3 * T, C, N)
    blk = [torch.from_numpy(np.ascontiguousarray(host[k * T:(k + 1) * T])).cuda() for k in range(3)]
    w0, w1, w2 = host[:T], host[T:2 * T], host[2 * T:]
    with corr.Correlator(N, C, T, npol, path=path) as xc:
        xc.accumulate(blk[0])
        a_sel = xc.dump_stations(st, corr.CORR_WHAT_AUTO, reset=True)
        c_sel = xc.dump_stations(st, corr.CORR_WHAT_CROSS, reset=True, device=False)
        xc.sync()
        assert np.array_equal(a_sel.cpu().numpy(), oracle.station_autos(w0, st, npol))
        assert np.array_equal(c_sel.numpy(), oracle.station_cross(w0, st, npol))
        xc.accumulate(blk[1])
        cross = xc.dump(corr.CORR_WHAT_CROSS).cpu().numpy()
        autos = xc.dump(corr.CORR_WHAT_AUTO).cpu().numpy()
        norm = xc.dump(corr.CORR_WHAT_CROSS, fmt=corr.CORR_FMT_CF32_NORM).cpu().numpy()
        anorm = xc.dump(corr.CORR_WHAT_AUTO, fmt=corr.CORR_FMT_CF32_NORM).cpu().numpy()
        snorm = xc.dump_stations(st, corr.CORR_WHAT_CROSS, fmt=corr.CORR_FMT_CF32_NORM).cpu().numpy()
        xc.sync()
        assert xc.samples(corr.CORR_WHAT_CROSS) == 2 * T
        # selected cells hold the second window only, the rest both windows
        want_c, want_a = oracle.correlate(np.concatenate([w0, w1]), npol)
        c1, a1 = oracle.correlate(w1, npol)
        sel = _selected_pairs(st)
        sel_in = [s * npol + p for s in st for p in range(npol)]
        want_c[:, sel] = c1[:, sel]
        want_a[:, sel_in] = a1[:, sel_in]
        assert np.array_equal(cross, want_c)
        assert np.array_equal(autos, want_a)
        # CF32_NORM divides each cell by its own sample count
        counts = np.full(want_c.shape[1], 2 * T)
        counts[sel] = T
        assert np.array_equal(norm, (want_c / counts[None, :, None, None]).astype(np.float32))
        acounts = np.full(N, 2 * T)
        acounts[sel_in] = T
        assert np.array_equal(anorm, (want_a / acounts[None, :]).astype(np.float32))
        assert np.array_equal(snorm, oracle.to_format(oracle.station_cross(w1, st, npol), oracle.FMT_CF32_NORM, T))
        # a full reset clears the per-cell counts too
        xc.reset()
        xc.accumulate(blk[2])
        c2, a2 = oracle.correlate(w2, npol)
        assert np.array_equal(xc.dump(corr.CORR_WHAT_CROSS).cpu().numpy(), c2)
        got = xc.dump(corr.CORR_WHAT_CROSS, fmt=corr.CORR_FMT_CF32_NORM).cpu().numpy()
        assert np.array_equal(got, oracle.to_format(c2, oracle.FMT_CF32_NORM, T))
        assert np.array_equal(xc.dump(corr.CORR_WHAT_AUTO).cpu().numpy(), a2)
        xc.sync()


def test_outrigger_autos_at_high_cadence(env):
    """Ten outrigger stations' total power dumped and zeroed every block (1 s in the paper) while the
    visibilities integrate over all blocks (9 s in the paper), on the 512-input tensor path."""
    corr, synth, torch = env
    N, C, T, npol, B = 512, 4, 1024, 2, 4
    out = [251, 252, 253, 254, 255, 3, 77, 128, 200, 9]
    spec = synth.Spec(kind="gauss_tone", seed=616)
    host = synth.generate_host(spec, B * T, C, N)
    with corr.Correlator(N, C, T, npol, path="fp8tc") as xc:
        for b in range(B):
            xc.accumulate(torch.from_numpy(np.ascontiguousarray(host[b * T:(b + 1) * T])).cuda())
            a = xc.dump_stations(out, corr.CORR_WHAT_AUTO, reset=True, device=False)
            xc.sync()
            assert np.array_equal(a.numpy(), oracle.station_autos(host[b * T:(b + 1) * T], out, npol)), b
        cross = xc.dump(corr.CORR_WHAT_CROSS, device=False)
        autos = xc.dump(corr.CORR_WHAT_AUTO, device=False)
        xc.sync()
    # the visibilities of the outriggers integrated over all blocks (sampled against the oracle)
    cells, idx = [], []
    for k, s in enumerate(out):
        for c in (0, 100, s):
            a_, c_ = max(s, c), min(s, c)
            cells.append((1, 2 * a_, 2 * c_ + 1))
            idx.append((a_ * (a_ + 1) // 2 + c_, 1))
    got = oracle.cells(host, cells)
    for k, (b, pq) in enumerate(idx):
        assert tuple(cross.numpy()[1, b, pq]) == tuple(got[k])
    # non-outrigger autos integrated over all blocks; outrigger autos restarted after the last dump
    full = oracle.autos(host)
    keep = [i for i in range(N) if i // 2 not in out]
    assert np.array_equal(autos.numpy()[:, keep], full[:, keep])
    assert not autos.numpy()[:, [2 * s + p for s in out for p in range(2)]].any()


def test_selective_dump_rejects_bad_lists(env):
    corr, synth, torch = env
    with corr.Correlator(8, 1, 128, 2) as xc:
        for bad in ([1, 1], [4], [-1], []):
            with pytest.raises(corr.CorrError):
                xc.dump_stations(bad, corr.CORR_WHAT_AUTO)
