"""GPU requantiser + corner turn (corr_requantize, the F-engine tail of Sec. 2.2) against the oracle:
bit-exact bytes for int32 (18+18-bit) and float32 PFB output, band and per-channel gains, the
symmetric clip, specials, ragged shapes, and the requantised data fed through the X-engine."""
import numpy as np
import pytest

from oracle import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1411_3751_gb300 import corr

    assert torch.cuda.is_available()
    return corr, torch


def _pfb_like_int(rng, N, T, F, sigma):
    return np.clip(np.rint(rng.standard_normal((N, T, F, 2)) * sigma), -(1 << 17), (1 << 17) - 1).astype(np.int32)


@pytest.mark.parametrize("shape", [(512, 16, 4096, 1229, 2398), (130, 9, 64, 5, 37), (6, 5, 40, 0, 40),
                                   (1, 1, 1, 0, 1), (257, 3, 100, 63, 33)])
def test_requantize_int32_band_gain(env, shape):
    corr, torch = env
    N, T, F, chan0, C = shape
    rng = np.random.default_rng(N * 7 + F)
    sigma = 3000.0
    x = _pfb_like_int(rng, N, T, F, sigma)
    gain = np.float32(2.5 / sigma)
    got = corr.requantize(torch.from_numpy(x).cuda(), chan0, C, gain=float(gain)).cpu().numpy()
    assert np.array_equal(got, oracle.requantize(x, chan0, C, gain=gain))
    got = corr.requantize(torch.from_numpy(x).cuda(), chan0, C, gain=2.0 ** -10, symmetric=True).cpu().numpy()
    assert np.array_equal(got, oracle.requantize(x, chan0, C, gain=2.0 ** -10, symmetric=True))


def test_requantize_float32_specials_and_channel_gains(env):
    corr, torch = env
    rng = np.random.default_rng(12)
    N, T, F, chan0, C = 96, 7, 300, 17, 250
    x = (rng.standard_normal((N, T, F, 2)) * 4).astype(np.float32)
    x[3, 2, 20] = (np.nan, np.inf)
    x[5, 0, 30] = (-np.inf, 7.5)
    x[7, 6, 40] = (-8.5, 6.5)
    x[9, 1, 50] = (0.5, -0.5)
    g = rng.uniform(0.25, 1.5, size=C).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    got = corr.requantize(xd, chan0, C, gains=torch.from_numpy(g).cuda()).cpu().numpy()
    assert np.array_equal(got, oracle.requantize(x, chan0, C, gains=g))
    got = corr.requantize(xd, chan0, C, gain=1.0).cpu().numpy()
    assert np.array_equal(got, oracle.requantize(x, chan0, C, gain=1.0))


@pytest.mark.parametrize("in_type", ["int32", "float32"])
def test_requantize_gain_product_in_single_precision(env, in_type):
    """v = +-3 with the float32 gains 0x3F555556 and 0x3F955555: the single-precision products are
    exactly +-2.5 and +-3.5 (the exact products are half an ulp off), so rint gives +-2 and +-4."""
    corr, torch = env
    gains = np.array([0x3F555556, 0x3F955555], dtype=np.uint32).view(np.float32)
    x = np.zeros((2, 1, 2, 2), dtype=np.int32 if in_type == "int32" else np.float32)
    x[0, 0, :] = (3, -3)
    x[1, 0, :] = (-3, 3)
    xd = torch.from_numpy(x).cuda()
    got = corr.requantize(xd, 0, 2, gains=torch.from_numpy(gains).cuda()).cpu().numpy()
    assert np.array_equal(got, oracle.requantize(x, 0, 2, gains=gains))
    assert got[0, 0, 0] == 0x2E and got[0, 1, 0] == 0x4C and got[0, 0, 1] == 0xE2 and got[0, 1, 1] == 0xC4
    for c, g in enumerate(gains):
        one = corr.requantize(xd, c, 1, gain=float(g)).cpu().numpy()
        assert np.array_equal(one[:, 0, :], got[:, c, :])


def test_requantized_data_through_the_x_engine(env):
    """F-engine tail -> X-engine on the device: visibilities of the requantised PFB output."""
    corr, torch = env
    rng = np.random.default_rng(21)
    N, T, F, chan0, C, npol = 64, 1024, 96, 10, 24, 2
    common = rng.standard_normal((1, T, F, 2)) * 1500.0  # a correlated component shared by all inputs
    x = np.clip(np.rint(rng.standard_normal((N, T, F, 2)) * 2500.0 + common), -(1 << 17), (1 << 17) - 1)
    x = x.astype(np.int32)
    gain = np.float32(2.5 / 2900.0)
    with corr.Correlator(N, C, T, npol) as xc:
        q = corr.requantize(torch.from_numpy(x).cuda(), chan0, C, gain=float(gain))
        xc.accumulate(q)
        cross = xc.dump(corr.CORR_WHAT_CROSS).cpu().numpy()
        autos = xc.dump(corr.CORR_WHAT_AUTO).cpu().numpy()
        xc.sync()
    want_c, want_a = oracle.correlate(oracle.requantize(x, chan0, C, gain=gain), npol, threads=8)
    assert np.array_equal(cross, want_c) and np.array_equal(autos, want_a)
    assert (cross[:, 1:, 0, 0] > 0).mean() > 0.9  # the common component correlates


def test_requantize_rejects_bad_arguments(env):
    corr, torch = env
    x = torch.zeros((4, 2, 8, 2), dtype=torch.int32, device="cuda")
    out = torch.empty((2, 4, 4), dtype=torch.uint8, device="cuda")
    with pytest.raises(corr.CorrError):  # channel range beyond the PFB
        corr.corr_requantize(x.data_ptr(), 0, 4, 2, 8, 6, 4, 1.0, None, 0, out.data_ptr(), None)
    with pytest.raises(corr.CorrError):  # misaligned samples
        corr.corr_requantize(x.data_ptr() + 4, 0, 4, 2, 8, 0, 4, 1.0, None, 0, out.data_ptr(), None)
    with pytest.raises(corr.CorrError):  # NaN gain
        corr.corr_requantize(x.data_ptr(), 0, 4, 2, 8, 0, 4, float("nan"), None, 0, out.data_ptr(), None)
