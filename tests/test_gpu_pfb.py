"""GPU PFB F-engine (corr_pfb, Sec. 2.2) against the float64 oracle, and the whole F -> X chain.

Tolerance (FP32 FFT of exact integer FIR sums): per spectrum t,
    max_k |X_gpu[k] - X[k]| <= 4 * log2(8192) * 2^-24 * 2^-13 * sqrt(8192) * ||y_t||_2,
i.e. a relative error of a few log2(M) single-precision roundings of the spectrum's L2 norm
(||X_t||_2 ~ 2^-13 sqrt(M / 2) ||y_t||_2 by Parseval), which covers the int32 -> FP32 conversion of
y (2^-24 relative per sample) and the three radix-16 passes and the split step."""
import math

import numpy as np
import pytest

from oracle import oracle

pytestmark = pytest.mark.gpu

M = 8192


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1411_3751_gb300 import corr

    assert torch.cuda.is_available()
    return corr, torch


def _tol(y):
    return 4 * math.log2(M) * 2.0 ** -24 * 2.0 ** -13 * math.sqrt(M) * np.sqrt((y.astype(np.float64) ** 2).sum(-1))


def _check(X_gpu, adc, n_taps):
    X = oracle.pfb(adc, M, n_taps)
    y = oracle.pfb_fir(adc, M, n_taps)
    err = np.abs(X_gpu[..., 0] + 1j * X_gpu[..., 1] - X).max(axis=-1)
    tol = _tol(y)
    assert np.all(err <= tol), float((err / tol).max())
    return float((err / tol).max())


@pytest.mark.parametrize("n_taps", [4, 1, 3])
def test_pfb_random_adc(env, n_taps):
    corr, torch = env
    rng = np.random.default_rng(40 + n_taps)
    N, T = 6, 9
    adc = np.clip(np.rint(rng.standard_normal((N, (T + n_taps - 1) * M)) * 20), -128, 127).astype(np.int8)
    X = corr.pfb(torch.from_numpy(adc).cuda(), n_taps=n_taps).cpu().numpy()
    assert X.shape == (N, T, M // 2, 2)
    _check(X, adc, n_taps)


@pytest.mark.parametrize("pad", [4096, 4])
def test_pfb_extreme_samples_and_strided_inputs(env, pad):
    """Full-scale samples (the int32 FIR sums reach 2^26) and inputs at a row stride beyond the data
    (pad 4: rows only 4-byte aligned, the narrow-load variant)."""
    corr, torch = env
    rng = np.random.default_rng(5)
    N, T, P = 3, 5, 4
    S = (T + P - 1) * M
    adc = rng.choice(np.array([-128, 127], dtype=np.int8), size=(N, S + pad))
    d = torch.from_numpy(adc).cuda()
    coeffs = torch.from_numpy(corr.corr_pfb_coeffs(M, P)).cuda()
    out = torch.empty((N, T, M // 2, 2), dtype=torch.float32, device="cuda")
    corr.corr_pfb(d.data_ptr(), N, d.stride(0), S, P, coeffs.data_ptr(), T, out.data_ptr(), None)
    _check(out.cpu().numpy(), adc[:, :S], P)


def test_pfb_tone_lands_in_its_channel(env):
    """An 8-bit tone at the centre of channel 1235 peaks there; the neighbours are down by the
    prototype filter's response (the 8-bit quantisation of the tone adds low-level spurs)."""
    corr, torch = env
    n = np.arange(7 * M)
    adc = np.rint(100 * np.cos(2 * np.pi * 1235 * n / M)).astype(np.int8)[None, :]
    Xg = corr.pfb(torch.from_numpy(adc).cuda()).cpu().numpy()
    _check(Xg, adc, 4)
    X = Xg[0]
    pw = (X[..., 0] ** 2 + X[..., 1] ** 2).mean(axis=0)
    assert int(np.argmax(pw)) == 1235
    rel = 10 * np.log10(pw / pw[1235] + 1e-30)
    assert rel[1234] < -45 and rel[1236] < -45 and np.r_[rel[1190:1233], rel[1238:1280]].max() < -60


def test_f_engine_to_x_engine_chain(env):
    """ADC -> PFB -> requantiser -> X-engine on the device. The requantised bytes equal the oracle's
    requantiser applied to the GPU PFB output (same float32 values, same decisions), and the
    visibilities equal the oracle's correlation of those bytes."""
    corr, torch = env
    rng = np.random.default_rng(77)
    N, T, P, chan0, C, npol = 32, 12, 4, 1000, 96, 2
    common = rng.standard_normal((T + P - 1) * M) * 12
    adc = np.clip(np.rint(rng.standard_normal((N, (T + P - 1) * M)) * 15 + common), -128, 127).astype(np.int8)
    X = corr.pfb(torch.from_numpy(adc).cuda())
    Xh = X.cpu().numpy()
    gain = float(np.float32(2.5 / Xh[:, :, chan0:chan0 + C].std()))  # about 2.5 levels per sigma
    q = corr.requantize(X, chan0, C, gain=gain)
    assert np.array_equal(q.cpu().numpy(), oracle.requantize(Xh, chan0, C, gain=gain))
    with corr.Correlator(N, C, T, npol) as xc:
        xc.accumulate(q)
        cross = xc.dump(corr.CORR_WHAT_CROSS).cpu().numpy()
        autos = xc.dump(corr.CORR_WHAT_AUTO).cpu().numpy()
        xc.sync()
    want_c, want_a = oracle.correlate(q.cpu().numpy(), npol, threads=8)
    assert np.array_equal(cross, want_c) and np.array_equal(autos, want_a)
    _check(Xh, adc, P)


def test_pfb_rejects_bad_arguments(env):
    corr, torch = env
    d = torch.zeros((2, 4 * M), dtype=torch.int8, device="cuda")
    coeffs = torch.from_numpy(corr.corr_pfb_coeffs(M, 4)).cuda()
    out = torch.empty((2, 2, M // 2, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(corr.CorrError):  # 2 spectra need 5 frames
        corr.corr_pfb(d.data_ptr(), 2, d.stride(0), 4 * M, 4, coeffs.data_ptr(), 2, out.data_ptr(), None)
    with pytest.raises(corr.CorrError):  # misaligned samples
        corr.corr_pfb(d.data_ptr() + 1, 2, d.stride(0), 4 * M - 1, 4, coeffs.data_ptr(), 1, out.data_ptr(), None)
