"""The seeded input generator: determinism, sub-block consistency, and the workload statistics it is
meant to have (sanity, not parity)."""
import numpy as np
import pytest

from oracle import oracle


@pytest.fixture(scope="module")
def synth():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1411_3751_gb300 import synth as s

    return s


def test_uniform_is_deterministic_and_subblocks_agree(synth):
    spec = synth.Spec(kind="uniform", seed=7)
    a = synth.generate_host(spec, 64, 5, 12)
    b = synth.generate_host(spec, 64, 5, 12)
    assert np.array_equal(a, b)
    sub = synth.generate_host(spec, 64, 5, 12, t_range=(10, 30), c_range=(2, 4))
    assert np.array_equal(sub, a[10:30, 2:4])
    shifted = synth.generate_host(spec, 20, 5, 12, t0=10)
    assert np.array_equal(shifted, a[10:30])
    other = synth.generate_host(synth.Spec(kind="uniform", seed=8), 64, 5, 12)
    assert not np.array_equal(a, other)


def test_uniform_nibbles_cover_range(synth):
    a = synth.generate_host(synth.Spec(kind="uniform", seed=3), 512, 4, 64)
    re, im = oracle.unpack(a)
    for comp in (re, im):
        counts = np.bincount((comp + 8).ravel(), minlength=16)
        assert counts.min() > 0.8 * comp.size / 16 and counts.max() < 1.2 * comp.size / 16


def test_gauss_tone_statistics(synth):
    spec = synth.Spec(kind="gauss_tone", seed=11, sigma=2.5, rho=0.1)
    T, C, N = 16384, 2, 6
    a = synth.generate_host(spec, T, C, N)
    re, im = oracle.unpack(a)
    x = re + 1j * im
    # per-component standard deviation close to sqrt(sigma^2 + A^2 / 2) (before light clipping)
    A = spec.tone_amplitude()
    want = np.sqrt(2.5 ** 2 + 1.0 / 12.0 + A * A / 2.0)  # + rounding noise
    assert abs(np.std(re) - want) < 0.08 and abs(np.std(im) - want) < 0.08
    # the injected common tone: V_mn / T ~ A^2 exp(i (phi_m - phi_n)), |rho| ~ 0.1
    ph = synth.phases_radians(spec, N)
    for m in range(1, N):
        v = np.mean(x[:, 0, m] * np.conj(x[:, 0, 0]))
        expect = A * A * np.exp(1j * (ph[m] - ph[0]))
        assert abs(v - expect) < 5.0 * (2 * 2.5 ** 2) / np.sqrt(T) + 0.05 * A * A


def test_saturate_profile_segments(synth):
    spec = synth.Spec(kind="saturate", seed=5, seg_len=256, m8_segment=3)
    a = synth.generate_host(spec, 1024, 1, 8)
    assert np.all(a[768:1024] == 0x88)
    re, _ = oracle.unpack(a)
    clip_lo = np.mean(np.abs(re[0:256]) >= 7)
    clip_hi = np.mean(np.abs(re[256:512]) >= 7)
    assert clip_hi > 3 * clip_lo


def test_bad_params_rejected(synth):
    with pytest.raises(ValueError):
        synth.generate_host(synth.Spec(kind="gauss_tone", sigma=40.0), 4, 1, 4)
