"""Pins for the CPU oracle: each test ties it to something other than itself.

* brute force with numpy integer matrix products (exact) on tiny inputs, every cell;
* closed forms: a rank-1 injected common signal (the exact version of the CW test tone of Sec. 5),
  orthogonal Walsh-Hadamard codes (rank > 1), constant extremes, alternating signs;
* an int64 overflow pin (a sum that wraps int32);
* invariants: Hermitian auto-station blocks, real non-negative autos, Cauchy-Schwarz, linearity
  in time, zero padding, permutation of inputs;
* golden fixtures under tests/golden/ with hand-derived values.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rand_bytes(rng, T, C, N):
    return rng.integers(0, 256, size=(T, C, N), dtype=np.uint8)


def _brute_full(samples):
    """Full N x N Hermitian matrix per channel via exact int64 matrix products."""
    re, im = oracle.unpack(samples)  # [T][C][N]
    out_re = np.einsum("tcn,tcm->cnm", re, re) + np.einsum("tcn,tcm->cnm", im, im)
    out_im = np.einsum("tcn,tcm->cnm", im, re) - np.einsum("tcn,tcm->cnm", re, im)
    return out_re, out_im


def _triangle_from_full(full_re, full_im, n_pol):
    C, N, _ = full_re.shape
    S = N // n_pol
    bs = S * (S + 1) // 2
    out = np.zeros((C, bs, n_pol * n_pol, 2), dtype=np.int64)
    for a in range(S):
        for c in range(a + 1):
            b = a * (a + 1) // 2 + c
            for p in range(n_pol):
                for q in range(n_pol):
                    i, j = a * n_pol + p, c * n_pol + q
                    out[:, b, p * n_pol + q, 0] = full_re[:, i, j]
                    out[:, b, p * n_pol + q, 1] = full_im[:, i, j]
    return out


@pytest.mark.parametrize("n_pol", [1, 2])
@pytest.mark.parametrize("shape", [(1, 1, 2), (7, 3, 4), (64, 2, 8), (33, 4, 6)])
def test_brute_force_every_cell(n_pol, shape):
    T, C, N = shape
    rng = np.random.default_rng(1000 + T * 7 + N)
    s = _rand_bytes(rng, T, C, N)
    cross, autos = oracle.correlate(s, n_pol)
    fr, fi = _brute_full(s)
    np.testing.assert_array_equal(cross, _triangle_from_full(fr, fi, n_pol))
    np.testing.assert_array_equal(autos, np.einsum("cnn->cn", fr))


def test_threads_do_not_change_result():
    rng = np.random.default_rng(5)
    s = _rand_bytes(rng, 50, 9, 10)
    a = oracle.correlate(s, 2, threads=1)
    b = oracle.correlate(s, 2, threads=4)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_cells_match_brute_force_any_order():
    rng = np.random.default_rng(6)
    s = _rand_bytes(rng, 40, 3, 8)
    fr, fi = _brute_full(s)
    cl = [(f, i, j) for f in range(3) for i in range(8) for j in range(8)]
    got = oracle.cells(s, cl)
    for k, (f, i, j) in enumerate(cl):
        assert got[k, 0] == fr[f, i, j] and got[k, 1] == fi[f, i, j]


def test_autos_entry_point_matches_brute_force():
    rng = np.random.default_rng(7)
    s = _rand_bytes(rng, 30, 5, 12)
    fr, _ = _brute_full(s)
    np.testing.assert_array_equal(oracle.autos(s), np.einsum("cnn->cn", fr))


def test_rank1_common_signal_closed_form():
    """x_m(t) = c_m s(t), s(t) in {1, -1, i, -i}: V[m, n] = T c_m conj(c_n), A[m] = T |c_m|^2."""
    rng = np.random.default_rng(11)
    T, C, N, n_pol = 96, 2, 12, 2
    cm = rng.integers(-7, 8, size=(C, N)) + 1j * rng.integers(-7, 8, size=(C, N))
    st = np.array([1, -1, 1j, -1j])[rng.integers(0, 4, size=(T, C))]
    x = st[:, :, None] * cm[None, :, :]
    s = oracle.pack(np.real(x).astype(np.int64), np.imag(x).astype(np.int64))
    cross, autos = oracle.correlate(s, n_pol)
    S = N // n_pol
    for f in range(C):
        for a in range(S):
            for c in range(a + 1):
                b = a * (a + 1) // 2 + c
                for p in range(n_pol):
                    for q in range(n_pol):
                        v = T * cm[f, a * n_pol + p] * np.conj(cm[f, c * n_pol + q])
                        assert cross[f, b, p * n_pol + q, 0] == int(round(v.real))
                        assert cross[f, b, p * n_pol + q, 1] == int(round(v.imag))
        np.testing.assert_array_equal(autos[f], (T * np.abs(cm[f]) ** 2).round().astype(np.int64))


def _hadamard(r):
    h = np.array([[1]], dtype=np.int64)
    for _ in range(r):
        h = np.block([[h, h], [h, -h]])
    return h


def test_walsh_hadamard_codes_closed_form():
    """x_m(t) = sum_k c_{mk} h_k(t) with orthogonal +-1 codes: V = T C C^H exactly (rank > 1)."""
    rng = np.random.default_rng(12)
    r, K, N, C = 6, 3, 10, 1
    T = 2 ** r
    h = _hadamard(r)[[3, 17, 40]]  # K codes, each length T
    cre = rng.integers(-2, 3, size=(N, K))
    cim = rng.integers(-2, 3, size=(N, K))
    xre = (cre @ h).T  # [T][N]
    xim = (cim @ h).T
    s = oracle.pack(xre[:, None, :], xim[:, None, :])
    cross, autos = oracle.correlate(s, 1)
    cm = cre + 1j * cim
    V = T * cm @ cm.conj().T
    for a in range(N):
        for c in range(a + 1):
            b = a * (a + 1) // 2 + c
            assert cross[0, b, 0, 0] == int(round(V[a, c].real))
            assert cross[0, b, 0, 1] == int(round(V[a, c].imag))
    np.testing.assert_array_equal(autos[0], np.round(np.real(np.diag(V))).astype(np.int64))
    assert np.linalg.matrix_rank(V) == K


@pytest.mark.parametrize("re,im,expect_re", [(-8, -8, 128), (7, 7, 98), (-8, 7, 113), (0, -8, 64)])
def test_constant_extremes(re, im, expect_re):
    T, C, N = 37, 2, 6
    s = oracle.pack(np.full((T, C, N), re), np.full((T, C, N), im))
    cross, autos = oracle.correlate(s, 2)
    assert np.all(cross[..., 0] == expect_re * T)
    assert np.all(cross[..., 1] == 0)
    assert np.all(autos == expect_re * T)


def test_alternating_signs_cancel():
    """Input 0 alternates sign each sample, input 1 is constant: their product sums to 0 over even T."""
    T = 64
    re = np.zeros((T, 1, 2), dtype=np.int64)
    im = np.zeros((T, 1, 2), dtype=np.int64)
    sign = np.where(np.arange(T) % 2 == 0, 1, -1)
    re[:, 0, 0] = 5 * sign
    im[:, 0, 0] = -3 * sign
    re[:, 0, 1] = 4
    im[:, 0, 1] = 2
    cross, autos = oracle.correlate(oracle.pack(re, im), 1)
    assert tuple(cross[0, 1, 0]) == (0, 0)  # pair (1, 0)
    assert autos[0, 0] == 34 * T and autos[0, 1] == 20 * T


def test_int64_overflow_pin():
    """2^25 samples of -8-8i: Re V = 128 * 2^25 = 2^32, which an int32 accumulator would wrap to 0."""
    T = 2 ** 25
    s = np.full((T, 1, 2), 0x88, dtype=np.uint8)
    cross, autos = oracle.correlate(s, 1)
    assert np.all(cross[0, :, 0, 0] == 2 ** 32)
    assert np.all(cross[0, :, 0, 1] == 0)
    assert np.all(autos == 2 ** 32)


def test_invariants_random():
    rng = np.random.default_rng(21)
    T, C, N, n_pol = 200, 3, 16, 2
    s = _rand_bytes(rng, T, C, N)
    cross, autos = oracle.correlate(s, n_pol)
    S = N // n_pol
    assert np.all(autos >= 0)
    for a in range(S):
        b = a * (a + 1) // 2 + a
        xx, xy, yx, yy = cross[:, b, 0], cross[:, b, 1], cross[:, b, 2], cross[:, b, 3]
        # auto-station XX / YY are real and equal the autos; YX = conj(XY)
        np.testing.assert_array_equal(xx[:, 0], autos[:, 2 * a])
        np.testing.assert_array_equal(yy[:, 0], autos[:, 2 * a + 1])
        assert np.all(xx[:, 1] == 0) and np.all(yy[:, 1] == 0)
        np.testing.assert_array_equal(yx[:, 0], xy[:, 0])
        np.testing.assert_array_equal(yx[:, 1], -xy[:, 1])
    # Cauchy-Schwarz |V_mn|^2 <= A_m A_n
    for a in range(S):
        for c in range(a + 1):
            b = a * (a + 1) // 2 + c
            for p in range(2):
                for q in range(2):
                    v = cross[:, b, p * 2 + q]
                    mag2 = v[:, 0] ** 2 + v[:, 1] ** 2
                    assert np.all(mag2 <= autos[:, 2 * a + p] * autos[:, 2 * c + q])


def test_linearity_and_zero_padding():
    rng = np.random.default_rng(22)
    s1 = _rand_bytes(rng, 57, 2, 8)
    s2 = _rand_bytes(rng, 31, 2, 8)
    c1, a1 = oracle.correlate(s1, 2)
    c2, a2 = oracle.correlate(s2, 2)
    c12, a12 = oracle.correlate(np.concatenate([s1, s2]), 2)
    np.testing.assert_array_equal(c12, c1 + c2)
    np.testing.assert_array_equal(a12, a1 + a2)
    cz, az = oracle.correlate(np.concatenate([s1, np.zeros((40, 2, 8), np.uint8)]), 2)
    np.testing.assert_array_equal(cz, c1)
    np.testing.assert_array_equal(az, a1)


def test_permutation_of_inputs():
    """Swapping inputs 1 and 4 (n_pol = 1) moves V[4, 1] to conj(V[4, 1]) at the swapped position."""
    rng = np.random.default_rng(23)
    s = _rand_bytes(rng, 45, 1, 6)
    c0, a0 = oracle.correlate(s, 1)
    perm = np.array([0, 4, 2, 3, 1, 5])
    cp, ap = oracle.correlate(s[:, :, perm], 1)
    np.testing.assert_array_equal(ap[0], a0[0][perm])

    def full(cr):
        V = np.zeros((6, 6), dtype=np.complex128)
        for a in range(6):
            for c in range(a + 1):
                v = cr[0, a * (a + 1) // 2 + c, 0]
                V[a, c] = v[0] + 1j * v[1]
                V[c, a] = v[0] - 1j * v[1]
        return V

    np.testing.assert_array_equal(full(cp), full(c0)[np.ix_(perm, perm)])


def test_dump_formats():
    v = np.array([0, 1, -3, 2 ** 31 + 1, 2 ** 40 + 3, -(2 ** 33) - 7], dtype=np.int64)
    np.testing.assert_array_equal(oracle.to_format(v, oracle.FMT_CI64, 10), v)
    f = oracle.to_format(v, oracle.FMT_CF32, 10)
    assert f.dtype == np.float32
    assert f[3] == np.float32(2 ** 31) and f[4] == np.float32(2 ** 40)
    n = oracle.to_format(v, oracle.FMT_CF32_NORM, 3)
    assert n[2] == np.float32(-1.0) and n[1] == np.float32(1 / 3)
    assert np.all(oracle.to_format(v, oracle.FMT_CF32_NORM, 0) == 0)


def test_golden_fixtures():
    """Hand-derived values (see each fixture's "derivation" field)."""
    files = sorted(f for f in os.listdir(GOLDEN) if f.startswith("xengine_") and f.endswith(".json"))
    assert files, "no golden fixtures"
    for name in files:
        with open(os.path.join(GOLDEN, name)) as fh:
            g = json.load(fh)
        re = np.array(g["re"], dtype=np.int64)
        im = np.array(g["im"], dtype=np.int64)
        s = oracle.pack(re, im)
        cross, autos = oracle.correlate(s, g["n_pol"])
        np.testing.assert_array_equal(cross, np.array(g["cross"], dtype=np.int64), err_msg=name)
        np.testing.assert_array_equal(autos, np.array(g["autos"], dtype=np.int64), err_msg=name)


def test_pack_unpack_roundtrip_and_range():
    vals = np.arange(-8, 8)
    re, im = np.meshgrid(vals, vals)
    b = oracle.pack(re, im)
    r2, i2 = oracle.unpack(b)
    np.testing.assert_array_equal(r2, re)
    np.testing.assert_array_equal(i2, im)
    assert oracle.pack(np.array([-8]), np.array([7]))[0] == 0x87
    with pytest.raises(ValueError):
        oracle.pack(np.array([8]), np.array([0]))


@pytest.mark.parametrize("n_pol", [1, 2])
def test_station_subset_brute_force(n_pol):
    """Selected-station cells (Sec. 2.6) against the brute-force Hermitian matrix, for an unordered
    station list: element (k, l, p, q) = V[st[k] p, st[l] q], conjugated storage when st[k] < st[l]."""
    rng = np.random.default_rng(31 + n_pol)
    T, C, S = 57, 3, 6
    s = _rand_bytes(rng, T, C, S * n_pol)
    fr, fi = _brute_full(s)
    st = [4, 1, 5, 0]
    got = oracle.station_cross(s, st, n_pol)
    for k in range(len(st)):
        for l in range(k + 1):
            for p in range(n_pol):
                for q in range(n_pol):
                    i, j = st[k] * n_pol + p, st[l] * n_pol + q
                    e = got[:, k * (k + 1) // 2 + l, p * n_pol + q]
                    np.testing.assert_array_equal(e[:, 0], fr[:, i, j])
                    np.testing.assert_array_equal(e[:, 1], fi[:, i, j])
    ga = oracle.station_autos(s, st, n_pol)
    for k, a in enumerate(st):
        for p in range(n_pol):
            np.testing.assert_array_equal(ga[:, k, p], np.einsum("cnn->cn", fr)[:, a * n_pol + p])


def test_station_subset_of_all_stations_is_the_full_dump():
    rng = np.random.default_rng(77)
    s = _rand_bytes(rng, 40, 2, 10)
    cross, autos = oracle.correlate(s, 2)
    np.testing.assert_array_equal(oracle.station_cross(s, range(5), 2), cross)
    np.testing.assert_array_equal(oracle.station_autos(s, range(5), 2).reshape(2, 10), autos)


def _half_even_div(v: int, k: int) -> int:
    """round(v / 2^k), ties to even, in exact integer arithmetic."""
    q, r = divmod(v, 1 << k)
    half = 1 << (k - 1)
    if r > half or (r == half and q % 2 == 1):
        q += 1
    return q


def test_requantize_power_of_two_gain_matches_integer_rounding():
    """gain = 2^-k makes the float product exact: the result is integer round-half-even then clip."""
    rng = np.random.default_rng(5)
    N, T, F = 3, 4, 9
    x = rng.integers(-(1 << 17), 1 << 17, size=(N, T, F, 2)).astype(np.int32)
    x[0, 0, 0] = (3 << 12, -(5 << 12))   # exact ties +-1.5 / 2.5 at k = 13
    x[0, 0, 1] = (1 << 12, -(1 << 12))   # +-0.5
    got = oracle.requantize(x, chan0=2, n_chans=6, gain=2.0 ** -13)
    for n in range(N):
        for t in range(T):
            for c in range(6):
                q = [min(7, max(-8, _half_even_div(int(v), 13))) for v in x[n, t, 2 + c]]
                assert got[t, c, n] == (((q[0] & 0xF) << 4) | (q[1] & 0xF))
    assert oracle.requantize(x, 0, 2, 2.0 ** -13)[0, 0, 0] == (((2 & 0xF) << 4) | (-2 & 0xF))
    assert oracle.requantize(x, 0, 2, 2.0 ** -13)[0, 1, 0] == 0x00


def test_requantize_identity_clip_and_specials():
    # integers already in range pass through unchanged with gain 1
    v = np.arange(-8, 8, dtype=np.int32)
    x = np.stack(np.meshgrid(v, v, indexing="ij"), axis=-1).reshape(1, 1, 256, 2)
    got = oracle.requantize(x, 0, 256, 1.0)
    np.testing.assert_array_equal(got[0, :, 0], oracle.pack(x[0, 0, :, 0], x[0, 0, :, 1]))
    # clipping, the symmetric variant, NaN and infinities
    f = np.array([[[[100.0, -100.0], [np.nan, np.inf], [-np.inf, 7.5], [-8.5, 6.5]]]], dtype=np.float32)
    full = oracle.requantize(f, 0, 4, 1.0)[0, :, 0]
    sym = oracle.requantize(f, 0, 4, 1.0, symmetric=True)[0, :, 0]
    np.testing.assert_array_equal(full, [0x78, 0x07, 0x87, 0x86])  # (7,-8) (0,7) (-8,7: 7.5 -> 8 -> 7) (-8, 6)
    np.testing.assert_array_equal(sym, [0x79, 0x07, 0x97, 0x96])


def test_requantize_gain_product_is_single_precision():
    """The gain product is one IEEE single-precision multiply, rounded before rint: for v = 3 and the
    float32 gains 0x3F555556 (13981014 / 2^24) and 0x3F955555 (9786709 / 2^23) the exact products are
    2.5 + 2^-23 and 3.5 - 2^-23, half an ulp from the half-integers, and round (ties to even) to 2.5
    and 3.5 in float32; rint then gives 2 and 4 where the exact products would give 3 and 3."""
    g1 = np.array([0x3F555556], dtype=np.uint32).view(np.float32)[0]
    g2 = np.array([0x3F955555], dtype=np.uint32).view(np.float32)[0]
    assert float(g1) == 13981014 / 2 ** 24 and float(g2) == 9786709 / 2 ** 23
    x = np.array([[[[3, -3]]]], dtype=np.int32)
    assert oracle.requantize(x, 0, 1, gain=g1)[0, 0, 0] == ((2 << 4) | (-2 & 0xF))   # 0x2E
    assert oracle.requantize(x, 0, 1, gain=g2)[0, 0, 0] == ((4 << 4) | (-4 & 0xF))   # 0x4C
    assert oracle.requantize(x.astype(np.float32), 0, 1, gains=np.array([g2], np.float32))[0, 0, 0] == 0x4C


def test_requantize_corner_turn_and_per_channel_gains():
    rng = np.random.default_rng(8)
    N, T, F = 5, 3, 11
    x = (rng.standard_normal((N, T, F, 2)) * 3).astype(np.float32)
    g = np.linspace(0.5, 2.0, 7).astype(np.float32)
    got = oracle.requantize(x, 3, 7, gains=g)
    for n in range(N):
        for t in range(T):
            for c in range(7):
                q = [int(min(7, max(-8, np.rint(np.float32(g[c]) * x[n, t, 3 + c, k])))) for k in range(2)]
                assert got[t, c, n] == (((q[0] & 0xF) << 4) | (q[1] & 0xF))
    np.testing.assert_array_equal(oracle.requantize(x, 3, 7, gains=np.full(7, 1.25, np.float32)),
                                  oracle.requantize(x, 3, 7, gain=1.25))


def test_pfb_coeffs_shape_symmetry_and_peak():
    h = oracle.pfb_coeffs(8192, 4)
    assert h.shape == (32768,) and np.abs(h).max() == 131071
    np.testing.assert_array_equal(h, h[::-1])                      # linear phase
    assert h[16383] == h[16384] == 131071                          # peak at the centre
    assert abs(h[0]) < 131071 * 0.08 / 1000 + 1                    # Hamming end value 0.08 x a tiny sinc
    g = oracle.pfb_coeffs(16, 3)
    np.testing.assert_array_equal(g, g[::-1])


def test_pfb_fir_and_dft_brute_force():
    """Tiny PFB (M = 8, 3 taps) against plain loops: FIR sums and the DFT definition."""
    rng = np.random.default_rng(3)
    M, P, T, N = 8, 3, 5, 2
    adc = rng.integers(-128, 128, size=(N, (T + P - 1) * M)).astype(np.int8)
    h = oracle.pfb_coeffs(M, P)
    X = oracle.pfb(adc, M, P)
    for n in range(N):
        for t in range(T):
            y = [sum(int(h[p * M + m]) * int(adc[n, (t + p) * M + m]) for p in range(P)) for m in range(M)]
            for k in range(M // 2):
                want = sum(y[m] * np.exp(-2j * np.pi * k * m / M) for m in range(M)) / M
                assert abs(X[n, t, k] - want) < 1e-9 * (1 + abs(want))


def test_pfb_channel_response_of_a_tone():
    """A tone at the centre of channel k0 lands in k0; the leakage follows the prototype filter's
    response: -50 dB one channel away (the transition band of the 4-tap Hamming design), below -68 dB
    two or more channels away, and a tone on a channel edge splits equally (-6 dB each)."""
    M, P = 8192, 4
    n = np.arange((P + 3) * M, dtype=np.float64)
    for k0 in (100, 1500, 3000):
        X = oracle.pfb(np.cos(2 * np.pi * k0 * n / M)[None, :], M, P)[0]
        pw = np.abs(X).mean(axis=0) ** 2
        assert np.argmax(pw) == k0
        rel = 10 * np.log10(pw / pw[k0])
        assert -51.0 < rel[k0 - 1] < -49.0 and -51.0 < rel[k0 + 1] < -49.0
        far = np.r_[rel[k0 - 40:k0 - 1], rel[k0 + 2:k0 + 41]]
        assert far.max() < -68.0
    X = oracle.pfb(np.cos(2 * np.pi * 700.5 * n / M)[None, :], M, P)[0]
    pw = np.abs(X).mean(axis=0) ** 2
    assert abs(10 * np.log10(pw[700] / pw[701])) < 0.01


def test_pfb_linearity():
    rng = np.random.default_rng(9)
    a = rng.standard_normal((2, 5 * 64))
    b = rng.standard_normal((2, 5 * 64))
    np.testing.assert_allclose(oracle.pfb(3 * a - 2 * b, 64, 4), 3 * oracle.pfb(a, 64, 4) - 2 * oracle.pfb(b, 64, 4),
                               atol=1e-12)
