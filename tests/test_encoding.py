"""The FP8 tensor path's number encoding and dump correction, checked on the CPU from their
definitions (no GPU, no library code):

* e4m3 (1 sign, 4 exponent bits with bias 7, 3 mantissa bits; exponent field 0 = subnormal): the
  bytes 0x00 .. 0x0F are exactly u * 2^-9 for u = 0 .. 15, so the operand byte of a 4-bit sample v is
  the nibble with its sign bit flipped (u = v + 8);
* a product of two such values is an integer times 2^-18 and every partial sum over at most 65536
  samples is an integer below 2^24 times 2^-18, hence exact in FP32;
* with u = x + 8 + 8i per sample and s = sum_t u per input, the offset-domain sums
  Vu = sum_t u_a conj(u_c) and Au = sum_t |u_a|^2 give back V = Vu - (8 - 8i) s_a - (8 + 8i) conj(s_c)
  + 128 T and A = Au - 16 (Re s + Im s) + 128 T, the cross products and total power of the paper's
  X-engine (Sec. 2.5), exactly in integers.
"""
import numpy as np

from oracle import oracle


def _e4m3(byte: int) -> float:
    sign = -1.0 if byte & 0x80 else 1.0
    e = (byte >> 3) & 0xF
    m = byte & 0x7
    if e == 0:
        return sign * (m / 8.0) * 2.0 ** (1 - 7)
    return sign * (1.0 + m / 8.0) * 2.0 ** (e - 7)


def test_low_e4m3_bytes_are_the_offset_nibbles():
    for u in range(16):
        assert _e4m3(u) == u * 2.0 ** -9
    for v in range(-8, 8):
        nibble = v & 0xF
        assert (nibble ^ 0x8) == v + 8  # flipping the sign bit of the two's-complement nibble


def test_fp32_partial_sums_are_exact_up_to_the_flush_bound():
    # largest |sum| of u_a u_c over 65536 samples, as an integer multiple of 2^-18
    assert 15 * 15 * 65536 < 2 ** 24
    x = np.float32(15 * 2 ** -9) * np.float32(15 * 2 ** -9)
    acc = np.float32(0.0)
    for _ in range(4):  # exact at any partial count: spot-check the top of the range
        acc = np.float32(acc + np.float32(x) * np.float32(16384))
    assert float(acc) * 2 ** 18 == 225 * 65536


def test_dump_correction_recovers_the_visibilities():
    rng = np.random.default_rng(1411)
    T, C, N = 300, 3, 10
    samples = rng.integers(0, 256, size=(T, C, N), dtype=np.uint8)
    samples[:40] = 0x88  # include the -8-8i extreme
    want_cross, want_autos = oracle.correlate(samples, 1)
    re, im = oracle.unpack(samples)
    u = (re + 8) + 1j * (im + 8)  # offset domain, components 0 .. 15
    s = u.sum(axis=0)  # [C][N]
    for f in range(C):
        Vu = np.einsum("ta,tc->ac", u[:, f], np.conj(u[:, f]))
        Au = (np.abs(u[:, f]) ** 2).sum(axis=0)
        V = Vu - (8 - 8j) * s[f][:, None] - (8 + 8j) * np.conj(s[f])[None, :] + 128 * T
        A = Au - 16 * (s[f].real + s[f].imag) + 128 * T
        for a in range(N):
            for c in range(a + 1):
                b = a * (a + 1) // 2 + c
                assert V[a, c].real == want_cross[f, b, 0, 0] and V[a, c].imag == want_cross[f, b, 0, 1]
        assert np.array_equal(np.rint(A).astype(np.int64), want_autos[f])
