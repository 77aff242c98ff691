"""Host-side checks of the C ABI: the library loads, exports every symbol declared in include/*.h,
and rejects bad arguments before touching the GPU. No compute calls (runs without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(inc, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(corr_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1411_3751_gb300 import corr

    return corr


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert "corr_create" in names and "corr_dump" in names and len(names) >= 15
    raw = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing
    bound = {n for n, _, _ in lib.SIGNATURES}
    assert set(names) <= bound, set(names) - bound


def test_host_only_helpers(lib):
    assert lib.corr_n_baselines(512, 2) == 32896
    assert lib.corr_n_baselines(32, 2) == 136
    assert lib.corr_n_baselines(7, 2) == 0
    assert lib.corr_n_baselines(0, 1) == 0
    fp = lib.corr_footprint_bytes(512, 128, 8192, 2, lib.CORR_PATH_FP8TC)
    acc = 128 * 32896 * 4 * 2 * 8 + 128 * 512 * 8
    assert fp >= acc
    assert fp >= acc + 128 * 8192 * 1024  # operand scratch of the two-pass tensor path
    assert lib.corr_footprint_bytes(512, 128, 8192, 2, lib.CORR_PATH_AUTO) == fp
    assert lib.corr_footprint_bytes(512, 128, 8192, 2, lib.CORR_PATH_FP32) < fp
    assert lib.corr_footprint_bytes(512, 128, 8192, 2, lib.CORR_PATH_FP8TC_FUSED) == fp  # may fall back to two passes
    assert lib.corr_footprint_bytes(512, 128, 8192, 2, lib.CORR_PATH_I8MMA) < fp  # no operand scratch
    assert lib.corr_footprint_bytes(4, 65536, 1, 2, lib.CORR_PATH_FP32) == 0     # channel limit
    assert lib.corr_footprint_bytes(0, 1, 1, 1, 0) == 0
    assert lib.corr_footprint_bytes(3, 1, 1, 2, 0) == 0
    assert lib.corr_footprint_bytes(4, 1, 1, 2, 99) == 0
    assert "sm_103a" in lib.corr_version()


@pytest.mark.parametrize("args", [(0, 1, 1, 1), (4, 0, 1, 2), (4, 1, 0, 2), (5, 1, 1, 2), (4, 1, 1, 3), (-2, 1, 1, 1),
                                  (4, 65536, 1, 2), (65536, 1, 1, 2)])
def test_create_rejects_bad_shapes(lib, args):
    with pytest.raises(lib.CorrError) as ei:
        lib.corr_create(*args)
    assert "invalid shape" in str(ei.value)


def test_null_context_errors(lib):
    assert lib._lib.corr_set_path(None, 0) == lib.CORR_ERR_ARG
    assert lib._lib.corr_accumulate(None, None, None) == lib.CORR_ERR_ARG
    assert lib._lib.corr_dump(None, None, 1, 1, 0, 0, None) == lib.CORR_ERR_ARG
    assert "NULL context" in lib.corr_last_error()
    assert lib._lib.corr_destroy(None) == lib.CORR_OK


def test_corner_turn_rejects_bad_bounds_before_touching_the_device(lib):
    import ctypes

    fake = ctypes.c_void_p(16)
    for bounds in ([0, 3], [1, 4], [0, 3, 2, 4], [0]):
        b = (ctypes.c_int * len(bounds))(*bounds)
        assert lib._lib.corr_corner_turn_pack(fake, 2, 4, 8, b, len(bounds) - 1, fake, None) == lib.CORR_ERR_ARG
        assert lib._lib.corr_corner_turn_unpack(fake, 2, 3, 4, b, len(bounds) - 1, fake, None) == lib.CORR_ERR_ARG
    assert "bounds" in lib.corr_last_error()


def test_probe_rejects_bad_sizes_before_touching_the_device(lib):
    for n_mma, n_cols in ((0, 256), (1 << 21, 256), (16, 64), (16, 192)):
        assert lib._lib.corr_probe_mma_rate(n_mma, n_cols, None, None, None) == lib.CORR_ERR_ARG
    assert "n_cols 128 or 256" in lib.corr_last_error()


def test_pfb_coeffs_match_the_oracle(lib):
    """The library's host-side PFB prototype filter equals the oracle's independent computation."""
    import numpy as np

    from oracle import oracle

    for n_fft, n_taps in ((8192, 4), (64, 3), (2, 1)):
        np.testing.assert_array_equal(lib.corr_pfb_coeffs(n_fft, n_taps), oracle.pfb_coeffs(n_fft, n_taps))
    with pytest.raises(lib.CorrError):
        lib.corr_pfb_coeffs(100, 4)


@pytest.mark.parametrize("plan", [0, 1, 2, 3])
def test_tile_plans_cover_the_triangle_exactly_once(plan):
    """Host logic of the tensor path's work decomposition: for every input count, the tiles of a
    channel (both halves of a plan-2 pair, both SMs of a plan-3 pair) cover each pair a >= c of real
    inputs exactly once, start within the padded operand rows (plans 0-2 also end within them), and
    use the MMA widths 128 and 256 only."""
    from paper_1411_3751_gb300 import corr

    for N in list(range(1, 200)) + [255, 256, 257, 383, 384, 511, 512, 513, 640, 1000, 1024]:
        R = -(-2 * N // 128) * 128
        seen = np.zeros((N, N), dtype=np.int32)
        for c0, a0, nb, extra in corr.corr_tile_plan(N, plan):
            halves = [(c0, a0, nb)]
            if plan == 2 and extra & 0xFFFF:
                halves.append((c0 + 64, a0 + 64 * (extra >> 16), extra & 0xFFFF))
            elif plan == 3:
                assert nb == 256 and extra == 0 and c0 % 128 == 0 and a0 % 128 == 0
                halves.append((c0 + 64, a0, nb))  # the pair's second SM: the next 64 c-inputs
            else:
                assert extra == 0 or plan == 2
            for cc, aa, w in halves:
                assert w in (128, 256) and cc % 64 == 0 and aa % 64 == 0
                if plan == 3:  # rows past R are read as zeros (inputs >= N)
                    assert 2 * aa < R and 2 * c0 < R, (N, plan, cc, aa, w)
                else:
                    assert 2 * aa + w <= R and 2 * cc + 128 <= R, (N, plan, cc, aa, w)
                c = np.arange(cc, min(cc + 64, N))[:, None]
                a = np.arange(aa, min(aa + w // 2, N))[None, :]
                m = (a >= c)
                seen[np.broadcast_to(c, m.shape)[m], np.broadcast_to(a, m.shape)[m]] += 1
        tri = np.triu(np.ones((N, N), dtype=np.int32))  # seen[c, a] for a >= c
        assert np.array_equal(seen, tri), (N, plan)
    with pytest.raises(corr.CorrError):
        corr.corr_tile_plan(0, plan)
    with pytest.raises(corr.CorrError):
        corr.corr_tile_plan(8, 4)


def test_channel_group_rule():
    """Host logic of the channel groups: under tile plans 0 and 1 an array of at most 16 inputs
    (32 operand rows per channel) multiplies 4 channels per work item and one of 17 .. 32 inputs (64
    rows) 2, each item being the one tile (0, 0, 128) of the plan that covers the whole triangle, so
    that the g channels fill the tile's 128 rows exactly; every other case takes one channel per
    item."""
    from paper_1411_3751_gb300 import corr

    for N in list(range(1, 70)) + [96, 512, 1 << 20]:
        for plan in range(4):
            g = corr.corr_channel_group(N, plan)
            want = (4 if N <= 16 else 2 if N <= 32 else 1) if plan < 2 else 1
            assert g == want, (N, plan, g)
            if g > 1:
                rows = -(-2 * N // 32) * 32  # operand rows stored per channel
                assert g * rows == 128, (N, g)
                assert corr.corr_tile_plan(N, plan) == [(0, 0, 128, 0)], (N, plan)
    for bad in ((0, 0), (1 << 21, 0), (8, 4), (8, -1)):
        with pytest.raises(corr.CorrError):
            corr.corr_channel_group(*bad)


def test_batch_launch_length_rule():
    """Host logic of corr_accumulate_batch's launch length: the benchmark's 512-input shape shares
    4 blocks of 8192 samples per launch, 256 inputs 2; every launch stays within 65536 samples (the
    FP32 partial sums' exactness bound) and its operand within 8 GiB unless one block alone exceeds
    that; at least one block; invalid shapes give 0."""
    from paper_1411_3751_gb300 import corr

    assert corr.corr_batch_blocks(512, 128, 8192, 2) == 4
    assert corr.corr_batch_blocks(256, 128, 8192, 2) == 2
    assert corr.corr_batch_blocks(0, 1, 1, 1) == 0 and corr.corr_batch_blocks(3, 1, 1, 2) == 0
    for N in (1, 2, 32, 64, 96, 200, 512, 1024, 2048):
        for C in (1, 8, 128, 2400):
            for T in (1, 240, 1000, 4096, 8192, 65536):
                K = corr.corr_batch_blocks(N, C, T, 1 if N % 2 else 2)
                T_pad = -(-T // 128) * 128
                op = C * T_pad * (-(-2 * N // 32) * 32)
                assert K >= 1, (N, C, T)
                assert K == 1 or K * T_pad <= 65536, (N, C, T, K)
                assert K == 1 or K * op <= 8 << 30, (N, C, T, K)
