"""The corner turn's device halves (libcorr's pack and unpack kernels) on one GPU: the ranks' all-to-all
is emulated by slicing the packed buffers, every rank's result is compared byte for byte with the
channel range of the full band, and one turned shard is correlated on the tensor path against the
oracle. (The exchange itself runs on gloo ranks in tests/test_replicas.py.)"""
import numpy as np
import pytest

from oracle import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1411_3751_gb300 import corr, replicas, synth

    assert torch.cuda.is_available()
    return corr, replicas, synth, torch


@pytest.mark.parametrize("world,N,C,T,npol", [(2, 512, 16, 256, 2), (3, 96, 7, 100, 2), (4, 30, 9, 33, 1),
                                              (5, 64, 3, 17, 2)])
def test_pack_unpack_emulated_all_to_all(env, world, N, C, T, npol):
    corr, replicas, synth, torch = env
    full_h = synth.generate_host(synth.Spec(kind="gauss_tone", seed=N + C), T, C, N)
    full = torch.from_numpy(full_h).cuda()
    ch = replicas.channel_shards(C, world)
    ins = replicas.input_shards(N, world, npol)
    stream = torch.cuda.current_stream().cuda_stream
    chan_bounds = [a for a, _ in ch] + [C]
    input_bounds = [a for a, _ in ins] + [N]
    sends = []
    for n0, n1 in ins:
        x = full[:, :, n0:n1].contiguous()
        send = torch.empty(T * C * (n1 - n0), dtype=torch.uint8, device="cuda")
        corr.corr_corner_turn_pack(x.data_ptr(), T, C, n1 - n0, chan_bounds, send.data_ptr(), stream)
        sends.append(send)
    for d, (c0, c1) in enumerate(ch):
        # what rank d receives: block d of every source's packed buffer, in source order
        parts = []
        for s, (n0, n1) in enumerate(ins):
            off = T * c0 * (n1 - n0)
            parts.append(sends[s][off:off + T * (c1 - c0) * (n1 - n0)])
        recv = torch.cat(parts)
        out = torch.empty((T, c1 - c0, N), dtype=torch.uint8, device="cuda")
        corr.corr_corner_turn_unpack(recv.data_ptr(), T, c1 - c0, N, input_bounds, out.data_ptr(), stream)
        assert torch.equal(out, full[:, c0:c1, :]), (d, c0, c1)
        if d == 0 and c1 > c0:
            with corr.Correlator(N, c1 - c0, T, npol) as xc:
                xc.accumulate(out)
                got_c = xc.dump(corr.CORR_WHAT_CROSS).cpu().numpy()
                got_a = xc.dump(corr.CORR_WHAT_AUTO).cpu().numpy()
                xc.sync()
            want_c, want_a = oracle.correlate(full_h[:, c0:c1, :], npol)
            assert np.array_equal(got_c, want_c) and np.array_equal(got_a, want_a)


def test_corner_turn_single_rank_is_the_identity(env):
    corr, replicas, synth, torch = env
    x = synth.generate_device(synth.Spec(kind="uniform", seed=3), 40, 5, 48)
    assert torch.equal(replicas.corner_turn(x, 48, 1, 0, 2), x)


def test_device_generator_channel_range(env):
    """The device generator's channel range gives the same bytes as those channels of the whole band."""
    corr, replicas, synth, torch = env
    spec = synth.Spec(kind="gauss_tone", seed=99)
    full = synth.generate_device(spec, 64, 12, 40)
    part = synth.generate_device(spec, 64, 12, 40, c_range=(5, 9))
    assert torch.equal(part, full[:, 5:9, :])
    assert np.array_equal(part.cpu().numpy(), synth.generate_host(spec, 64, 12, 40, c_range=(5, 9)))


def test_bounds_are_checked(env):
    corr, _, _, torch = env
    x = torch.zeros(64, dtype=torch.uint8, device="cuda")
    for bounds in ([0, 3], [1, 4], [0, 3, 2, 4], [0]):
        with pytest.raises(corr.CorrError):
            corr.corr_corner_turn_pack(x.data_ptr(), 2, 4, 8, bounds, x.data_ptr(), 0)
