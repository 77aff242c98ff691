"""Multi-rank host logic on CPU (gloo, world size 2): channel shards, barrier and max-over-ranks.
Each rank correlates its own contiguous channel range with no data-path collective; the shards,
gathered here only for the check, reassemble into the single-process result."""
import os
import time
import socket

import numpy as np
import pytest

from paper_1411_3751_gb300 import replicas


def test_channel_shards_cover_contiguously():
    for C, W in ((2398, 22), (128, 1), (128, 8), (5, 8), (0, 3)):
        sh = replicas.channel_shards(C, W)
        assert len(sh) == W and sh[0][0] == 0 and sh[-1][1] == C
        assert all(a[1] == b[0] for a, b in zip(sh, sh[1:]))
        sizes = [c1 - c0 for c0, c1 in sh]
        assert max(sizes) - min(sizes) <= 1
    assert replicas.channel_shards(2398, 22)[0] == (0, 109)  # the paper's 109 channels per GPU
    with pytest.raises(ValueError):
        replicas.channel_shards(4, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    from oracle import oracle
    from paper_1411_3751_gb300 import synth

    w, r, _ = replicas.init("gloo")
    C, T, N = 11, 200, 12
    c0, c1 = replicas.channel_shards(C, w)[r]
    x = synth.generate_host(synth.Spec(kind="gauss_tone", seed=77), T, C, N, c_range=(c0, c1))
    cross, autos = oracle.correlate(x, 2)
    replicas.barrier(w)
    slowest = replicas.max_over_ranks(1.5 * (r + 1), w, "cpu")
    shards = [None] * w
    dist.all_gather_object(shards, (c0, c1, cross, autos))
    if r == 0:
        q.put((slowest, shards))
    replicas.finalize(w)


def test_two_ranks_gloo_shards_and_timing():
    import torch.multiprocessing as mp

    from oracle import oracle
    from paper_1411_3751_gb300 import synth

    oracle.build()
    synth._lib_host()  # build the host generator once, before the ranks start
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    mp.start_processes(_worker, args=(2, _free_port(), q), nprocs=2, join=True, start_method="spawn")
    slowest, shards = q.get(timeout=60)
    assert slowest == 3.0
    full = synth.generate_host(synth.Spec(kind="gauss_tone", seed=77), 200, 11, 12)
    want_c, want_a = oracle.correlate(full, 2)
    got_c = np.concatenate([s[2] for s in shards])
    got_a = np.concatenate([s[3] for s in shards])
    assert [s[:2] for s in shards] == [(0, 6), (6, 11)]
    assert np.array_equal(got_c, want_c) and np.array_equal(got_a, want_a)


def _dying_worker(r, w, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(r), WORLD_SIZE=str(w),
                      LOCAL_RANK=str(r))
    from paper_1411_3751_gb300 import replicas

    replicas.init("gloo", timeout_s=10)
    if r == 1:
        os._exit(3)  # leaves between steps: no collective of its own in flight
    t0 = time.monotonic()
    try:
        replicas.barrier(w)
        q.put(("not detected", time.monotonic() - t0))
    except Exception as e:  # the backend's error for a lost peer or a timed-out collective
        q.put(("detected", time.monotonic() - t0))


def test_a_dead_replica_is_detected_at_the_next_barrier():
    """Two gloo ranks on CPU; rank 1 exits after joining. Rank 0's next barrier must raise (lost peer
    or the 10 s collective timeout) instead of waiting forever."""
    import multiprocessing as mpl

    ctx = mpl.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dying_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        status, waited = q.get(timeout=120)
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    assert status == "detected" and waited < 60, (status, waited)
    assert procs[1].exitcode == 3


def test_input_shards_are_whole_stations():
    assert replicas.input_shards(512, 22, 2)[0] == (0, 24)
    for N, W, P in ((512, 2, 2), (512, 3, 2), (12, 5, 2), (7, 3, 1), (4, 8, 2)):
        sh = replicas.input_shards(N, W, P)
        assert len(sh) == W and sh[0][0] == 0 and sh[-1][1] == N
        assert all(a[1] == b[0] for a, b in zip(sh, sh[1:])) and all((b - a) % P == 0 for a, b in sh)
    with pytest.raises(ValueError):
        replicas.input_shards(7, 2, 2)


def _turn_worker(rank, world, port, q, N, C, T, npol):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist

    from oracle import oracle
    from paper_1411_3751_gb300 import synth

    w, r, _ = replicas.init("gloo", timeout_s=60)
    # this rank's F-engine output: every channel of its own inputs
    n0, n1 = replicas.input_shards(N, w, npol)[r]
    full = synth.generate_host(synth.Spec(kind="gauss_tone", seed=1411), T, C, N)
    x_local = torch.from_numpy(np.ascontiguousarray(full[:, :, n0:n1]))
    shard = replicas.corner_turn(x_local, N, w, r, npol).numpy()
    c0, c1 = replicas.channel_shards(C, w)[r]
    cross, autos = oracle.correlate(shard, npol)
    got = [None] * w
    dist.all_gather_object(got, (c0, c1, shard, cross, autos))
    if r == 0:
        q.put(got)
    replicas.finalize(w)


@pytest.mark.parametrize("world,N,C,T,npol", [(2, 12, 11, 64, 2), (3, 10, 7, 40, 2), (3, 9, 5, 33, 1)])
def test_corner_turn_then_correlate_reassembles_the_band(world, N, C, T, npol):
    """gloo ranks on CPU, each holding every channel of its own inputs (an F-engine's output, Sec. 2.3):
    after the all-to-all corner turn each holds every input of its own channels, correlates them with
    the oracle, and the shards reassemble bit-exactly into the single-process result; uneven input and
    channel shards included."""
    import torch.multiprocessing as mp

    from oracle import oracle
    from paper_1411_3751_gb300 import synth

    oracle.build()
    synth._lib_host()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    mp.start_processes(_turn_worker, args=(world, _free_port(), q, N, C, T, npol), nprocs=world, join=True,
                       start_method="spawn")
    got = q.get(timeout=60)
    full = synth.generate_host(synth.Spec(kind="gauss_tone", seed=1411), T, C, N)
    want_c, want_a = oracle.correlate(full, npol)
    assert [g[:2] for g in got] == replicas.channel_shards(C, world)
    for c0, c1, shard, _, _ in got:
        assert np.array_equal(shard, full[:, c0:c1, :])
    assert np.array_equal(np.concatenate([g[3] for g in got]), want_c)
    assert np.array_equal(np.concatenate([g[4] for g in got]), want_a)
