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
