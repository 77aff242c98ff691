"""One process per GPU: channel shards, the corner turn, and the host-side collectives of the benchmark.

The X-engine has no exchange between channels (the paper gives each GPU its own 109 channels and
never combines GPUs in the X stage, Sec. 2.5): rank r owns a contiguous range of channels
(``channel_shards``) and no collective touches the X-engine's data path. The one exchange of the
paper's system is upstream of it, the corner turn (Sec. 2.3, Fig. 2): each F-engine holds every
channel of its own antennas, and each X-engine GPU needs every antenna of its own channels.
``corner_turn`` does it with one all-to-all between the ranks. The other collectives are the timing
barrier and the max-over-ranks of the timed region.
"""
from __future__ import annotations

import os


def channel_shards(n_chans: int, world: int):
    """Contiguous channel ranges [(c0, c1)] for `world` ranks, sizes differing by at most one."""
    if n_chans < 0 or world < 1:
        raise ValueError("need n_chans >= 0 and world >= 1")
    base, extra = divmod(n_chans, world)
    out, c0 = [], 0
    for r in range(world):
        c1 = c0 + base + (1 if r < extra else 0)
        out.append((c0, c1))
        c0 = c1
    return out


def input_shards(n_inputs: int, world: int, n_pol: int = 1):
    """Contiguous input ranges [(n0, n1)] for `world` F-engine ranks: whole stations of n_pol inputs,
    station counts differing by at most one."""
    if n_pol < 1 or n_inputs % n_pol:
        raise ValueError("n_inputs must be a multiple of n_pol")
    return [(a * n_pol, b * n_pol) for a, b in channel_shards(n_inputs // n_pol, world)]


def corner_turn(x_local, n_inputs: int, world: int, rank: int, n_pol: int = 1, group=None):
    """Turn per-antenna data into per-channel data across the ranks (Sec. 2.3).

    x_local: uint8 tensor [T][C][n_r] holding this rank's inputs ``input_shards(n_inputs, world,
    n_pol)[rank]`` for every channel (CPU or CUDA). Returns [T][C_r][n_inputs] holding every input of
    this rank's channels ``channel_shards(C, world)[rank]``. The exchange is one all_to_all_single.
    For CUDA tensors the local pack and unpack run in libcorr's corner-turn kernels on the current
    stream, which the collective is ordered with; for CPU tensors (the gloo path) they are plain
    tensor copies into the same layout.
    """
    import torch

    T, C, n_r = (int(v) for v in x_local.shape)
    ch = channel_shards(C, world)
    ins = input_shards(n_inputs, world, n_pol)
    if ins[rank][1] - ins[rank][0] != n_r:
        raise ValueError("x_local holds %d inputs; rank %d owns %s" % (n_r, rank, ins[rank]))
    chan_bounds = [c0 for c0, _ in ch] + [C]
    input_bounds = [n0 for n0, _ in ins] + [n_inputs]
    c0, c1 = ch[rank]
    C_r = c1 - c0
    send_splits = [T * (b - a) * n_r for a, b in ch]
    recv_splits = [T * C_r * (b - a) for a, b in ins]
    x_local = x_local.contiguous()
    if x_local.is_cuda:
        from . import corr

        sh = corr._stream_handle(None)
        send = torch.empty(T * C * n_r, dtype=torch.uint8, device=x_local.device)
        corr.corr_corner_turn_pack(x_local.data_ptr(), T, C, n_r, chan_bounds, send.data_ptr(), sh)
    else:
        send = torch.cat([x_local[:, a:b, :].reshape(-1) for a, b in ch])
    recv = torch.empty(sum(recv_splits), dtype=torch.uint8, device=x_local.device)
    if world > 1:
        import torch.distributed as dist

        dist.all_to_all_single(recv, send, recv_splits, send_splits, group=group)
    else:
        recv.copy_(send)
    if x_local.is_cuda:
        out = torch.empty((T, C_r, n_inputs), dtype=torch.uint8, device=x_local.device)
        corr.corr_corner_turn_unpack(recv.data_ptr(), T, C_r, n_inputs, input_bounds, out.data_ptr(), sh)
        return out
    parts = torch.split(recv, recv_splits)
    return torch.cat([p.view(T, C_r, b - a) for p, (a, b) in zip(parts, ins)], dim=2)


def init(backend: str = "nccl", timeout_s: float | None = None):
    """(world, rank, local_rank) from the torchrun environment; joins the process group if world > 1.

    timeout_s bounds every collective: a rank that died or never reaches the next barrier makes the
    others' barrier raise after at most that long instead of waiting indefinitely."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import datetime

        import torch
        import torch.distributed as dist

        if backend == "nccl":
            torch.cuda.set_device(local)
        if not dist.is_initialized():
            kw = {} if timeout_s is None else {"timeout": datetime.timedelta(seconds=timeout_s)}
            dist.init_process_group(backend, **kw)
    return world, rank, local


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """Largest value of x over the ranks (the timed region ends when the slowest rank ends)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def finalize(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
