"""One process per GPU: channel shards and the few host-side collectives the benchmark needs.

The X-engine has no exchange between channels (the paper gives each GPU its own 109 channels and
never combines GPUs in the X stage, Sec. 2.5), so several GPUs run independent replicas: rank r
owns a contiguous range of channels (``channel_shards``) and no collective touches the data path.
The only collectives are the timing barrier and the max-over-ranks of the timed region.
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
