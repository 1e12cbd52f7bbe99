"""Host-side helpers for running BITS across ranks (one GPU per process).

Queries, shuffles and (set, database) pairs are independent (Sec. 2.4
"pleasingly parallel"), so work shards with no exchange in the data path:
every rank keeps its own copy of the database and counts its own share.
The only exchanges are at the end of a call: totals add, and a sharded
Monte-Carlo test gathers the per-shuffle totals so that every rank can form
the same tally and p-value (Sec. 3.2).  These helpers work with any
torch.distributed backend (gloo on CPU, nccl on GPUs).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard_bounds(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [lo, hi) slice of n units for `rank`; slices differ by at most one."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def shuffle_range(n_shuffles: int, rank: int, world: int, begin: int = 0) -> tuple[int, int]:
    """[shuffle_begin, shuffle_end) of this rank's share of a Monte-Carlo run."""
    lo, hi = shard_bounds(n_shuffles, rank, world)
    return begin + lo, begin + hi


def combine_totals(local_total: int, group=None) -> int:
    """Sum of every rank's uint64 total (exact: int64 lanes of a 2-word split)."""
    t = torch.tensor([local_total & 0xFFFFFFFF, local_total >> 32], dtype=torch.int64,
                     device=_device(group))
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return int(t[0].item()) + (int(t[1].item()) << 32)


def gather_shuffle_totals(local_totals: torch.Tensor, n_shuffles: int, group=None) -> torch.Tensor:
    """All ranks' per-shuffle totals, in shuffle order (ranks hold consecutive ranges)."""
    world = dist.get_world_size(group)
    dev = _device(group)
    counts = [shard_bounds(n_shuffles, r, world) for r in range(world)]
    width = max(hi - lo for lo, hi in counts)
    buf = torch.zeros(width, dtype=torch.int64, device=dev)
    loc = local_totals.to(dev).view(torch.int64) if local_totals.dtype == torch.uint64 else \
        local_totals.to(dev, torch.int64)
    buf[: loc.numel()] = loc
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return torch.cat([p[: hi - lo] for p, (lo, hi) in zip(parts, counts)]).cpu()


def tally(totals: torch.Tensor, observed: int) -> tuple[int, float]:
    """k_ge = #{s : T_s >= T_obs} and p = (k_ge + 1) / (N + 1) (one IEEE division)."""
    k = int((totals.to(torch.int64) >= observed).sum().item())
    return k, (k + 1) / (totals.numel() + 1)


def max_over_ranks(x: float, group=None) -> float:
    """Slowest rank's time (the benchmark's step time)."""
    t = torch.tensor([x], dtype=torch.float64, device=_device(group))
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def _device(group) -> torch.device:
    return torch.device("cuda", torch.cuda.current_device()) \
        if dist.get_backend(group) == "nccl" else torch.device("cpu")
