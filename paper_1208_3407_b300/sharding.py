"""Host-side helpers for running BITS across ranks (one GPU per process).

Queries, shuffles and (set, database) pairs are independent (Sec. "Parallel BITS"
"pleasingly parallel"), so work shards with no exchange in the data path:
every rank keeps its own copy of the database and counts its own share.
The only exchanges are at the end of a call: totals add, and a sharded
Monte-Carlo test gathers the per-shuffle totals so that every rank can form
the same tally and p-value (Sec. "Monte Carlo Simulations") -- computed by the library's
bits_mc_summary kernel, never in Python.  The exchange helpers work with
any torch.distributed backend (gloo on CPU, nccl on GPUs).
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
    """All ranks' per-shuffle totals, in shuffle order (ranks hold consecutive
    ranges), as int64 words holding the uint64 totals' bits, on the group's
    device (the GPU for nccl, the host for gloo)."""
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
    return torch.cat([p[: hi - lo] for p, (lo, hi) in zip(parts, counts)])


def sharded_mc(db, a: torch.Tensor, contig_off: torch.Tensor, contig_len: torch.Tensor, *,
               seed: int, n_shuffles: int, method: int = 0, group=None) -> tuple[torch.Tensor, dict]:
    """One Monte-Carlo test (Sec. "Monte Carlo Simulations") split over the ranks of `group` by
    shuffle range: each rank runs bits_mc on its own range of
    [0, n_shuffles) against its own copy of the database, the ranges'
    totals are gathered in shuffle order, and bits_mc_summary forms the
    tally, p-values and Fig. 3 score of the whole run on the GPU.  Returns
    (all totals as a uint64 CUDA tensor, the summary as a dict).  Needs the
    nccl backend (the totals stay on the GPU)."""
    from . import mc_summary

    rank, world = dist.get_rank(group), dist.get_world_size(group)
    s0, s1 = shuffle_range(n_shuffles, rank, world)
    local, observed, _, _ = db.mc(a, contig_off, contig_len, seed=seed, shuffle_begin=s0,
                                  shuffle_end=s1, method=method)
    totals = gather_shuffle_totals(local, n_shuffles, group).view(torch.uint64)
    obs = torch.tensor([observed], dtype=torch.uint64, device=totals.device)
    stats = mc_summary(totals.view(1, -1), obs).to_dicts()[0]
    return totals, stats


def max_over_ranks(x: float, group=None) -> float:
    """Slowest rank's time (the benchmark's step time)."""
    t = torch.tensor([x], dtype=torch.float64, device=_device(group))
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def _device(group) -> torch.device:
    return torch.device("cuda", torch.cuda.current_device()) \
        if dist.get_backend(group) == "nccl" else torch.device("cpu")
