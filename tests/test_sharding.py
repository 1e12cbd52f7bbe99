"""The multi-rank path on CPU: two gloo ranks share a count and a Monte-Carlo run.

Every rank counts its slice of the queries (and its range of shuffles) with
the oracle; the package's host-side helpers combine them.  The combined
total, the gathered per-shuffle totals and the tally of the gathered
totals must equal a single-process oracle run.  No GPU is used.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bits_synth as synth
    import oracle
    from paper_1208_3407_b300 import sharding

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    o = oracle.get()
    genome, a, b = synth.config3(n_a=3001, n_b=20_000, n_hot=500)
    co, cl = synth.mc_contig_table(genome)
    bs, be = o.build(b)
    lo, hi = sharding.shard_bounds(a.shape[0], rank, world)
    _, t_local = o.count_sorted(a[lo:hi], bs, be)
    total = sharding.combine_totals(t_local)
    s0, s1 = sharding.shuffle_range(97, rank, world, begin=5)
    local, obs, _, _ = o.mc(a, co, cl, bs, be, seed=9, s_begin=s0, s_end=s1)
    gathered = sharding.gather_shuffle_totals(torch.from_numpy(local.astype(np.int64)), 97)
    # The tally of the gathered totals (bits_mc_summary on a GPU; the
    # oracle's summary stands in for it on these CPU ranks).
    st = o.mc_summary(gathered.numpy().view(np.uint64), obs)
    slowest = sharding.max_over_ranks(float(rank + 1))
    out.put((rank, lo, hi, total, gathered.numpy().tolist(), st["k_ge"], st["p_enrich"], slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_match_single_process():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0

    import bits_synth as synth
    import oracle
    o = oracle.get()
    genome, a, b = synth.config3(n_a=3001, n_b=20_000, n_hot=500)
    co, cl = synth.mc_contig_table(genome)
    bs, be = o.build(b)
    _, full_total = o.count_sorted(a, bs, be)
    totals, obs, k, p = o.mc(a, co, cl, bs, be, seed=9, s_begin=5, s_end=102)
    (r0, lo0, hi0, *_), (r1, lo1, hi1, *_) = res
    assert (lo0, hi1) == (0, a.shape[0]) and hi0 == lo1          # slices tile the queries
    for _, _, _, total, gathered, kk, pp, slowest in res:
        assert total == full_total
        assert gathered == totals.astype(np.int64).tolist()
        assert (kk, pp) == (k, p)
        assert slowest == 2.0


@pytest.mark.parametrize("n,world", [(0, 3), (7, 3), (10, 4), (1_000_003, 8)])
def test_shard_bounds_tile(n, world):
    from paper_1208_3407_b300 import sharding
    bounds = [sharding.shard_bounds(n, r, world) for r in range(world)]
    assert bounds[0][0] == 0 and bounds[-1][1] == n
    assert all(bounds[i][1] == bounds[i + 1][0] for i in range(world - 1))
    sizes = [hi - lo for lo, hi in bounds]
    assert max(sizes) - min(sizes) <= 1
