"""Run one named workload a few times, for profiling the library's kernels.

    python workloads.py <name> [--method search|rmi|mergepath] [--reps N]

Workloads (inputs from the seeded generator ``bits_synth``):
    count-200k-20m   bits_count, 200,000 queries vs 20,000,000 reads (exome-vs-reads)
    count-100m-100m  bits_count, 100M queries vs 100M intervals (learned index built)
    count-10m-100m   the first 10M of those queries vs the same 100M intervals (a
                     reduced case for multi-pass ncu captures; DRAM bytes per
                     query scale with the queries)
    build-20m        bits_build_db of the 20,000,000 reads
    enumerate-200k-20m  every intersecting pair of those queries and reads
    mc-100k-1m       bits_mc, 100,000 intervals vs 1,000,000, 10,000 shuffles
    allpairs-64x32   bits_count_matrix, 64 query sets x 32 databases
    allpairs-16x8    the same on the first 16 query sets and 8 databases
    allpairs-db-64x32, allpairs-db-16x8
                     bits_count_matrix_db on those sets with the query sets
                     built as databases too
    mc-screen-64x32  bits_mc_matrix over those sets, 4 shuffles, with the summary
    mc-screen-16x8   the same on the first 16 query sets and 8 databases
                     (--shuffles N: shuffles per call, default 4)

Every call checks the device error word at the end; the script prints one
line per workload with the device time of the last repetition.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import bits_synth  # noqa: E402

from paper_1208_3407_b300 import (METHOD_MERGEPATH, METHOD_RMI, METHOD_SEARCH,  # noqa: E402
                                  Database, count_matrix, count_matrix_db, mc_matrix, set_tuning)

METHODS = {"search": METHOD_SEARCH, "rmi": METHOD_RMI, "mergepath": METHOD_MERGEPATH}


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint32)).cuda()


def _timed(fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("name")
    ap.add_argument("--method", default="search", choices=sorted(METHODS))
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--shuffles", type=int, default=4, help="shuffles per Monte-Carlo screen call")
    ap.add_argument("--top-raise", type=int, default=0,
                    help="pinned shared-memory top (no autotuning runs inside a profile)")
    ap.add_argument("--block", type=int, default=512)
    args = ap.parse_args(argv)
    # Profiles capture the kernels of one configuration: pin the launch
    # parameters so that the autotuner times no candidates here.
    set_tuning(top_raise=args.top_raise, block=args.block, mc_shuffles=256, mc_chunk=1024,
               ap_chunk=8192)
    m = METHODS[args.method]
    ms = 0.0
    if args.name in ("count-200k-20m", "count-100m-100m", "count-10m-100m"):
        if args.name == "count-200k-20m":
            _, a_np, b_np = bits_synth.config2()
        else:
            a_np, b_np = bits_synth.config4()
            if args.name == "count-10m-100m":
                a_np = a_np[:10_000_000]
        db = Database(_dev(b_np), rmi_leaves_log2=16)
        a = _dev(a_np)
        counts = torch.empty(a_np.shape[0], dtype=torch.uint32, device="cuda")
        total = torch.empty(1, dtype=torch.uint64, device="cuda")
        for _ in range(args.reps):
            ms = _timed(lambda: db.count(a, counts=counts, total=total, method=m, check=False))
        db.check()
    elif args.name == "enumerate-200k-20m":
        _, a_np, b_np = bits_synth.config2()
        db = Database(_dev(b_np), enumerate=True)
        a = _dev(a_np)
        for _ in range(args.reps):
            ms = _timed(lambda: db.enumerate(a, check=False))
        db.check()
    elif args.name == "build-20m":
        _, _, b_np = bits_synth.config2()
        b = _dev(b_np)
        for _ in range(args.reps):
            holder = []
            ms = _timed(lambda: holder.append(Database(b)))
            holder[0].free()
    elif args.name == "mc-100k-1m":
        genome, a_np, b_np = bits_synth.config3()
        co, cl = bits_synth.mc_contig_table(genome)
        db = Database(_dev(b_np), rmi_leaves_log2=16)
        a, dco, dcl = _dev(a_np), _dev(co), _dev(cl)
        totals = torch.empty(10_000, dtype=torch.uint64, device="cuda")
        for _ in range(args.reps):
            ms = _timed(lambda: db.mc(a, dco, dcl, seed=7, shuffle_end=10_000, totals=totals,
                                      method=m))
    elif args.name in ("allpairs-64x32", "allpairs-16x8"):
        _, a_sets, b_sets = bits_synth.config5()
        if args.name == "allpairs-16x8":
            a_sets, b_sets = a_sets[:16], b_sets[:8]
        dbs = [Database(_dev(b), rmi_leaves_log2=16) for b in b_sets]
        a = [_dev(x) for x in a_sets]
        out = torch.empty((len(a), len(dbs)), dtype=torch.uint64, device="cuda")
        for _ in range(args.reps):
            ms = _timed(lambda: count_matrix(dbs, a, out=out))
        for d in dbs:
            d.check()
    elif args.name in ("allpairs-db-64x32", "allpairs-db-16x8"):
        _, a_sets, b_sets = bits_synth.config5()
        if args.name == "allpairs-db-16x8":
            a_sets, b_sets = a_sets[:16], b_sets[:8]
        a_dbs = [Database(_dev(a)) for a in a_sets]
        b_dbs = [Database(_dev(b)) for b in b_sets]
        out = torch.empty((len(a_dbs), len(b_dbs)), dtype=torch.uint64, device="cuda")
        for _ in range(args.reps):
            ms = _timed(lambda: count_matrix_db(a_dbs, b_dbs, out=out))
        for d in a_dbs + b_dbs:
            d.check()
    elif args.name in ("mc-screen-64x32", "mc-screen-16x8"):
        genome, a_sets, b_sets = bits_synth.config5()
        if args.name == "mc-screen-16x8":
            a_sets, b_sets = a_sets[:16], b_sets[:8]
        co, cl = bits_synth.mc_contig_table(genome)
        dbs = [Database(_dev(b)) for b in b_sets]
        a = [_dev(x) for x in a_sets]
        dco, dcl = _dev(co), _dev(cl)
        ns = args.shuffles
        out = (torch.empty((len(a), len(dbs)), dtype=torch.uint64, device="cuda"),
               torch.empty((len(a), len(dbs), ns), dtype=torch.uint64, device="cuda"),
               torch.empty((len(a), len(dbs), 8), dtype=torch.uint64, device="cuda"))
        for _ in range(args.reps):
            ms = _timed(lambda: mc_matrix(dbs, a, dco, dcl, seed=17, shuffle_end=ns, out=out))
        for d in dbs:
            d.check()
    else:
        ap.error(f"unknown workload {args.name}")
    print(f"{args.name} method={args.method} last_ms={ms:.4f}")


if __name__ == "__main__":
    main()
