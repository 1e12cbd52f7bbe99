"""Write the full-size expected values of the Monte-Carlo test and the
all-pairs screen, computed by the CPU oracle alone.

    python tests/golden/make_fullsize.py [--threads N] [--only mc|allpairs]

Outputs (plain text, next to this script):

  mc_100k_1m_10000.txt   the Monte-Carlo significance test of Sec. "Monte
                         Carlo Simulations" at Table 1's 1e5-interval,
                         1e4-round corner: 100,000
                         uniform intervals re-placed 10,000 times (seed 7)
                         against 1,000,000 clustered intervals on the
                         24-contig genome; the observed total, k_ge, the
                         p-value as an exact fraction, and all 10,000
                         per-shuffle totals.
  allpairs_64x32.txt     the all-pairs total matrix of the screen of Sec.
                         "Novel genomic relationships": M[i][j] =
                         total(A_i, B_j) for the 64
                         query sets and 32 databases (sizes log-uniform in
                         [1e3, 2e7], seed 11), all 2,048 entries.

Inputs come from the seeded generators in bits_synth (the same calls the
GPU tests make); every number comes from oracle/ (std::sort, then
std::lower_bound / std::upper_bound per query, and the oracle's own
Philox4x32-10 for the re-placements).  Nothing here touches the CUDA
library.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import bits_synth as synth  # noqa: E402
import oracle  # noqa: E402

MC_FILE = os.path.join(HERE, "mc_100k_1m_10000.txt")
AP_FILE = os.path.join(HERE, "allpairs_64x32.txt")
MC_SEED, MC_SHUFFLES = 7, 10_000


def write_mc(threads: int) -> None:
    o = oracle.get()
    genome, a, b = synth.config3()
    co, cl = synth.mc_contig_table(genome)
    bs, be = o.build(b)
    t0 = time.time()
    totals, obs, k, _ = o.mc(a, co, cl, bs, be, seed=MC_SEED, s_begin=0, s_end=MC_SHUFFLES,
                             threads=threads)
    dt = time.time() - t0
    with open(MC_FILE, "w") as f:
        f.write("# Monte-Carlo significance test (Sec. 'Monte Carlo Simulations'), Table 1's\n"
                "# 1e5 x 1e4 corner:\n"
                "# bits_synth.config3() -- 100,000 uniform query intervals (len U[100, 2000])\n"
                "# vs 1,000,000 clustered database intervals on the 24-contig genome --\n"
                f"# seed {MC_SEED}, shuffles [0, {MC_SHUFFLES}).  Written by\n"
                "# tests/golden/make_fullsize.py from the CPU oracle alone "
                f"({threads} threads, {dt:.0f} s).\n"
                "# OBSERVED <total of the unshuffled queries>\n"
                "# K_GE <#{s : T_s >= observed}>\n"
                "# P <k_ge + 1>/<N + 1>\n"
                "# then one line per shuffle s: <s> <T_s>\n")
        f.write(f"OBSERVED {obs}\nK_GE {k}\nP {k + 1}/{MC_SHUFFLES + 1}\n")
        for s, t in enumerate(totals):
            f.write(f"{s} {int(t)}\n")
    print(f"mc: observed {obs}, k_ge {k}, {dt:.0f} s -> {MC_FILE}")


def write_allpairs(threads: int) -> None:
    o = oracle.get()
    _, a_sets, b_sets = synth.config5()
    m = np.zeros((len(a_sets), len(b_sets)), np.uint64)
    t0 = time.time()
    for j, b in enumerate(b_sets):
        bs, be = o.build(b)
        for i, a in enumerate(a_sets):
            m[i, j] = o.count_sorted(a, bs, be, threads=threads, want_counts=False)[1]
        print(f"  database {j}: {b.shape[0]} intervals, {time.time() - t0:.0f} s", flush=True)
    dt = time.time() - t0
    with open(AP_FILE, "w") as f:
        f.write("# All-pairs total matrix of the screen (Sec. 'Novel genomic relationships'):\n"
                "# M[i][j] = total(A_i, B_j)\n"
                "# for bits_synth.config5() -- 64 query sets x 32 databases on the 24-contig\n"
                "# genome, sizes log-uniform in [1e3, 2e7] (seed 11), lengths U[50, 5000].\n"
                "# Written by tests/golden/make_fullsize.py from the CPU oracle alone "
                f"({threads} threads, {dt:.0f} s).\n"
                "# One line per query set i: <i> <M[i][0]> ... <M[i][31]>\n")
        for i in range(m.shape[0]):
            f.write(f"{i} " + " ".join(str(int(x)) for x in m[i]) + "\n")
    print(f"allpairs: {dt:.0f} s -> {AP_FILE}")


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--only", choices=["mc", "allpairs"])
    args = ap.parse_args()
    if args.only in (None, "mc"):
        write_mc(args.threads)
    if args.only in (None, "allpairs"):
        write_allpairs(args.threads)


if __name__ == "__main__":
    main()
