"""Readers for the hand-worked fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_count_fixture(name):
    """Returns (A uint32[n,2], B uint32[m,2], expected counts, expected total)."""
    a, b, exp, total = [], [], [], None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            if line[0] == "B":
                b.append((int(line[1]), int(line[2])))
            elif line[0] == "A":
                a.append((int(line[1]), int(line[2])))
                exp.append(int(line[3]))
            elif line[0] == "TOTAL":
                total = int(line[1])
    return (np.array(a, np.uint32).reshape(-1, 2), np.array(b, np.uint32).reshape(-1, 2),
            np.array(exp, np.uint32), total)


def read_philox_kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line:
                w = [int(x, 16) for x in line]
                rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def read_projection_fixture():
    """Returns (contig_off, contig_len, chrom, start, end, half_open, closed); the last two
    are lists of (start, end) or None for a rejected row."""
    table, rows = {}, []
    with open(os.path.join(GOLDEN, "projection.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            if line[0] == "C":
                table[int(line[1])] = (int(line[2]), int(line[3]))
            elif line[0] == "P":
                v = line[1:]
                ho = None if v[3] == "x" else (int(v[3]), int(v[4]))
                cl = None if v[5] == "x" else (int(v[5]), int(v[6]))
                rows.append((int(v[0]), int(v[1]), int(v[2]), ho, cl))
    ids = sorted(table)
    assert ids == list(range(len(ids)))
    co = np.array([table[i][0] for i in ids], np.uint32)
    cl_ = np.array([table[i][1] for i in ids], np.uint32)
    chrom = np.array([r[0] for r in rows], np.uint32)
    start = np.array([r[1] for r in rows], np.uint32)
    end = np.array([r[2] for r in rows], np.uint32)
    return co, cl_, chrom, start, end, [r[3] for r in rows], [r[4] for r in rows]


def read_mc_summary_fixture():
    """Rows of (observed, totals, expected dict) from mc_summary.txt."""
    from fractions import Fraction
    rows = []
    with open(os.path.join(GOLDEN, "mc_summary.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            head, tot, tail = [x.split() for x in line.split("|")]
            assert head[0] == "S"
            v = tail
            rows.append((int(head[1]), np.array([int(x) for x in tot], np.uint64), {
                "k_ge": int(v[0]), "k_le": int(v[1]), "median_lo": int(v[2]),
                "median_hi": int(v[3]), "p_enrich": Fraction(v[4]), "p_deplete": Fraction(v[5]),
                "score": v[6]}))
    return rows


def read_enumerate_fixture():
    """(A, B, expected counts, total, partner lists in scan order) from enumerate.txt."""
    a, b, exp, total = read_count_fixture("enumerate.txt")
    partners = {}
    with open(os.path.join(GOLDEN, "enumerate.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line and line[0] == "E":
                partners[int(line[1])] = [int(x) for x in line[2:]]
    return a, b, exp, total, [partners[i] for i in range(a.shape[0])]


def read_mc_fullsize():
    """Full-size Monte-Carlo expected values (make_fullsize.py): returns
    (observed, k_ge, (p numerator, p denominator), totals uint64[10000])."""
    obs = k = p = None
    totals = []
    with open(os.path.join(GOLDEN, "mc_100k_1m_10000.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            if line[0] == "OBSERVED":
                obs = int(line[1])
            elif line[0] == "K_GE":
                k = int(line[1])
            elif line[0] == "P":
                num, den = line[1].split("/")
                p = (int(num), int(den))
            else:
                assert int(line[0]) == len(totals)
                totals.append(int(line[1]))
    return obs, k, p, np.array(totals, np.uint64)


def read_allpairs_fullsize():
    """Full-size all-pairs expected matrix (make_fullsize.py): uint64[64, 32]."""
    rows = []
    with open(os.path.join(GOLDEN, "allpairs_64x32.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line:
                assert int(line[0]) == len(rows)
                rows.append([int(x) for x in line[1:]])
    return np.array(rows, np.uint64)
