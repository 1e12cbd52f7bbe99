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
