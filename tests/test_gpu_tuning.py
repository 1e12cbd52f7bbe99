"""Every launch configuration the autotuner can choose gives the oracle's
results, bit for bit, and the autotuner records and reuses its choices.

The tuned parameters (include/bits.h, bits_tuning) only change how work is
laid out: the shared-memory top of the plain search (the database's default
top level or one or two levels above it), the threads per CTA of the count
kernels, the Monte-Carlo work-unit shape, and the all-pairs chunk.  Each is
pinned here in turn with bits_set_tuning and the results compared with the
CPU oracle on the same seeded inputs.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import bits_synth as synth
import oracle

pytestmark = pytest.mark.gpu

O = oracle.get()
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MC_SHAPES = [(256, 1024), (128, 1024), (256, 512), (256, 2048), (128, 2048)]


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint32)).cuda()


@pytest.fixture(scope="module")
def bits():
    import paper_1208_3407_b300 as bits
    yield bits
    bits.set_tuning()


@pytest.fixture(scope="module")
def count_case():
    genome, a, b = synth.config2(n_a=70_001, n_b=2_000_003, n_hot=20_000, seed_a=51, seed_b=52)
    bs, be = O.build(b)
    oc, ot = O.count_sorted(a, bs, be, threads=8)
    return a, b, oc, ot


@pytest.mark.parametrize("raise_", [0, 1, 2])
@pytest.mark.parametrize("block", [256, 512])
def test_count_every_top_and_block(bits, count_case, raise_, block):
    a, b, oc, ot = count_case
    db = bits.Database(dev(b), rmi_leaves_log2=14)
    try:
        with bits.tuning(top_raise=raise_, block=block):
            for m in (bits.METHOD_SEARCH, bits.METHOD_RMI):
                c, t = db.count(dev(a), method=m)
                np.testing.assert_array_equal(c.cpu().numpy(), oc)
                assert int(t.cpu().numpy()[0]) == ot
            h, ht = db.count_host(a, method=bits.METHOD_SEARCH)
            np.testing.assert_array_equal(h.numpy(), oc)
            assert ht == ot
    finally:
        db.free()


def test_raise_is_clamped_on_small_databases(bits):
    a, b = synth.config1(n_a=500, n_b=40)        # one level: no smaller top exists
    oc, ot = O.count_brute(a, b)
    db = bits.Database(dev(b))
    with bits.tuning(top_raise=2, block=256):
        c, t = db.count(dev(a), method=bits.METHOD_SEARCH)
    db.free()
    np.testing.assert_array_equal(c.cpu().numpy(), oc)
    assert int(t.cpu().numpy()[0]) == ot


@pytest.mark.parametrize("shape", MC_SHAPES)
@pytest.mark.parametrize("raise_", [0, 1])
def test_mc_every_shape_and_top(bits, shape, raise_):
    genome, a, b = synth.config3(n_a=3001, n_b=60_000, n_hot=3000, seed_a=53, seed_b=54)
    co, cl = synth.mc_contig_table(genome)
    bs, be = O.build(b)
    ot, oobs, ok, op = O.mc(a, co, cl, bs, be, seed=11, s_begin=3, s_end=303, threads=8)
    db = bits.Database(dev(b), rmi_leaves_log2=12)
    try:
        with bits.tuning(top_raise=raise_, mc_shuffles=shape[0], mc_chunk=shape[1]):
            for m in (bits.METHOD_SEARCH, bits.METHOD_RMI):
                t, obs, k, p = db.mc(dev(a), dev(co), dev(cl), seed=11, shuffle_begin=3,
                                     shuffle_end=303, method=m)
                np.testing.assert_array_equal(t.cpu().numpy(), ot)
                assert (obs, k, p) == (oobs, ok, op)
    finally:
        db.free()


@pytest.mark.parametrize("chunk", [4096, 8192, 16384, 32768])
def test_allpairs_every_chunk(bits, chunk):
    genome, a_sets, b_sets = synth.config5(n_sets_a=6, n_sets_b=5, hi=150_000, seed=55)
    expected = np.zeros((6, 5), np.uint64)
    for j, b in enumerate(b_sets):
        bs, be = O.build(b)
        for i, a in enumerate(a_sets):
            expected[i, j] = O.count_sorted(a, bs, be, want_counts=False)[1]
    dbs = [bits.Database(dev(b), rmi_leaves_log2=10 if j % 2 else 0) for j, b in enumerate(b_sets)]
    try:
        with bits.tuning(ap_chunk=chunk):
            m = bits.count_matrix(dbs, [dev(a) for a in a_sets])
        np.testing.assert_array_equal(m.cpu().numpy(), expected)
    finally:
        for d in dbs:
            d.free()


def test_bad_tuning_is_rejected(bits):
    for kw in ({"top_raise": 3}, {"block": 300}, {"mc_shuffles": 128, "mc_chunk": 512},
               {"ap_chunk": 1000}):
        with pytest.raises(bits.BitsError):
            bits.set_tuning(**kw)
    assert bits.get_tuning() == {"top_raise": -1, "block": 0, "mc_shuffles": 0, "mc_chunk": 0,
                                 "ap_chunk": 0}


_CHILD = r"""
import json, sys
sys.path.insert(0, {root!r})
import numpy as np, torch
import bits_synth as synth, oracle
import paper_1208_3407_b300 as bits
O = oracle.get()
d = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint32)).cuda()
out = {{}}
genome, a, b = synth.config2(n_a=40_000, n_b=1_000_000, n_hot=10_000, seed_a=61, seed_b=62)
db = bits.Database(d(b), rmi_leaves_log2=12)
c, t = db.count(d(a))                                   # AUTO: tuned here
bs, be = O.build(b)
oc, ot = O.count_sorted(a, bs, be, threads=8)
out["count"] = bool(np.array_equal(c.cpu().numpy(), oc) and int(t.cpu().numpy()[0]) == ot)
g3, a3, b3 = synth.config3(n_a=2000, n_b=40_000, n_hot=2000, seed_a=63, seed_b=64)
co, cl = synth.mc_contig_table(g3)
db3 = bits.Database(d(b3))
tt, obs, k, p = db3.mc(d(a3), d(co), d(cl), seed=5, shuffle_end=700, method=bits.METHOD_SEARCH)
bs3, be3 = O.build(b3)
ref = O.mc(a3, co, cl, bs3, be3, seed=5, s_begin=0, s_end=700, threads=8)
out["mc"] = bool(np.array_equal(tt.cpu().numpy(), ref[0]) and (obs, k, p) == ref[1:])
_, a_sets, b_sets = synth.config5(n_sets_a=4, n_sets_b=3, hi=60_000, seed=65)
dbs = [bits.Database(d(x)) for x in b_sets]
m = bits.count_matrix(dbs, [d(x) for x in a_sets]).cpu().numpy()
exp = np.array([[O.count(x, y)[1] for y in b_sets] for x in a_sets], np.uint64)
out["allpairs"] = bool(np.array_equal(m, exp))
print(json.dumps(out))
"""


def test_autotuner_records_and_reuses_choices(tmp_path):
    cache = tmp_path / "tune.txt"
    env = dict(os.environ, BITS_AUTOTUNE_CACHE=str(cache))
    code = _CHILD.format(root=ROOT)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res == {"count": True, "mc": True, "allpairs": True}
    lines = cache.read_text().splitlines()
    kinds = {ln.split()[1] for ln in lines}
    assert {"count", "mc", "allpairs"} <= kinds
    for ln in lines:
        f = ln.split()
        vals = [int(x) for x in f[5:]]
        if f[1] == "count":
            assert vals[0] in (1, 2, 3) and 0 <= vals[1] <= 2 and vals[2] in (256, 512)
        elif f[1] == "mc":
            assert tuple(vals[:2]) in MC_SHAPES and vals[2] in (0, 1)
        else:
            assert vals[0] in (4096, 8192, 16384, 32768)
    # A second process reads the records and times nothing new.
    r2 = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                        timeout=600)
    assert r2.returncode == 0, r2.stderr[-3000:]
    assert json.loads(r2.stdout.strip().splitlines()[-1]) == res
    assert cache.read_text().splitlines() == lines
