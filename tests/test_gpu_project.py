"""Parity of the CUDA projection (Sec. "BITS Algorithm" (projection)) and
closed-interval mode (Sec. "Interval Set Intersection problem") with the CPU
oracle, bit for bit, plus end-to-end closed-interval counts.
"""
import numpy as np
import pytest
import torch

import bits_synth as synth
import oracle
from goldens import read_count_fixture, read_projection_fixture

pytestmark = pytest.mark.gpu

O = oracle.get()
GENOME = synth.make_genome()


def dev(x) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint32)).cuda()


@pytest.fixture(scope="module")
def bits():
    import paper_1208_3407_b300 as bits
    return bits


def gpu_project(bits, chrom, s, e, co=None, cl=None, closed=False, shift=0):
    """Runs bits_project; `shift` > 0 offsets every device array by that many
    words so the kernel takes its unaligned (scalar) path."""
    def place(x):
        t = torch.zeros(len(x) + shift, dtype=torch.uint32, device="cuda")
        t[shift:] = dev(x)
        return t[shift:]
    kw = {}
    if co is not None:
        kw = dict(contig=place(chrom), contig_off=dev(co), contig_len=dev(cl))
    out = None
    if shift:
        buf = torch.zeros((len(s) + 1, 2), dtype=torch.uint32, device="cuda")
        out = buf[1:]
    out, rej = bits.project(place(s), place(e), closed=closed, out=out, **kw)
    torch.cuda.synchronize()
    return out.cpu().numpy(), int(rej.cpu().numpy()[0])


@pytest.mark.parametrize("closed", [False, True])
def test_golden_fixture(bits, closed):
    co, cl, chrom, s, e, ho, cc = read_projection_fixture()
    out, bad = gpu_project(bits, chrom, s, e, co, cl, closed=closed)
    exp, nbad = O.project(chrom, s, e, co, cl, closed=closed)
    np.testing.assert_array_equal(out, exp)
    assert bad == nbad
    rows = cc if closed else ho
    assert bad == sum(r is None for r in rows)


@pytest.mark.parametrize("n", [0, 1, 3, 4, 5, 1027, 65_537, 1_000_003])
@pytest.mark.parametrize("closed", [False, True])
@pytest.mark.parametrize("shift", [0, 1])
def test_parity_random(bits, n, closed, shift):
    chrom, s, e = synth.local_intervals(GENOME, n, seed=100 + n, closed=closed, bad_frac=0.02)
    out, bad = gpu_project(bits, chrom, s, e, GENOME.offsets, GENOME.lengths, closed, shift)
    exp, nbad = O.project(chrom, s, e, GENOME.offsets, GENOME.lengths, closed=closed)
    np.testing.assert_array_equal(out, exp)
    assert bad == nbad


def test_no_contig_table_and_extremes(bits):
    top = 0xFFFFFFFF
    s = np.array([0, 0, 5, top, top - 1, 7], np.uint32)
    e = np.array([top, top, 4, top, top - 1, 7], np.uint32)
    for closed in (False, True):
        out, bad = gpu_project(bits, None, s, e, closed=closed)
        exp, nbad = O.project(None, s, e, closed=closed)
        np.testing.assert_array_equal(out, exp)
        assert bad == nbad
    # A chromosome ending exactly at 2^32 - 1.
    co, cl = np.array([top - 10], np.uint32), np.array([11], np.uint32)
    c = np.zeros(3, np.uint32)
    s, e = np.array([0, 0, 3], np.uint32), np.array([10, 11, 10], np.uint32)
    for closed in (False, True):
        out, bad = gpu_project(bits, c, s, e, co, cl, closed=closed)
        exp, nbad = O.project(c, s, e, co, cl, closed=closed)
        np.testing.assert_array_equal(out, exp)
        assert bad == nbad


def test_full_size_reads(bits):
    # 20,000,000 read-length intervals (the database size of the exome-vs-reads
    # workload), in chromosome-local closed coordinates.
    chrom, s, e = synth.local_intervals(GENOME, 20_000_000, seed=5, lo=100, hi=100, closed=True,
                                        bad_frac=1e-4)
    out, bad = gpu_project(bits, chrom, s, e, GENOME.offsets, GENOME.lengths, closed=True)
    exp, nbad = O.project(chrom, s, e, GENOME.offsets, GENOME.lengths, closed=True)
    assert bad == nbad and bad > 0
    np.testing.assert_array_equal(out, exp)


def test_closed_counts_end_to_end(bits):
    # Hand-counted closed fixture: project both sets, build, count on the GPU.
    a, b, exp, total = read_count_fixture("closed.txt")
    pa, _ = bits.project(dev(a[:, 0]), dev(a[:, 1]), closed=True)
    pb, _ = bits.project(dev(b[:, 0]), dev(b[:, 1]), closed=True)
    db = bits.Database(pb)
    c, t = db.count(pa)
    np.testing.assert_array_equal(c.cpu().numpy(), exp)
    assert int(t.cpu().numpy()[0]) == total
    db.free()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_closed_random_vs_brute_force(bits, seed):
    # Closed intervals on chromosomes, counted by the printed predicate per
    # chromosome (oracle brute force on each chromosome's own coordinates).
    genome = synth.make_genome(n_contigs=5, lo=300, hi=900, seed=seed)
    ca, sa, ea = synth.local_intervals(genome, 700, seed=10 + seed, lo=1, hi=30, closed=True)
    cb, sb, eb = synth.local_intervals(genome, 900, seed=20 + seed, lo=1, hi=30, closed=True)
    expect = np.zeros(ca.shape[0], np.uint32)
    for k in range(genome.n_contigs):
        ia, ib = np.flatnonzero(ca == k), np.flatnonzero(cb == k)
        if ia.size:
            c, _ = O.count_brute_closed(np.stack([sa[ia], ea[ia]], 1),
                                        np.stack([sb[ib], eb[ib]], 1).reshape(-1, 2))
            expect[ia] = c
    pa, ra = bits.project(dev(sa), dev(ea), contig=dev(ca), contig_off=dev(genome.offsets),
                          contig_len=dev(genome.lengths), closed=True)
    pb, rb = bits.project(dev(sb), dev(eb), contig=dev(cb), contig_off=dev(genome.offsets),
                          contig_len=dev(genome.lengths), closed=True)
    assert int(ra.cpu()[0]) == 0 and int(rb.cpu()[0]) == 0
    db = bits.Database(pb)
    c, t = db.count(pa)
    np.testing.assert_array_equal(c.cpu().numpy(), expect)
    assert int(t.cpu().numpy()[0]) == int(expect.sum())
    db.free()


def test_rejected_rows_fail_downstream(bits):
    chrom = np.array([0, 99], np.uint32)
    s = np.array([10, 10], np.uint32)
    e = np.array([20, 20], np.uint32)
    out, rej = bits.project(dev(s), dev(e), contig=dev(chrom), contig_off=dev(GENOME.offsets),
                            contig_len=dev(GENOME.lengths))
    assert int(rej.cpu()[0]) == 1
    with pytest.raises(bits.BitsError) as ei:
        bits.Database(out)
    assert ei.value.status == 1
    db = bits.Database(out[:1].contiguous())
    with pytest.raises(bits.BitsError) as ei:
        db.count(out)
    assert ei.value.status == 1
    db.free()


def test_argument_errors(bits):
    lib = bits._lib.load()
    assert lib.bits_project(None, None, None, 1 << 32, None, None, 0, 0, None, None, None) == 4
    assert lib.bits_project(None, None, None, 1, None, None, 0, 0, None, None, None) == 1
    assert lib.bits_project(None, None, None, 0, None, None, 0, 2, None, None, None) == 1
    assert lib.bits_project(None, None, None, 0, None, None, 0, 0, None, None, None) == 0
