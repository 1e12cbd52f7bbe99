"""The seeded workload generators follow the input recipe the benchmark and the
parity tests rely on (sizes, length laws, placement inside contigs, seeds).

CPU only; the large workloads are drawn at reduced sizes with the same laws.
"""
import numpy as np

import bits_synth as synth


def inside_one_contig(iv: np.ndarray, genome: synth.Genome) -> bool:
    """Every [start, end) lies inside a single contig of the genome."""
    s = iv[:, 0].astype(np.int64)
    e = iv[:, 1].astype(np.int64)
    offs = genome.offsets.astype(np.int64)
    c = np.searchsorted(offs, s, side="right") - 1
    return bool((c >= 0).all() and (e <= offs[c] + genome.lengths.astype(np.int64)[c]).all()
                and (e > s).all())


def test_genome():
    g = synth.make_genome()
    lens = g.lengths.astype(np.int64)
    assert g.n_contigs == 24
    assert (lens >= 50_000_000).all() and (lens <= 250_000_000).all()
    assert g.size == int(lens.sum()) == 3_170_234_504 < 2**32
    assert g.offsets[0] == 0
    np.testing.assert_array_equal(g.offsets[1:].astype(np.int64), np.cumsum(lens)[:-1])


def test_config1():
    a, b = synth.config1()
    for x in (a, b):
        assert x.shape == (10_000, 2) and x.dtype == np.uint32
        ln = x[:, 1].astype(np.int64) - x[:, 0]
        assert ln.min() >= 50 and ln.max() <= 500 and int(x[:, 1].max()) <= 1_000_000
    a2, b2 = synth.config1()
    assert np.array_equal(a, a2) and np.array_equal(b, b2)
    assert not np.array_equal(a, b)


def test_config2_shape_laws():
    g, a, b = synth.config2(n_a=50_000, n_b=200_000, n_hot=2_000)
    la = a[:, 1].astype(np.int64) - a[:, 0]
    assert la.min() >= 50 and la.max() <= 400 and abs(la.mean() - 150.0) < 1.0
    assert (b[:, 1].astype(np.int64) - b[:, 0] == 100).all()
    assert inside_one_contig(a, g) and inside_one_contig(b, g)
    # 70 % of the reads sit in hotspots: far fewer 10 kbp bins are occupied
    # than a uniform placement of as many reads would occupy.
    bins = g.size // 10_000
    occupied = np.unique(b[:, 0] // 10_000).shape[0]
    uniform = bins * (1.0 - np.exp(-b.shape[0] / bins))
    assert occupied < 0.6 * uniform
    _, a2, b2 = synth.config2(n_a=50_000, n_b=200_000, n_hot=2_000)
    assert np.array_equal(a, a2) and np.array_equal(b, b2)


def test_config3_shape_laws():
    g, a, b = synth.config3(n_a=20_000, n_b=100_000, n_hot=5_000)
    for x in (a, b):
        ln = x[:, 1].astype(np.int64) - x[:, 0]
        assert ln.min() >= 100 and ln.max() <= 2000
        assert inside_one_contig(x, g)


def test_config4_shape_laws():
    a, b = synth.config4(n_a=200_000, n_b=200_000)
    for x in (a, b):
        ln = x[:, 1].astype(np.int64) - x[:, 0]
        assert ln.min() >= 50 and ln.max() <= 10_000
        # log-uniform on [50, 1e4]: the median is the geometric mean, ~707
        assert abs(np.median(ln) / np.sqrt(50 * 10_000) - 1.0) < 0.05
        assert int(x[:, 1].max()) <= 3_000_000_000


def test_config5_sizes_and_sets():
    sa, sb = synth.config5_sizes()
    assert sa.shape == (64,) and sb.shape == (32,)
    for s in (sa, sb):
        assert s.min() >= 1_000 and s.max() <= 20_000_000
    assert int(sa.sum()) == 110_123_722
    g = synth.make_genome()
    for index in (2, 3):  # one clustered (even) and one uniform (odd) set
        x = synth.config5_set(index, 30_000, g)
        ln = x[:, 1].astype(np.int64) - x[:, 0]
        assert x.shape == (30_000, 2) and ln.min() >= 50 and ln.max() <= 5000
        assert inside_one_contig(x, g)
    assert np.array_equal(synth.config5_set(2, 1000, g), synth.config5_set(2, 1000, g))
    assert not np.array_equal(synth.config5_set(2, 1000, g), synth.config5_set(4, 1000, g))
