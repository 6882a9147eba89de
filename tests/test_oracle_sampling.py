"""R16 random voxel sampling in the oracle (the Discussion's question: Mattes samples at random, MICUDA uses
every voxel).  The subset is fixed by a counter-based hash of the voxel index and a seed."""
import numpy as np

import oracle
from paper_1909_10690_gb300 import phantoms


def test_fmix32_is_a_bijection_with_full_avalanche():
    ks = np.arange(1 << 16, dtype=np.uint64)
    out = np.array([oracle.fmix32(int(k)) for k in ks], dtype=np.uint64)
    assert len(np.unique(out)) == len(ks)
    assert oracle.fmix32(0) == 0
    # flipping any one input bit changes about half of the 32 output bits (a dropped step or a wrong shift
    # leaves some bits barely mixed)
    rng = np.random.default_rng(1)
    xs = rng.integers(0, 1 << 32, 400, dtype=np.uint64)
    for bit in range(32):
        flips = [bin(oracle.fmix32(int(x)) ^ oracle.fmix32(int(x) ^ (1 << bit))).count("1") for x in xs]
        assert 14.5 < np.mean(flips) < 17.5, (bit, np.mean(flips))


def test_kept_fraction_and_seeds():
    n = 40000
    for frac in (0.1, 0.5, 0.9):
        thr = oracle.sample_threshold(frac)
        assert thr == int(np.floor(frac * 2 ** 32))
        kept = sum(oracle.sampled(x, 12345, thr) for x in range(n))
        assert abs(kept - frac * n) < 5 * np.sqrt(n * frac * (1 - frac))
    thr = oracle.sample_threshold(0.5)
    a = [oracle.sampled(x, 1, thr) for x in range(2000)]
    b = [oracle.sampled(x, 2, thr) for x in range(2000)]
    assert a != b and a == [oracle.sampled(x, 1, thr) for x in range(2000)]
    assert oracle.sample_threshold(0.0) == 0 and oracle.sample_threshold(1.0) == 0


def test_sampled_mi_is_the_mi_of_the_kept_voxels():
    f, m = phantoms.ellipsoid_pair(shape=(18, 20, 22), seed=15)
    m = np.maximum(m, 1).astype(np.uint8)  # no zero values: a resampled 0 marks a voxel outside the overlap
    bins = 16
    q16 = oracle.affine_q16(oracle.affine(phantoms.TINY_MOTION, f.shape, (1, 1, 1), m.shape, (1, 1, 1)))
    rs = oracle.resample(m, q16, f.shape, depth=8)
    fb = oracle.bin_volume(f, bins, 8).astype(np.int64).ravel()
    mb = oracle.bin_volume(rs, bins, 8).astype(np.int64).ravel()
    inside = rs.ravel() > 0
    for frac, seed in ((0.3, 7), (0.75, 99)):
        thr = oracle.sample_threshold(frac)
        keep = np.array([oracle.sampled(x, seed, thr) for x in range(f.size)])
        sel = inside & keep
        h = np.zeros((bins, bins), np.float64)
        np.add.at(h, (fb[sel], mb[sel]), 1.0)
        mi_b, h_b = oracle.entropies(h, [1.0, 1.5])
        mi, hh, cnt = oracle.mi_eval_q16(f, m, bins, q16[None], [1.0, 1.5], fixed_depth=8, moving_depth=8,
                                         sample_fraction=frac, sample_seed=seed)
        assert cnt[0] == sel.sum()
        np.testing.assert_allclose(mi[0], mi_b, rtol=0, atol=1e-12)
    # fraction 1 (or 0) is every voxel
    full = oracle.mi_eval_q16(f, m, bins, q16[None], [1.0], fixed_depth=8, moving_depth=8)
    one = oracle.mi_eval_q16(f, m, bins, q16[None], [1.0], fixed_depth=8, moving_depth=8, sample_fraction=1.0)
    np.testing.assert_array_equal(full[0], one[0])
    assert full[2][0] == inside.sum()
