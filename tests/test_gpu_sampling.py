"""GPU parity of random voxel sampling (R16: the fixed voxels whose hashed index falls below
floor(fraction 2^32)), every histogram variant, plain and batched paths."""
import numpy as np
import pytest

import oracle
from paper_1909_10690_gb300 import phantoms

pytestmark = pytest.mark.gpu

VARIANTS = list(range(16))


@pytest.mark.parametrize("variant", VARIANTS)
def test_sampled_histograms_bit_exact(cuda_lib, variant):
    f, m = phantoms.head_pair(shape=(29, 41, 75), spacing=(1, 1, 1), seed=80)
    m = np.ascontiguousarray(m[:, :37, :71])
    bins, frac, seed = 64, 0.3, 1234
    ctx = cuda_lib.Context(f, m, bins=bins, fixed_depth=12, moving_depth=12, hist_variant=variant,
                           sample_fraction=frac, sample_seed=seed)
    prm = phantoms.random_transforms(12, seed=81, t_mm=4, r_deg=10, s_range=(0.9, 1.1))
    q16 = np.stack([oracle.affine_q16(oracle.affine(p, f.shape, (1, 1, 1), m.shape, (1, 1, 1))) for p in prm])
    for path in (cuda_lib.PATH_PLAIN, cuda_lib.PATH_BATCHED):
        H = ctx.hist(affines=q16, path=path)
        for t in range(0, len(q16), 4):
            ho, n = oracle.joint_hist(f, m, q16[t], bins, 12, 12, sample_fraction=frac, sample_seed=seed)
            np.testing.assert_array_equal(H[t], ho.astype(np.uint32))


def test_sampled_mi_counts_and_seeds(cuda_lib):
    f, m = phantoms.head_pair(shape=(48, 56, 60), spacing=(1, 1, 1), seed=82)
    prm = phantoms.random_transforms(20, seed=83, t_mm=5, r_deg=10, s_range=(0.9, 1.1))
    q16 = np.stack([oracle.affine_q16(oracle.affine(p, f.shape, (1, 1, 1), m.shape, (1, 1, 1))) for p in prm])
    qs = [1.0, 0.5, 2.0]
    counts = {}
    for frac, seed in ((0.1, 1), (0.5, 1), (0.5, 2)):
        ctx = cuda_lib.Context(f, m, bins=128, fixed_depth=12, moving_depth=12, sample_fraction=frac, sample_seed=seed)
        mi, h, cnt = ctx.eval(prm, qs, with_entropies=True)
        mi_o, h_o, cnt_o = oracle.mi_eval_q16(f, m, 128, q16, qs, fixed_depth=12, moving_depth=12, nthreads=8,
                                              sample_fraction=frac, sample_seed=seed)
        np.testing.assert_array_equal(cnt, cnt_o)
        scale = np.maximum(np.abs(mi_o), h_o[..., 2])
        assert np.all(np.abs(mi - mi_o) <= 1e-6 * scale)
        counts[(frac, seed)] = cnt
    full = cuda_lib.Context(f, m, bins=128, fixed_depth=12, moving_depth=12).eval(prm, qs, with_entropies=True)[2]
    for (frac, seed), c in counts.items():
        assert np.all(np.abs(c / full - frac) < 0.05)  # about that fraction of the overlap
    assert not np.array_equal(counts[(0.5, 1)], counts[(0.5, 2)])


def test_sampled_parzen_mi_and_gradient(cuda_lib):
    # the Mattes-like combination: a Parzen soft histogram over a random voxel subset; the oracle's
    # voxel set is the mask (sampled and inside the overlap)
    f, m = phantoms.head_pair(shape=(30, 34, 38), spacing=(1, 1, 1), seed=87, dtype=np.float32)
    B, frac, seed, qs = 32, 0.35, 21, [1.0, 1.3]
    ctx = cuda_lib.Context(f, m, bins=B, kernel="parzen", sample_fraction=frac, sample_seed=seed)
    thr = oracle.sample_threshold(frac)
    keep = np.array([oracle.sampled(x, seed, thr) for x in range(f.size)], np.uint8).reshape(f.shape)
    prm = phantoms.random_transforms(3, seed=88, t_mm=4, r_deg=8, s_range=(0.95, 1.05))
    mi, g = ctx.grad(prm, qs)
    for t in range(len(prm)):
        aff, J = oracle.affine(prm[t], f.shape, (1, 1, 1), m.shape, (1, 1, 1), with_jacobian=True)
        mask = keep & oracle.overlap_mask(f.shape, m.shape, aff)
        mi_o, g_o, n = oracle.parzen(f, m, aff, B, qs, daff=J, mask=mask)
        assert n == int(mask.sum()) and 0.25 * f.size < n < 0.45 * f.size
        assert np.all(np.abs(mi[t] - mi_o) <= 1e-6 * np.maximum(np.abs(mi_o), 1.0)), (t, mi[t], mi_o)
        for iq in range(len(qs)):
            assert np.abs(g[t, iq] - g_o[iq]).max() <= 1e-4 * np.abs(g_o[iq]).max(), (t, iq)
    with pytest.raises(cuda_lib.MIError):
        cuda_lib.Context(f, m, bins=16, sample_fraction=1.5)


def test_sampled_empty_overlap_and_uneven_pairs(cuda_lib):
    # a transform with no overlap gives NaN and MI_EEMPTY after the rest of the batch is done
    f, m = phantoms.head_pair(shape=(24, 26, 28), spacing=(1, 1, 1), seed=85)
    ctx = cuda_lib.Context(f, m, bins=32, fixed_depth=12, moving_depth=12, sample_fraction=0.4, sample_seed=9)
    prm = phantoms.random_transforms(3, seed=86, t_mm=2, r_deg=3, s_range=(0.98, 1.02))
    prm[1, :3] = 500.0
    with pytest.raises(cuda_lib.MIError) as e:
        ctx.eval(prm, [1.0], allow_empty=False)
    assert e.value.status == cuda_lib.MI_EEMPTY
    mi = ctx.eval(prm, [1.0])
    assert np.isnan(mi[1, 0]) and np.all(np.isfinite(mi[[0, 2], 0]))
    # each pair of an uneven batch has its own sampled subset
    specs = [((20, 22, 24), np.uint8, 8, 32), ((26, 18, 30), np.uint16, 12, 64)]
    pairs, vols = [], []
    for i, (shape, dt, depth, bins) in enumerate(specs):
        fi, mi_ = phantoms.head_pair(shape=shape, spacing=(1, 1, 1), depth=depth, seed=90 + i, dtype=dt)
        vols.append((fi, mi_, depth, bins))
        pairs.append(dict(fixed=fi, moving=mi_, bins=bins, fixed_depth=depth, moving_depth=depth))
    bctx = cuda_lib.Context(pairs=pairs, sample_fraction=0.6, sample_seed=17)
    prm = phantoms.random_transforms(8, seed=92, t_mm=3, r_deg=6, s_range=(0.95, 1.05))
    pair_of = np.array([0, 1] * 4, np.int32)
    got, h, cnt = bctx.batch_eval(pair_of, prm, [1.0, 2.0], with_entropies=True)
    for p, (fi, mi_, depth, bins) in enumerate(vols):
        sel = np.nonzero(pair_of == p)[0]
        q16 = np.stack([oracle.affine_q16(oracle.affine(prm[t], fi.shape, (1, 1, 1), mi_.shape, (1, 1, 1))) for t in sel])
        mo, ho, co = oracle.mi_eval_q16(fi, mi_, bins, q16, [1.0, 2.0], fixed_depth=depth, moving_depth=depth,
                                        sample_fraction=0.6, sample_seed=17)
        np.testing.assert_array_equal(cnt[sel], co)
        assert np.all(np.abs(got[sel] - mo) <= 1e-6 * np.maximum(np.abs(mo), ho[..., 2]))
