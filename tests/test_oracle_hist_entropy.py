"""Pins of the oracle's fixed-point resampling (R3/R4), joint histogram (R5)
and entropies (Eq. 1, Eq. 2, Tsallis R7).

Expectations come from hand enumeration (tests/golden), exact permutations,
numpy slicing, library routines (scipy.stats.entropy) and theorems
(pseudo-additivity of Tsallis entropy, Miller-Madow bias).
"""
import math

import numpy as np
import pytest

import hand_cases
import oracle
from paper_1909_10690_gb300 import phantoms

IDENT = np.array([65536, 0, 0, 0, 0, 65536, 0, 0, 0, 0, 65536, 0], dtype=np.int32)
VOLUMES, CASES = hand_cases.load()


@pytest.mark.parametrize("case", CASES, ids=lambda c: c["name"])
def test_hand_enumerated_4x4x4(case):
    fx, mv = hand_cases.volume(VOLUMES[case["fixed"]]), hand_cases.volume(VOLUMES[case["moving"]])
    h, n = oracle.joint_hist(fx, mv, case["q16"], hand_cases.bins_of(case))
    np.testing.assert_array_equal(h, hand_cases.expected_hist(case))
    assert n == case["N"]
    for q, v in case["mi"].items():
        mi, _ = oracle.entropies(h, [float(q)])
        assert abs(mi[0] - v) < 1e-12
    for q, v in case.get("mi_pseudo_additive", {}).items():
        mi, _ = oracle.entropies(h, [float(q)], form=1)
        assert abs(mi[0] - v) < 1e-12


def test_identity_gives_diagonal_and_mi_equals_h():
    fx, _ = phantoms.ellipsoid_pair(shape=(24, 20, 18), seed=7)
    for bins in (8, 32, 256):
        h, n = oracle.joint_hist(fx, fx, IDENT, bins)
        assert n == fx.size
        assert np.count_nonzero(h - np.diag(np.diag(h))) == 0
        mi, hh = oracle.entropies(h, [1.0, 0.5, 2.0])
        # MI(A, A) = H(A) (Eq. 2 with H(A, A) = H(A)); additive Tsallis I_q(A, A) = S_q(A)
        np.testing.assert_allclose(mi, hh[:, 0], rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(hh[:, 0], hh[:, 2], rtol=1e-13)


def test_shannon_matches_scipy_entropy():
    from scipy.stats import entropy

    fx, mv = phantoms.ellipsoid_pair(shape=(20, 22, 24), seed=8)
    q16 = oracle.affine_q16(oracle.affine(phantoms.TINY_MOTION, fx.shape, (1, 1, 1), mv.shape, (1, 1, 1)))
    h, n = oracle.joint_hist(fx, mv, q16, 32)
    hd = h.astype(np.float64)
    mi, hh = oracle.entropies(h, [1.0])
    assert abs(hh[0, 0] - entropy(hd.sum(1))) < 1e-12
    assert abs(hh[0, 1] - entropy(hd.sum(0))) < 1e-12
    assert abs(hh[0, 2] - entropy(hd.ravel())) < 1e-12
    _, hb = oracle.entropies(h, [1.0], bits=True)
    assert abs(hb[0, 2] - entropy(hd.ravel(), base=2)) < 1e-12


def test_integer_translation_exact_pairs():
    rng = np.random.default_rng(4)
    fx = rng.integers(0, 256, size=(9, 10, 11), dtype=np.uint8)
    mv = rng.integers(0, 256, size=(9, 10, 11), dtype=np.uint8)
    for d in [(1, 0, 0), (-2, 3, 1), (0, 0, -4), (5, -5, 2)]:
        q = IDENT.copy()
        q[3], q[7], q[11] = d[0] * 65536, d[1] * 65536, d[2] * 65536
        h, n = oracle.joint_hist(fx, mv, q, 16)
        dx, dy, dz = d
        nz, ny, nx = fx.shape
        assert n == (nx - abs(dx)) * (ny - abs(dy)) * (nz - abs(dz))
        # brute force with numpy slicing: fixed voxel i pairs with moving voxel i + d
        sl_f = tuple(slice(max(0, -s), n_ - max(0, s)) for s, n_ in zip((dz, dy, dx), fx.shape))
        sl_m = tuple(slice(max(0, s), n_ - max(0, -s)) for s, n_ in zip((dz, dy, dx), fx.shape))
        bf = (fx[sl_f].astype(np.int64) * 16) >> 8
        bm = (mv[sl_m].astype(np.int64) * 16) >> 8
        want = np.bincount((bf * 16 + bm).ravel(), minlength=256).reshape(16, 16)
        np.testing.assert_array_equal(h, want)


def test_rotations_about_centre_are_exact_permutations():
    rng = np.random.default_rng(5)
    mv = rng.integers(0, 4096, size=(7, 7, 7), dtype=np.uint16)
    fshape = mv.shape
    for axis, ang in [(5, 90.0), (5, 180.0), (5, -90.0), (3, 90.0), (4, 180.0)]:
        p = phantoms.identity_params(1)[0]
        p[axis] = ang
        q = oracle.affine_q16(oracle.affine(p, fshape, (1, 1, 1), fshape, (1, 1, 1)))
        out = oracle.resample(mv, q, fshape, depth=12)
        A = q[:, :3] // 65536
        b = q[:, 3] // 65536
        # every fixed voxel reads exactly one moving voxel
        k, j, i = np.meshgrid(np.arange(7), np.arange(7), np.arange(7), indexing="ij")
        src = np.einsum("ab,bzyx->azyx", A, np.stack([i, j, k])) + b[:, None, None, None]
        np.testing.assert_array_equal(out, mv[src[2], src[1], src[0]])


def test_resample_exact_at_integers_and_bounded_between_neighbours():
    rng = np.random.default_rng(6)
    mv = rng.integers(0, 4096, size=(12, 13, 14), dtype=np.uint16)
    for _ in range(10):
        p = phantoms.random_transforms(1, seed=int(rng.integers(1 << 30)), t_mm=2, r_deg=10, s_range=(0.9, 1.1))[0]
        q = oracle.affine_q16(oracle.affine(p, mv.shape, (1, 1, 1), mv.shape, (1, 1, 1)))
        out = oracle.resample(mv, q, mv.shape, depth=12)
        k, j, i = np.meshgrid(*(np.arange(s) for s in mv.shape), indexing="ij")
        U = np.stack([q[a, 0].astype(np.int64) * i + q[a, 1] * j + q[a, 2] * k + q[a, 3] for a in range(3)])
        u = U / 65536.0
        n = np.array(mv.shape[::-1])[:, None, None, None]
        inside = np.all((u >= 0) & (u <= n - 1), axis=0)
        assert np.all(out[~inside] == 0)
        lo = np.floor(u).astype(np.int64)
        hi = np.minimum(lo + 1, n - 1)
        corners = []
        for cz in (lo[2], hi[2]):
            for cy in (lo[1], hi[1]):
                for cx in (lo[0], hi[0]):
                    corners.append(mv[np.clip(cz, 0, mv.shape[0] - 1), np.clip(cy, 0, mv.shape[1] - 1),
                                      np.clip(cx, 0, mv.shape[2] - 1)])
        corners = np.stack(corners)
        o = out.astype(np.int64)
        assert np.all(o[inside] >= corners.min(0)[inside]) and np.all(o[inside] <= corners.max(0)[inside])
    # integer coordinates reproduce the moving value exactly
    q = IDENT.copy()
    q[3] = 2 * 65536
    out = oracle.resample(mv, q, mv.shape, depth=12)
    np.testing.assert_array_equal(out[:, :, :-2], mv[:, :, 2:])


def test_two_and_four_class_closed_forms():
    z, y, x = np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij")
    two = np.where(x < 4, 50, 200).astype(np.uint8)
    four = (((x >= 4) * 2 + (y >= 4)) * 60 + 10).astype(np.uint8)
    for vol, k in ((two, 2), (four, 4)):
        h, n = oracle.joint_hist(vol, vol, IDENT, 32)
        mi, hh = oracle.entropies(h, [1.0, 2.0])
        assert abs(mi[0] - math.log(k)) < 1e-13
        assert abs(mi[1] - (1 - 1 / k)) < 1e-13


def test_tsallis_limits():
    fx, mv = phantoms.ellipsoid_pair(shape=(20, 20, 20), seed=9)
    q16 = oracle.affine_q16(oracle.affine(phantoms.TINY_MOTION, fx.shape, (1, 1, 1), mv.shape, (1, 1, 1)))
    h, _ = oracle.joint_hist(fx, mv, q16, 32)
    p = h.astype(np.float64) / h.sum()
    _, hh = oracle.entropies(h, [1.0, 2.0, 0.0, 1 + 1e-4, 1 - 1e-4])
    H = hh[0, 2]
    assert abs(hh[1, 2] - (1 - np.sum(p * p))) < 1e-13        # S_2 = 1 - sum p^2
    assert abs(hh[2, 2] - (np.count_nonzero(h) - 1)) < 1e-9     # S_0 = #nonzero - 1
    d_plus, d_minus = hh[3, 2] - H, hh[4, 2] - H                  # S_q -> H linearly as q -> 1
    assert abs(d_plus) < 1e-3 and abs(d_minus) < 1e-3
    assert abs(d_plus + d_minus) < 1e-6 * max(abs(d_plus), 1e-12) * 1e3


def test_tsallis_pseudo_additivity_on_product_distribution():
    # for independent F, M: S_q(F,M) = S_q(F) + S_q(M) + (1-q) S_q(F) S_q(M)
    rng = np.random.default_rng(10)
    a = rng.integers(1, 50, 16).astype(np.float64)
    b = rng.integers(1, 50, 16).astype(np.float64)
    h = np.outer(a, b)
    for q in (0.5, 0.8, 1.5, 2.0):
        mi_pa, hh = oracle.entropies(h, [q], form=1)
        assert abs(mi_pa[0]) < 1e-12
        mi_add, _ = oracle.entropies(h, [q], form=0)
        assert abs(mi_add[0] + (1 - q) * hh[0, 0] * hh[0, 1]) < 1e-12
    mi, _ = oracle.entropies(h, [1.0])
    assert abs(mi[0]) < 1e-13


def test_mi_invariant_under_moving_bin_permutation():
    # MI depends only on the joint partition: permuting whole bins of the moving image changes nothing
    fx, mv = phantoms.ellipsoid_pair(shape=(16, 18, 20), seed=11)
    rng = np.random.default_rng(11)
    perm = rng.permutation(32)
    mv2 = (perm[mv >> 3] * 8 + (mv & 7)).astype(np.uint8)
    for d in [(0, 0, 0), (2, -1, 3)]:
        q = IDENT.copy()
        q[3], q[7], q[11] = d[0] * 65536, d[1] * 65536, d[2] * 65536
        m1, _, _ = oracle.mi_eval_q16(fx, mv, 32, q, [1.0, 0.5, 2.0])
        m2, _, _ = oracle.mi_eval_q16(fx, mv2, 32, q, [1.0, 0.5, 2.0])
        np.testing.assert_allclose(m1, m2, rtol=1e-12, atol=1e-14)


def test_swapping_the_volumes_transposes_the_histogram():
    # Eq. 2 is symmetric in its two images: with equal grids, swapping fixed and moving under the inverse
    # of a whole-voxel shift maps the same voxel pairs, so the joint histogram transposes, the marginal
    # entropies trade places and every MI (Shannon, both Tsallis forms) is unchanged
    fx, mv = phantoms.ellipsoid_pair(shape=(16, 18, 20), seed=14)
    assert fx.shape == mv.shape
    for d in [(0, 0, 0), (3, -2, 1), (-4, 5, -2)]:
        q, qi = IDENT.copy(), IDENT.copy()
        q[3], q[7], q[11] = d[0] * 65536, d[1] * 65536, d[2] * 65536
        qi[3], qi[7], qi[11] = -d[0] * 65536, -d[1] * 65536, -d[2] * 65536
        h1, n1 = oracle.joint_hist(fx, mv, q, 32)
        h2, n2 = oracle.joint_hist(mv, fx, qi, 32)
        assert n1 == n2 > 0
        np.testing.assert_array_equal(h1, h2.T)
        for form in (0, 1):
            mi1, hh1 = oracle.entropies(h1, [1.0, 0.5, 2.0], form=form)
            mi2, hh2 = oracle.entropies(h2, [1.0, 0.5, 2.0], form=form)
            np.testing.assert_allclose(mi1, mi2, rtol=1e-12, atol=1e-14)
            np.testing.assert_allclose(hh1[:, 0], hh2[:, 1], rtol=1e-12)
            np.testing.assert_allclose(hh1[:, 1], hh2[:, 0], rtol=1e-12)
            np.testing.assert_allclose(hh1[:, 2], hh2[:, 2], rtol=1e-12)


def test_shannon_mi_between_zero_and_the_smaller_marginal_entropy():
    # 0 <= I(F; M) <= min(H(F), H(M)) for any joint distribution (Eq. 2 with H(F, M) >= max(H(F), H(M))
    # and subadditivity): a sign or term slip in the reduction breaks one side on some transform
    fx, mv = phantoms.ellipsoid_pair(shape=(20, 22, 24), seed=15)
    prm = phantoms.random_transforms(12, seed=16, t_mm=4, r_deg=20, s_range=(0.85, 1.15))
    mi, hh, _ = oracle.mi_eval(fx, mv, 32, prm, [1.0])
    assert np.all(mi[:, 0] >= -1e-12)
    assert np.all(mi[:, 0] <= np.minimum(hh[:, 0, 0], hh[:, 0, 1]) + 1e-12)
    assert np.all(hh[:, 0, 2] >= np.maximum(hh[:, 0, 0], hh[:, 0, 1]) - 1e-12)


def test_independent_noise_miller_madow_band():
    rng = np.random.default_rng(12)
    shape = (64, 64, 64)
    bins = 32
    vals = []
    for _ in range(3):
        a = rng.integers(0, 256, shape, dtype=np.uint8)
        b = rng.integers(0, 256, shape, dtype=np.uint8)
        mi, _, _ = oracle.mi_eval_q16(a, b, bins, IDENT, [1.0])
        vals.append(mi[0, 0])
    bias = (bins - 1) ** 2 / (2 * np.prod(shape))
    assert 0.8 * bias < np.mean(vals) < 1.2 * bias


def test_empty_overlap_is_nan():
    fx, mv = phantoms.ellipsoid_pair(shape=(8, 8, 8), seed=13)
    q = IDENT.copy()
    q[3] = 100 * 65536
    mi, hh, cnt = oracle.mi_eval_q16(fx, mv, 16, q, [1.0, 2.0])
    assert cnt[0] == 0 and np.all(np.isnan(mi)) and np.all(np.isnan(hh))


def test_mi_eval_params_equals_q16_path_and_peaks_at_true_motion():
    fx, mv = phantoms.ellipsoid_pair(shape=(40, 40, 40), seed=14)
    prm = phantoms.tiny_sweep()
    mi, hh, cnt = oracle.mi_eval(fx, mv, 32, prm, [1.0, 0.5, 1.5], nthreads=2)
    q16 = np.stack([oracle.affine_q16(oracle.affine(p, fx.shape, (1, 1, 1), mv.shape, (1, 1, 1))) for p in prm])
    mi2, _, cnt2 = oracle.mi_eval_q16(fx, mv, 32, q16, [1.0, 0.5, 1.5])
    np.testing.assert_array_equal(mi, mi2)
    np.testing.assert_array_equal(cnt, cnt2)
    # the phantom's true motion beats every pure x translation (the paper's gold standard is the true pose)
    assert mi[0, 0] > mi[1:, 0].max()


def test_values_above_bit_depth_are_clamped_on_load():
    # depth 12: 5000 reads as 4095 before interpolation, so a half-voxel shift between
    # 100 and 5000 gives (100*128 + 4095*128 + 128) >> 8 = 2098, not the unclamped 2550
    mv = np.zeros((2, 2, 2), dtype=np.uint16)
    mv[:, :, 0] = 100
    mv[:, :, 1] = 5000
    q = IDENT.copy()
    q[3] = 32768
    out = oracle.resample(mv, q, (2, 2, 2), depth=12)
    assert out[0, 0, 0] == (100 * 128 + 4095 * 128 + 128) >> 8
