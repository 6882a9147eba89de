"""Pins of the oracle's Parzen soft histogram (R8) and its gradient (R9).

Expectations come from library routines (scipy's trilinear map_coordinates
and cubic B-spline basis), the B-spline partition of unity, product
distributions and central finite differences of the oracle's own FP64 MI.
"""
import numpy as np
import pytest

import oracle
from paper_1909_10690_gb300 import phantoms


def _small_pair(shape=(14, 16, 18), seed=21):
    f, m = phantoms.head_pair(shape=shape, spacing=(1.0, 1.0, 1.0), seed=seed, dtype=np.float32, noise=0.01)
    return f, m


def test_beta3_partition_of_unity_and_derivative():
    from scipy.interpolate import BSpline

    b = BSpline.basis_element(np.arange(-2.0, 3.0))
    rng = np.random.default_rng(0)
    for x in rng.uniform(-3, 3, 200):
        want = float(b(x)) if -2 < x < 2 else 0.0
        assert abs(oracle.beta3(x) - want) < 1e-14
        h = 1e-6
        assert abs(oracle.dbeta3(x) - (oracle.beta3(x + h) - oracle.beta3(x - h)) / (2 * h)) < 1e-8
    for x in rng.uniform(0, 50, 100):
        ks = np.arange(int(np.floor(x)) - 3, int(np.floor(x)) + 4)
        assert abs(sum(oracle.beta3(k - x) for k in ks) - 1.0) < 1e-14
        assert abs(sum(oracle.dbeta3(k - x) for k in ks)) < 1e-14


def test_parzen_fixed_bin_rule():
    B = 32
    vol = np.array([0, 1, 2048, 4095], dtype=np.uint16).reshape(1, 1, 4)
    fb = oracle.parzen_fixed_bins(vol, B, depth=12)
    assert fb.ravel()[0] == 2 and fb.ravel()[-1] == B - 2
    ramp = np.arange(4096, dtype=np.uint16).reshape(1, 16, 256)
    fb = oracle.parzen_fixed_bins(ramp, B, depth=12).ravel()
    assert np.all(np.diff(fb) >= 0) and set(fb) == set(range(2, B - 1))
    f32 = np.array([0.0, 0.5, 1.0, 1.5, -1.0], dtype=np.float32).reshape(1, 1, 5)
    assert list(oracle.parzen_fixed_bins(f32, B).ravel()) == [2, 2 + (B - 4) // 2, B - 2, B - 2, 2]


def test_parzen_histogram_matches_scipy_brute_force():
    from scipy.interpolate import BSpline
    from scipy.ndimage import map_coordinates

    f, m = _small_pair(shape=(6, 7, 8), seed=22)
    B = 16
    p = np.array([0.7, -0.4, 0.3, 6.0, -4.0, 9.0, 1.05, 0.95, 1.02], dtype=np.float32)
    aff = oracle.affine(p, f.shape, (1, 1, 1), m.shape, (1, 1, 1))
    mi, _, n, P = oracle.parzen(f, m, aff, B, [1.0], want_hist=True)
    k, j, i = np.meshgrid(*(np.arange(s) for s in f.shape), indexing="ij")
    u = np.stack([aff[a, 0] * i + aff[a, 1] * j + aff[a, 2] * k + aff[a, 3] for a in range(3)])
    nm = np.array(m.shape[::-1])[:, None, None, None]
    inside = np.all((u >= 0) & (u <= nm - 1), axis=0)
    vals = map_coordinates(m.astype(np.float64), [u[2][inside], u[1][inside], u[0][inside]], order=1,
                           mode="nearest")
    fb = np.floor(np.clip(f[inside].astype(np.float64), 0, 1) * (B - 4)).astype(int) + 2
    mt = vals * (B - 4) + 2
    b3 = BSpline.basis_element(np.arange(-2.0, 3.0), extrapolate=False)
    want = np.zeros((B, B))
    for r, x in zip(fb, mt):
        for kk in range(B):
            w = b3(kk - x)
            if np.isfinite(w):
                want[r, kk] += w
    assert n == inside.sum()
    np.testing.assert_allclose(P, want / n, rtol=0, atol=1e-13)
    # partition of unity: the soft histogram sums to 1
    assert abs(P.sum() - 1.0) < 1e-13


def test_parzen_constant_moving_gives_zero_mi_and_gradient():
    f, _ = _small_pair(seed=23)
    m = np.full(f.shape, 0.37, dtype=np.float32)
    p = np.array([0.3, 0.2, -0.1, 3, 2, -4, 1.02, 0.98, 1.0], dtype=np.float32)
    aff, J = oracle.affine(p, f.shape, (1, 1, 1), m.shape, (1, 1, 1), with_jacobian=True)
    mi, g, n = oracle.parzen(f, m, aff, 32, [1.0, 0.7, 1.3], daff=J, form=1)
    assert n > 0
    np.testing.assert_allclose(mi, 0.0, atol=1e-12)
    np.testing.assert_allclose(g, 0.0, atol=1e-12)


def _fd_worst(form, h, trials=3, seed=25, qs=(1.0, 0.7, 1.3)):
    f, m = _small_pair(shape=(16, 18, 20), seed=24)
    B = 32
    rng = np.random.default_rng(seed)
    worst = 0.0
    for trial in range(trials):
        p = np.array([*rng.uniform(-2, 2, 3), *rng.uniform(-8, 8, 3), *rng.uniform(0.93, 1.07, 3)], dtype=np.float32)
        aff, J = oracle.affine(p, f.shape, (1, 1, 1), m.shape, (1, 1, 1), with_jacobian=True)
        mi, g, n = oracle.parzen(f, m, aff, B, list(qs), daff=J, form=form)
        mask = oracle.overlap_mask(f.shape, m.shape, aff)
        fd = np.zeros((len(qs), 9))
        for k in range(9):
            # step along the exact Jacobian column: the builder's Jacobian is pinned separately
            ap = aff + h * J[:, k].reshape(3, 4)
            am = aff - h * J[:, k].reshape(3, 4)
            mp, _, _ = oracle.parzen(f, m, ap, B, list(qs), form=form, mask=mask)
            mm, _, _ = oracle.parzen(f, m, am, B, list(qs), form=form, mask=mask)
            fd[:, k] = (mp - mm) / (2 * h)
        for iq in range(len(qs)):
            worst = max(worst, np.abs(g[iq] - fd[iq]).max() / np.abs(fd[iq]).max())
    return worst


@pytest.mark.parametrize("form", [0, 1])
def test_parzen_gradient_matches_central_differences(form):
    # small step: few voxels cross a trilinear kink (the gap shrinks linearly with h),
    # so FD converges to the analytic adjoint
    assert _fd_worst(form, 1e-6) < 1e-6


def test_parzen_gradient_fd_at_1e_3_kink_bound():
    # at h = 1e-3 the scale steps move far voxels by ~1e-2 voxel and cross trilinear
    # kinks (grid planes); on this small volume the gap stays below 20 percent
    assert _fd_worst(0, 1e-3, trials=2) < 0.2


def test_parzen_mask_reproduces_overlap():
    f, m = _small_pair(seed=26)
    p = np.array([1.5, -0.5, 0.25, 5, -3, 2, 1.05, 1.0, 0.95], dtype=np.float32)
    aff = oracle.affine(p, f.shape, (1, 1, 1), m.shape, (1, 1, 1))
    mask = oracle.overlap_mask(f.shape, m.shape, aff)
    a, _, n1 = oracle.parzen(f, m, aff, 24, [1.0, 2.0])
    b, _, n2 = oracle.parzen(f, m, aff, 24, [1.0, 2.0], mask=mask)
    assert n1 == n2 == mask.sum()
    np.testing.assert_array_equal(a, b)


def test_parzen_empty_overlap_nan():
    f, m = _small_pair(shape=(6, 6, 6), seed=27)
    aff = np.hstack([np.eye(3), np.full((3, 1), 100.0)])
    mi, g, n = oracle.parzen(f, m, aff, 16, [1.0], daff=np.zeros((12, 9)))
    assert n == 0 and np.isnan(mi[0]) and np.all(np.isnan(g))


def _mirror_symmetric(shape, seed):
    # a value per (|i - c_x|, |j - c_y|, |k - c_z|): exactly symmetric under each axis mirror
    rng = np.random.default_rng(seed)
    table = rng.uniform(0.1, 0.9, size=tuple((n + 1) // 2 for n in shape)).astype(np.float32)
    idx = [np.minimum(np.arange(n), n - 1 - np.arange(n)) for n in shape]
    return table[np.ix_(idx[0], idx[1], idx[2])]


def test_parzen_symmetric_pair_has_no_translation_or_rotation_gradient():
    # f = m mirror-symmetric about the centre on every axis, uniform scale sigma != 1 (samples off the
    # grid planes, even sizes): a mirror maps t to -t and each rotation angle to its negative, so MI is
    # even in them and their derivatives vanish; the scale derivatives do not
    f = _mirror_symmetric((12, 14, 16), seed=28)
    assert np.array_equal(f, f[::-1, :, :]) and np.array_equal(f, f[:, ::-1, :]) and np.array_equal(f, f[:, :, ::-1])
    p = np.array([0, 0, 0, 0, 0, 0, 1.04, 1.04, 1.04], dtype=np.float32)
    aff, J = oracle.affine(p, f.shape, (1, 1, 1), f.shape, (1, 1, 1), with_jacobian=True)
    mi, g, n = oracle.parzen(f, f, aff, 32, [1.0, 0.7, 1.3], daff=J)
    for iq in range(3):
        assert np.abs(g[iq, 6:]).max() > 1e-3
        assert np.abs(g[iq, :6]).max() <= 1e-10 * np.abs(g[iq, 6:]).max()


def test_parzen_mi_of_aligned_separated_classes_is_the_class_entropy():
    # classes in distinct fixed bins and >= 4 moving bins apart: the B-spline spread adds the same
    # entropy to H(M) and H(F, M), so Shannon Parzen MI = H(class proportions) exactly (the hard MI)
    f = np.full((8, 10, 12), 0.2, np.float32)
    f[:, :, 9:] = 0.8  # a quarter of the voxels
    aff = np.hstack([np.eye(3), np.zeros((3, 1))])
    for B in (16, 32, 64):
        mi, _, n = oracle.parzen(f, f, aff, B, [1.0])
        want = -(0.25 * np.log(0.25) + 0.75 * np.log(0.75))
        assert n == f.size
        assert abs(mi[0] - want) < 1e-12, (B, mi[0], want)
