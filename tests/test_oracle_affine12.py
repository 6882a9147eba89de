"""Pins of the oracle's general affine (R17): [M | t], the Methodology's 12 degrees of freedom.

Expectations come from facts other than the builder's own formula: the
identity, the phantom module's physical motion (R diag(sigma), t) of the
9-parameter form, an integer shear whose joint histogram has a closed-form
overlap count and a numpy brute force, and finite differences.
"""
import numpy as np
import pytest

import oracle
from paper_1909_10690_gb300 import phantoms

GEOM = [((30, 24, 20), (1.0, 0.875, 1.25), (26, 28, 22), (1.125, 1.0, 1.375)),
        ((16, 16, 16), (1.0, 1.0, 1.0), (16, 16, 16), (1.0, 1.0, 1.0))]


def _mt(M, t):
    return np.hstack([np.asarray(M, np.float64), np.asarray(t, np.float64).reshape(3, 1)]).astype(np.float32).ravel()


def test_affine12_identity_is_exact():
    for fs in [(16, 16, 16), (9, 14, 21)]:
        for sp in [(1.0, 1.0, 1.0), (0.5, 1.25, 2.0)]:
            a = oracle.affine(_mt(np.eye(3), [0, 0, 0]), fs, sp, fs, sp, transform="affine")
            assert np.array_equal(a, np.hstack([np.eye(3), np.zeros((3, 1))]))


@pytest.mark.parametrize("geom", GEOM)
def test_affine12_of_the_motion_equals_the_parameter_form(geom):
    # M = R diag(sigma) and t of a 9-parameter motion (the phantom module's own rotation code) give the
    # same index-space affine as the 9-parameter builder, up to M's rounding to float32
    fs, sf, ms, sm = geom
    rng = np.random.default_rng(40)
    for _ in range(20):
        p = phantoms.random_transforms(1, seed=int(rng.integers(1 << 30)))[0]
        L, t = phantoms.motion_matrix(p.astype(np.float64))
        a12 = oracle.affine(_mt(L, t), fs, sf, ms, sm, transform="affine")
        a9 = oracle.affine(p, fs, sf, ms, sm)
        np.testing.assert_allclose(a12, a9, rtol=0, atol=3e-5)


def test_affine12_integer_shear_histogram_closed_form():
    # x' = x + (y - c_y) about the centre (M = [[1, 1, 0], [0, 1, 0], [0, 0, 1]], unit spacing, odd ny):
    # every coordinate is an integer, fixed voxel (i, j, k) pairs with moving voxel (i + j - c_y, j, k), and
    # the overlap holds sum_j (nx - |j - c_y|) * nz voxels
    rng = np.random.default_rng(41)
    nz, ny, nx = 7, 9, 13
    fx = rng.integers(0, 256, size=(nz, ny, nx), dtype=np.uint8)
    mv = rng.integers(0, 256, size=(nz, ny, nx), dtype=np.uint8)
    for shear in (1, -1, 2):
        M = np.eye(3)
        M[0, 1] = shear
        aff = oracle.affine(_mt(M, [0, 0, 0]), fx.shape, (1, 1, 1), mv.shape, (1, 1, 1), transform="affine")
        q = oracle.affine_q16(aff)
        assert np.all(q % 65536 == 0)
        h, n = oracle.joint_hist(fx, mv, q, 32)
        cy = (ny - 1) // 2
        assert n == sum(max(0, nx - abs(shear * (j - cy))) for j in range(ny)) * nz
        want = np.zeros((32, 32), np.int64)
        for j in range(ny):
            d = shear * (j - cy)
            i = np.arange(nx)
            ok = (i + d >= 0) & (i + d < nx)
            bf = (fx[:, j, i[ok]].astype(np.int64) * 32) >> 8
            bm = (mv[:, j, i[ok] + d].astype(np.int64) * 32) >> 8
            np.add.at(want, (bf.ravel(), bm.ravel()), 1)
        np.testing.assert_array_equal(h, want)


def test_affine12_jacobian_matches_finite_differences():
    fs, sf, ms, sm = GEOM[0]
    lib = oracle._load()
    nf = np.array(fs[::-1], np.int32)
    nm = np.array(ms[::-1], np.int32)
    sfa = np.array(sf, np.float32)
    sma = np.array(sm, np.float32)
    rng = np.random.default_rng(42)
    for _ in range(5):
        p = _mt(np.eye(3) + rng.uniform(-0.2, 0.2, (3, 3)), rng.uniform(-5, 5, 3))
        _, J = oracle.affine(p, fs, sf, ms, sm, transform="affine", with_jacobian=True)
        assert J.shape == (12, 12)
        for k in range(12):
            h = np.float32(2.0 ** -8)
            pp, pm = p.copy(), p.copy()
            pp[k] += h
            pm[k] -= h
            ap, am = np.empty(12), np.empty(12)
            lib.orc_affine_matrix(oracle._p(pp), oracle._p(nf), oracle._p(sfa), oracle._p(nm), oracle._p(sma),
                                  oracle._p(ap), None)
            lib.orc_affine_matrix(oracle._p(pm), oracle._p(nf), oracle._p(sfa), oracle._p(nm), oracle._p(sma),
                                  oracle._p(am), None)
            fd = (ap - am) / float(pp[k] - pm[k])
            np.testing.assert_allclose(J[:, k], fd, rtol=1e-9, atol=1e-9)


def test_affine12_parzen_gradient_matches_central_differences():
    f, m = phantoms.head_pair(shape=(16, 18, 20), spacing=(1.0, 1.0, 1.0), seed=24, dtype=np.float32, noise=0.01)
    rng = np.random.default_rng(43)
    qs = [1.0, 0.7, 1.3]
    h = 1e-6
    for _ in range(2):
        p = _mt(np.eye(3) + rng.uniform(-0.08, 0.08, (3, 3)), rng.uniform(-2, 2, 3))
        aff, J = oracle.affine(p, f.shape, (1, 1, 1), m.shape, (1, 1, 1), transform="affine", with_jacobian=True)
        mi, g, n = oracle.parzen(f, m, aff, 32, qs, daff=J)
        assert g.shape == (3, 12) and n > 0
        mask = oracle.overlap_mask(f.shape, m.shape, aff)
        fd = np.zeros((3, 12))
        for k in range(12):
            mp, _, _ = oracle.parzen(f, m, aff + h * J[:, k].reshape(3, 4), 32, qs, mask=mask)
            mm, _, _ = oracle.parzen(f, m, aff - h * J[:, k].reshape(3, 4), 32, qs, mask=mask)
            fd[:, k] = (mp - mm) / (2 * h)
        for iq in range(3):
            assert np.abs(g[iq] - fd[iq]).max() / np.abs(fd[iq]).max() < 1e-6


def test_affine12_singular_and_reflection_closed_forms():
    # M = 0 sends every fixed voxel to the moving centre (an integer index for odd sizes): all counts fall
    # in the centre value's bin, distributed like the fixed histogram.  M = diag(-1, 1, 1) mirrors x about
    # the centre: fixed voxel (i, j, k) pairs with moving voxel (nx - 1 - i, j, k)
    rng = np.random.default_rng(44)
    f = rng.integers(0, 256, size=(5, 7, 9), dtype=np.uint8)
    m = rng.integers(0, 256, size=(5, 7, 9), dtype=np.uint8)
    bins = 16
    bf = (f.astype(np.int64) * bins) >> 8
    q = oracle.affine_q16(oracle.affine(_mt(np.zeros((3, 3)), [0, 0, 0]), f.shape, (1, 1, 1), m.shape, (1, 1, 1),
                                        transform="affine"))
    assert np.all(q[:, :3] == 0)
    h, n = oracle.joint_hist(f, m, q, bins)
    assert n == f.size
    want = np.zeros((bins, bins), np.int64)
    want[:, (int(m[2, 3, 4]) * bins) >> 8] = np.bincount(bf.ravel(), minlength=bins)
    np.testing.assert_array_equal(h, want)
    q = oracle.affine_q16(oracle.affine(_mt(np.diag([-1.0, 1.0, 1.0]), [0, 0, 0]), f.shape, (1, 1, 1), m.shape,
                                        (1, 1, 1), transform="affine"))
    h, n = oracle.joint_hist(f, m, q, bins)
    bm = (m[:, :, ::-1].astype(np.int64) * bins) >> 8
    assert n == f.size
    np.testing.assert_array_equal(h, np.bincount((bf * bins + bm).ravel(), minlength=bins * bins).reshape(bins, bins))
