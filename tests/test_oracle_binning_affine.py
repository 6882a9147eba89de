"""Pins of the oracle's binning (R1), transform builder (R2) and 16.16 quantiser (R3).

Each expectation comes from a fact other than the oracle's own formula:
equal-width bins, exact rotations, geometric identities, finite differences.
"""
import numpy as np
import pytest

import oracle
from paper_1909_10690_gb300 import phantoms


def test_bins_equal_width_power_of_two():
    # 2^d / bins grey levels per bin: bin = v // width for every value
    for depth, bins in [(8, 32), (8, 256), (12, 64), (12, 128), (12, 256), (8, 2)]:
        width = (1 << depth) // bins
        for v in range(0, 1 << depth, max(1, (1 << depth) // 512)):
            assert oracle.bin_of(v, bins, depth) == v // width


def test_bins_full_histogram_is_identity():
    # bins = 2^d is one bin per grey level ("full histogram", Discussion)
    for v in range(256):
        assert oracle.bin_of(v, 256, 8) == v


@pytest.mark.parametrize("bins", [3, 5, 7, 100, 255])
def test_bins_partition_any_count(bins):
    # any bin count: contiguous, non-decreasing, all bins used, sizes differ by <= 1
    depth = 8
    b = np.array([oracle.bin_of(v, bins, depth) for v in range(256)])
    assert b[0] == 0 and b[-1] == bins - 1
    assert np.all(np.diff(b) >= 0) and np.all(np.diff(b) <= 1)
    sizes = np.bincount(b, minlength=bins)
    assert sizes.min() >= 1 and sizes.max() - sizes.min() <= 1


def test_bins_clamp_above_depth():
    assert oracle.bin_of(4095, 64, 12) == 63
    assert oracle.bin_of(4096, 64, 12) == 63
    assert oracle.bin_of(65535, 64, 12) == 63


def test_f32_to_u16_round_half_even_and_clamp():
    x = np.array([0.0, 1.0, -0.5, 2.0, np.nan, 0.5 / 65535, 1.5 / 65535], dtype=np.float32)
    out = oracle.f32_to_u16(x.reshape(1, 1, -1)).ravel()
    assert list(out[:5]) == [0, 65535, 0, 65535, 0]
    # exact ties are rare in float; check the nearest integer instead
    assert out[5] in (0, 1) and out[6] in (1, 2)


def _aff(params, fs=(16, 16, 16), sf=(1, 1, 1), ms=None, sm=None):
    return oracle.affine(params, fs, sf, ms or fs, sm or sf)


def test_affine_identity_and_translation():
    p = phantoms.identity_params(1)[0]
    a = _aff(p)
    assert np.array_equal(a, np.hstack([np.eye(3), np.zeros((3, 1))]))
    p = p.copy()
    p[0:3] = [2.5, -3.0, 1.2]
    a = _aff(p, fs=(20, 18, 16), sf=(1.0, 2.0, 1.2))
    # translation in mm divides by the moving spacing
    np.testing.assert_allclose(a[:, 3], [2.5 / 1.0, -3.0 / 2.0, 1.2 / 1.2], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(a[:, :3], np.eye(3))


def test_affine_maps_centre_to_centre_plus_t():
    rng = np.random.default_rng(0)
    for _ in range(20):
        p = phantoms.random_transforms(1, seed=int(rng.integers(1 << 30)))[0]
        fs, ms = (30, 24, 20), (26, 28, 22)
        sf, sm = (1.0, 0.875, 1.25), (1.125, 1.0, 1.375)
        a = oracle.affine(p, fs, sf, ms, sm)
        cf = (np.array(fs[::-1]) - 1) / 2.0
        cm = (np.array(ms[::-1]) - 1) / 2.0
        u = a[:, :3] @ cf + a[:, 3]
        np.testing.assert_allclose(u * np.array(sm), cm * np.array(sm) + p[0:3].astype(np.float64), atol=1e-9)


def test_affine_matches_geometric_motion():
    # the affine in index space is the phantom module's physical motion conjugated by the spacings
    rng = np.random.default_rng(1)
    fs, ms = (30, 24, 20), (26, 28, 22)
    sf, sm = np.array([1.0, 0.875, 1.25]), np.array([1.125, 1.0, 1.375])
    for _ in range(20):
        p = phantoms.random_transforms(1, seed=int(rng.integers(1 << 30)))[0].astype(np.float64)
        L, t = phantoms.motion_matrix(p)
        cf = sf * (np.array(fs[::-1]) - 1) / 2
        cm = sm * (np.array(ms[::-1]) - 1) / 2
        idx = rng.uniform(0, 20, 3)
        pm = L @ (sf * idx - cf) + cm + t
        a = oracle.affine(p.astype(np.float32), fs, tuple(sf.astype(np.float32)), ms, tuple(sm.astype(np.float32)))
        np.testing.assert_allclose(a[:, :3] @ idx + a[:, 3], pm / sm, atol=1e-5)


def test_affine_rotation_z_90_exact_q16():
    p = phantoms.identity_params(1)[0]
    p[5] = 90.0
    q = oracle.affine_q16(_aff(p, fs=(5, 5, 5)))
    # cos and sin quantise to exactly 0 and +-1 in 16.16; centre (2, 2, 2) is fixed
    np.testing.assert_array_equal(q[:, :3], np.array([[0, -65536, 0], [65536, 0, 0], [0, 0, 65536]]))
    np.testing.assert_array_equal(q[:, 3], [4 * 65536, 0, 0])


def test_affine_rotations_are_orthonormal_and_right_handed():
    rng = np.random.default_rng(2)
    for _ in range(20):
        p = phantoms.identity_params(1)[0]
        p[3:6] = rng.uniform(-180, 180, 3)
        A = _aff(p)[:, :3]
        np.testing.assert_allclose(A @ A.T, np.eye(3), atol=1e-12)
        assert abs(np.linalg.det(A) - 1.0) < 1e-12
    p = phantoms.identity_params(1)[0]
    p[5] = 30.0  # positive rz turns +x towards +y
    A = _aff(p)[:, :3]
    np.testing.assert_allclose(A @ [1, 0, 0], [np.cos(np.pi / 6), np.sin(np.pi / 6), 0], atol=1e-12)
    p = phantoms.identity_params(1)[0]
    p[3] = 30.0  # positive rx turns +y towards +z
    A = _aff(p)[:, :3]
    np.testing.assert_allclose(A @ [0, 1, 0], [0, np.cos(np.pi / 6), np.sin(np.pi / 6)], atol=1e-12)


def test_affine_scale_factors():
    p = phantoms.identity_params(1)[0]
    p[6:9] = [1.25, 0.5, 2.0]
    a = _aff(p, fs=(9, 9, 9))
    np.testing.assert_allclose(np.diag(a[:, :3]), [1.25, 0.5, 2.0])
    # the centre stays put: b = c - S c
    np.testing.assert_allclose(a[:, 3], 4 * (1 - np.array([1.25, 0.5, 2.0])))


def test_affine_jacobian_matches_finite_differences():
    rng = np.random.default_rng(3)
    fs, ms, sf, sm = (30, 24, 20), (26, 28, 22), (1.0, 0.9, 1.2), (1.1, 1.0, 1.3)
    lib = oracle._load()
    import ctypes
    nf = np.array(fs[::-1], np.int32)
    nm = np.array(ms[::-1], np.int32)
    sfa = np.array(sf, np.float32)
    sma = np.array(sm, np.float32)
    for _ in range(5):
        p = phantoms.random_transforms(1, seed=int(rng.integers(1 << 30)))[0]
        _, J = oracle.affine(p, fs, sf, ms, sm, with_jacobian=True)
        # central differences of the FP64 builder; parameters perturbed in float64 through float32 is too coarse,
        # so differentiate a float64 re-evaluation of the same builder via small float32-representable steps
        for k in range(9):
            h = 2.0 ** -10
            pp, pm = p.copy(), p.copy()
            pp[k] += np.float32(h)
            pm[k] -= np.float32(h)
            ap, am = np.empty(12), np.empty(12)
            lib.orc_affine(oracle._p(pp), oracle._p(nf), oracle._p(sfa), oracle._p(nm), oracle._p(sma), oracle._p(ap), None)
            lib.orc_affine(oracle._p(pm), oracle._p(nf), oracle._p(sfa), oracle._p(nm), oracle._p(sma), oracle._p(am), None)
            fd = (ap - am) / float(pp[k] - pm[k])
            np.testing.assert_allclose(J[:, k], fd, rtol=1e-5, atol=1e-6)


def test_q16_rounding_and_range():
    a = np.zeros((3, 4))
    a[0, 0] = 1.0
    a[0, 1] = 0.5 / 65536  # exact tie rounds away from zero (llround)
    a[0, 2] = -0.5 / 65536
    a[1, 3] = 1.25
    q = oracle.affine_q16(a)
    assert q[0, 0] == 65536 and q[0, 1] == 1 and q[0, 2] == -1 and q[1, 3] == 81920
    a[2, 3] = 40000.0  # 40000 * 65536 > 2^31
    with pytest.raises(OverflowError):
        oracle.affine_q16(a)


# --- R14 unit-ball (versor) rotation and R15 zero-centred scale -------------------------------------------------

def _rot_of(p, rotation="versor", scale="factor"):
    # with equal unit spacings, equal shapes and unit scale, A is the rotation matrix itself
    return oracle.affine(p, (9, 9, 9), (1, 1, 1), (9, 9, 9), (1, 1, 1), rotation=rotation, scale=scale)[:, :3]


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_versor_on_an_axis_is_the_euler_rotation(axis):
    # v = sin(theta / 2) e_axis is the turn by theta about that axis: compare with the Euler builder at the
    # angle the float32 parameter actually represents
    for theta_deg in (-150.0, -33.0, 5.0, 90.0, 171.0):
        s = np.float32(np.sin(np.radians(theta_deg) / 2))
        v = np.zeros(9, np.float32)
        v[6:] = 1
        v[3 + axis] = s
        e = np.zeros(9, np.float32)
        e[6:] = 1
        e[3 + axis] = np.float32(np.degrees(2 * np.arcsin(np.float64(s))))
        np.testing.assert_allclose(_rot_of(v), _rot_of(e, rotation="euler"), atol=2e-7)


def test_versor_rotations_are_proper_with_the_unit_ball_angle():
    rng = np.random.default_rng(21)
    for _ in range(200):
        v = rng.uniform(-1, 1, 3)
        p = np.concatenate([[0, 0, 0], v, [1, 1, 1]]).astype(np.float32)
        R = _rot_of(p)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)
        assert abs(np.linalg.det(R) - 1) < 1e-12
        n = min(np.linalg.norm(p[3:6].astype(np.float64)), 1.0)
        # trace = 1 + 2 cos(angle), angle = 2 asin |v| (a half turn on and outside the sphere)
        assert abs(np.trace(R) - (1 + 2 * np.cos(2 * np.arcsin(n)))) < 1e-9
        axis = p[3:6].astype(np.float64)
        np.testing.assert_allclose(R @ axis, axis, atol=1e-9)  # the axis is fixed


def test_versor_outside_the_ball_lands_on_the_sphere():
    for v in ([0, 0, 2.0], [0.9, -0.9, 0.4], [1.0, 0, 0]):
        p = np.concatenate([[0, 0, 0], v, [1, 1, 1]]).astype(np.float32)
        R = _rot_of(p)
        np.testing.assert_allclose(R @ R, np.eye(3), atol=1e-12)  # a half turn
        q = p.copy()
        q[3:6] = p[3:6] * np.float32(3.0)  # further out along the same ray: the same point of the sphere
        np.testing.assert_allclose(_rot_of(q), R, atol=1e-7)


def test_zero_centred_scale_is_one_plus_offset():
    fs, ms, sf, sm = (20, 22, 18), (19, 21, 23), (1.0, 0.8, 1.25), (1.0, 1.0, 0.5)
    for s in ([0.25, -0.5, 0.125], [0, 0, 0], [-0.75, 0.5, 1.0]):
        off = np.array([1, -2, 3, 10, -20, 5, *s], np.float32)
        fac = off.copy()
        fac[6:] = 1 + np.array(s, np.float32)  # exact in float32 for these offsets
        np.testing.assert_array_equal(oracle.affine(off, fs, sf, ms, sm, scale="offset"), oracle.affine(fac, fs, sf, ms, sm))


@pytest.mark.parametrize("inside", [True, False])
def test_versor_and_offset_jacobian_match_finite_differences(inside):
    rng = np.random.default_rng(5 if inside else 6)
    fs, ms, sf, sm = (30, 24, 20), (26, 28, 22), (1.0, 0.9, 1.2), (1.1, 1.0, 1.3)
    for _ in range(5):
        v = rng.normal(size=3)
        v *= (rng.uniform(0.1, 0.8) if inside else rng.uniform(1.2, 2.0)) / np.linalg.norm(v)
        p = np.concatenate([rng.uniform(-5, 5, 3), v, rng.uniform(-0.2, 0.2, 3)]).astype(np.float32)
        _, J = oracle.affine(p, fs, sf, ms, sm, with_jacobian=True, rotation="versor", scale="offset")
        for k in range(9):
            h = np.float32(2.0 ** -12)
            pp, pm = p.copy(), p.copy()
            pp[k] += h
            pm[k] -= h
            ap = oracle.affine(pp, fs, sf, ms, sm, rotation="versor", scale="offset").ravel()
            am = oracle.affine(pm, fs, sf, ms, sm, rotation="versor", scale="offset").ravel()
            fd = (ap - am) / float(pp[k] - pm[k])
            np.testing.assert_allclose(J[:, k], fd, rtol=1e-4, atol=1e-5)
