"""A translation map of the metric through the batched path (the Methodology's parameter-space maps)."""
import numpy as np
import pytest

import oracle
from paper_1909_10690_gb300 import maps, phantoms

pytestmark = pytest.mark.gpu


def test_translation_map_matches_oracle_and_peaks_at_the_motion(cuda_lib):
    motion = (2, -2, 1, 0, 0, 0, 1, 1, 1)  # whole voxels (1 mm spacing): a grid point of the map below
    f, m = phantoms.ellipsoid_pair(shape=(48, 48, 48), seed=70, motion=motion)
    ctx = cuda_lib.Context(f, m, bins=32)
    steps = 9
    mp = maps.param_map(ctx, "translation", -4, 4, steps, q=[1.0, 1.5], chunk=200)
    assert mp.shape == (steps, steps, steps, 2)
    T = maps.grid("translation", -4, 4, steps)
    rng = np.random.default_rng(71)
    sample = rng.choice(len(T), 6, replace=False)
    mi_o, h_o, _ = oracle.mi_eval(f, m, 32, T[sample], [1.0, 1.5], fixed_depth=8, moving_depth=8, nthreads=8)
    got = mp.reshape(-1, 2)[sample]
    scale = np.maximum(np.abs(mi_o), h_o[..., 2])
    assert np.all(np.abs(got - mi_o) <= 1e-6 * scale)
    # Eq. 3: the map's maximum is the motion, and the ascent from most of the map ends there
    truth = (2 + 4, -2 + 4, 1 + 4)
    assert np.unravel_index(np.argmax(mp[..., 0]), mp.shape[:3]) == truth
    assert maps.capture_fraction(mp[..., 0], truth) > 0.5
    path = maps.ascent_path(mp[..., 0], (0, 8, 0))
    assert all(mp[b][0] > mp[a][0] for a, b in zip(path, path[1:]))


def _oracle_on_grid(f, m, bins, T, qs, rotation, scale):
    q16 = np.stack([oracle.affine_q16(oracle.affine(p, f.shape, (1, 1, 1), m.shape, (1, 1, 1), rotation=rotation,
                                                    scale=scale)) for p in T])
    return oracle.mi_eval_q16(f, m, bins, q16, qs, fixed_depth=8, moving_depth=8, nthreads=8)


def test_rotation_map_on_the_unit_ball_crosses_its_surface(cuda_lib):
    # the Results' rotation maps: the three parameters are a unit-ball versor, points outside the
    # ball (|v| up to 0.7 sqrt 3 = 1.21 at the corners) land on its surface (half turns).  The moving
    # phantom is turned 2 asin(0.175) about z, the grid point (0, 0, 0.175) of a 9^3 grid on +-0.7
    vz = 0.175
    motion = (0, 0, 0, 0, 0, np.degrees(2 * np.arcsin(vz)), 1, 1, 1)
    f, m = phantoms.ellipsoid_pair(shape=(40, 44, 48), seed=72, motion=motion)
    ctx = cuda_lib.Context(f, m, bins=32, rotation="versor")
    steps, qs = 9, [1.0, 1.5]
    mp = maps.param_map(ctx, "rotation", -0.7, 0.7, steps, q=qs, chunk=300)
    T = maps.grid("rotation", -0.7, 0.7, steps)
    norm = np.linalg.norm(T[:, 3:6].astype(np.float64), axis=1)
    rng = np.random.default_rng(73)
    inside, outside = np.nonzero(norm < 1.0)[0], np.nonzero(norm > 1.0)[0]
    sample = np.concatenate([rng.choice(inside, 5, replace=False), rng.choice(outside, 5, replace=False)])
    mi_o, h_o, _ = _oracle_on_grid(f, m, 32, T[sample], qs, "versor", "factor")
    got = mp.reshape(-1, 2)[sample]
    assert np.all(np.abs(got - mi_o) <= 1e-6 * np.maximum(np.abs(mi_o), h_o[..., 2])), (got, mi_o)
    # Eq. 3 on the map: the Shannon maximum is the grid point of the true rotation
    assert np.unravel_index(np.argmax(mp[..., 0]), mp.shape[:3]) == (4, 4, 5)
    # outside the ball only the direction counts: a corner and twice the corner are the same half turn
    far = maps.identity()
    far[3:6] = (0.7, 0.7, 0.7)
    farther = far.copy()
    farther[3:6] *= 2
    _, q, _ = ctx.affine(np.stack([far, farther]))
    np.testing.assert_array_equal(q[0], q[1])
    a, b = ctx.eval(np.stack([far, farther]), qs)
    np.testing.assert_array_equal(a, b)


def test_scale_map_with_zero_centred_parameters(cuda_lib):
    # the Results' scale maps: zero-centred parameters sigma = 1 + s; the moving phantom is scaled by
    # (1.05, 0.95, 1.10), the grid point (0.05, -0.05, 0.10) of a 9^3 grid on +-0.2
    motion = (0, 0, 0, 0, 0, 0, 1.05, 0.95, 1.10)
    f, m = phantoms.ellipsoid_pair(shape=(40, 44, 48), seed=74, motion=motion)
    ctx = cuda_lib.Context(f, m, bins=32, scale="offset")
    steps, qs = 9, [1.0, 0.5]
    mp = maps.param_map(ctx, "scale", -0.2, 0.2, steps, q=qs, chunk=300)
    T = maps.grid("scale", -0.2, 0.2, steps, scale="offset")
    assert np.all(T[:, 6:9].min(axis=0) == np.float32(-0.2)) and np.all(T[:, 3:6] == 0)
    rng = np.random.default_rng(75)
    sample = rng.choice(len(T), 10, replace=False)
    mi_o, h_o, _ = _oracle_on_grid(f, m, 32, T[sample], qs, "euler", "offset")
    got = mp.reshape(-1, 2)[sample]
    assert np.all(np.abs(got - mi_o) <= 1e-6 * np.maximum(np.abs(mi_o), h_o[..., 2])), (got, mi_o)
    assert np.unravel_index(np.argmax(mp[..., 0]), mp.shape[:3]) == (5, 3, 6)
    assert maps.capture_fraction(mp[..., 0], (5, 3, 6)) > 0.3
