"""Ascent paths on parameter-space maps (host post-processing of the metric maps of the Results)."""
import numpy as np

from paper_1909_10690_gb300 import maps


def _bowl(shape, c):
    i = np.indices(shape).astype(np.float64)
    return -sum((i[a] - c[a]) ** 2 for a in range(3))


def test_grid_order_and_identity_base():
    g = maps.grid("translation", -1, 1, 3)
    assert g.shape == (27, 9)
    np.testing.assert_array_equal(g[0, :3], [-1, -1, -1])
    np.testing.assert_array_equal(g[5, :3], [-1, 0, 1])  # C order, p0 slowest
    np.testing.assert_array_equal(g[:, 6:], 1)
    s = maps.grid("scale", -0.2, 0.2, 5, scale="offset")
    np.testing.assert_array_equal(s[:, :6], 0)
    np.testing.assert_allclose(s[-1, 6:], 0.2)
    r = maps.grid("rotation", -1, 1, 51)
    assert r.shape == (51 ** 3, 9) and np.allclose(r[51 ** 3 // 2, 3:6], 0)


def test_every_point_of_a_bowl_climbs_to_its_centre():
    m = _bowl((11, 9, 13), (3, 7, 5))
    sink, maxima = maps.ascent_sinks(m)
    assert list(maxima) == [np.ravel_multi_index((3, 7, 5), m.shape)]
    assert maps.capture_fraction(m, (3, 7, 5)) == 1.0
    path = maps.ascent_path(m, (10, 0, 12))
    vals = [m[p] for p in path]
    assert path[-1] == (3, 7, 5) and all(b > a for a, b in zip(vals, vals[1:]))
    # with one step covering one voxel per axis, the path takes max |offset| steps
    assert len(path) - 1 == max(abs(10 - 3), abs(0 - 7), abs(12 - 5))
    # minimisation of the negated map gives the same basins
    np.testing.assert_array_equal(maps.ascent_sinks(-m, maximize=False)[0], sink)


def test_two_maxima_split_the_map_at_the_valley():
    x = np.arange(11, dtype=np.float64)
    g = np.where(x <= 5, -(x - 2) ** 2, 2 - (x - 8) ** 2)  # maxima at 2 (0) and 8 (2), valley at 5
    h = -(np.arange(9, dtype=np.float64) - 4) ** 2
    k = -(np.arange(7, dtype=np.float64) - 3) ** 2
    m = g[:, None, None] + h[None, :, None] + k[None, None, :]
    sink, maxima = maps.ascent_sinks(m)
    a = np.ravel_multi_index((2, 4, 3), m.shape)
    b = np.ravel_multi_index((8, 4, 3), m.shape)
    assert sorted(maxima) == sorted([a, b])
    assert np.all(sink[:5] == a) and np.all(sink[6:] == b)
    # x = 5: g(4) = -4 against g(6) = -2, so the valley drains towards the higher maximum
    assert np.all(sink[5] == b)
    assert abs(maps.capture_fraction(m, (8, 4, 3)) - 6 / 11) < 1e-12


def test_nan_points_are_never_entered():
    m = _bowl((7, 7, 7), (3, 3, 3))
    m[3, 3, 3] = np.nan  # a failed evaluation at the peak: it counts as the worst value
    sink, maxima = maps.ascent_sinks(m)
    assert np.all(np.isfinite(m.ravel()[maxima]))
    assert np.all(sink != np.ravel_multi_index((3, 3, 3), m.shape))
