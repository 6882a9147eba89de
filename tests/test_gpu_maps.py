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
