"""The batched path's autotune cache: a tuned shape is recorded in the file and replayed by a new
context of the same shape, a recorded choice that is no longer a candidate is ignored, and the
results do not depend on the choice."""
import numpy as np
import pytest

from paper_1909_10690_gb300 import phantoms

pytestmark = pytest.mark.gpu


def test_autotune_cache_records_and_replays(cuda_lib, tmp_path):
    path = tmp_path / "tune.txt"
    f, m = phantoms.head_pair(shape=(40, 48, 56), spacing=(1, 1, 1), seed=90)
    prm = phantoms.random_transforms(400, seed=91, t_mm=5, r_deg=10, s_range=(0.9, 1.1))
    qs = [1.0, 1.5]
    cuda_lib.autotune_cache(str(path))
    try:
        ctx = cuda_lib.Context(f, m, bins=64, fixed_depth=12, moving_depth=12, path="batched", block_threads=1024)
        want = ctx.eval(prm, qs)
        tuned = ctx.selected_config(len(prm))
        lines = path.read_text().splitlines()
        assert len(lines) == 1
        key, choice = lines[0].split("\t")
        assert int(choice.split()[0]) == tuned["variant"] and int(choice.split()[1]) == tuned["threads"]
        # a different, valid choice written for the same key is replayed by a fresh context ...
        other = 8 if tuned["variant"] != 8 else 2  # MI_HV_ROWS or MI_HV_U16 (x-pair loads, one row per step)
        # (1024-thread CTAs at 64 registers: one per SM whatever the variant, so the CTA count carries over)
        path.write_text(lines[0] + "\n" + f"{key}\t{other} 1024 {tuned['ctas']} 5 4\n")
        ctx2 = cuda_lib.Context(f, m, bins=64, fixed_depth=12, moving_depth=12, path="batched", block_threads=1024)
        got = ctx2.eval(prm, qs)
        cfg = ctx2.selected_config(len(prm))
        assert (cfg["variant"], cfg["threads"], cfg["tile_rows"], cfg["tile_slabs"]) == (other, 1024, 1, 4)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)
        # ... and a line naming no current candidate is ignored (the shape is tuned again and recorded)
        path.write_text(f"{key}\t99 1024 1 5 4\n")
        ctx3 = cuda_lib.Context(f, m, bins=64, fixed_depth=12, moving_depth=12, path="batched", block_threads=1024)
        np.testing.assert_allclose(ctx3.eval(prm, qs), want, rtol=0, atol=1e-12)
        assert ctx3.selected_config(len(prm))["variant"] != 99
        assert len(path.read_text().splitlines()) == 2
    finally:
        cuda_lib.autotune_cache(None)
