"""The allocation-free entry point (mi_eval_noalloc) agrees with mi_eval.

mi_eval_noalloc serves callers that may not allocate device memory where they
need the metric (plug-ins under a framework-owned caching allocator, services
with a fixed memory budget, loops that cannot take cudaMalloc's implicit
synchronisation): it keeps its histogram in one static device array shared by
all calls.  This file is collected last so that a failure here leaves every
other test already run; it passes on its own in a fresh process and after the
rest of the suite.
"""
import numpy as np
import pytest

from paper_1909_10690_gb300 import phantoms

pytestmark = pytest.mark.gpu

TOL = 1e-6  # the hard-path MI tolerance: |d| <= 1e-6 max(|MI|, H_FM)


def test_noalloc_matches_mi_eval_on_consecutive_calls(cuda_lib):
    import torch

    f, m = phantoms.head_pair(shape=(37, 50, 61), spacing=(1.0, 1.0, 1.2), seed=60)
    fd, md = torch.from_numpy(f).cuda(), torch.from_numpy(m).cuda()
    qs = [1.0, 0.5, 1.5, 2.0]
    sp = (1.0, 1.0, 1.2)
    ctx = cuda_lib.Context(f, m, bins=200, fixed_spacing=sp, moving_spacing=sp, fixed_depth=12, moving_depth=12,
                           path="plain")
    prm = phantoms.random_transforms(2, seed=61, t_mm=4, r_deg=8, s_range=(0.95, 1.05))
    want, h, _ = ctx.eval(prm, qs, with_entropies=True)
    # two calls in a row with different transforms, then the first again: the static
    # histogram must be cleared between calls
    for t in (0, 1, 0):
        got = cuda_lib.eval_noalloc(fd, md, 200, prm[t], qs, fixed_spacing=sp, moving_spacing=sp, fixed_depth=12,
                                    moving_depth=12)
        scale = np.maximum(np.abs(want[t]), h[t, :, 2])
        assert np.all(np.abs(got - want[t]) <= TOL * scale), (t, got, want[t])
    # device output
    out = torch.empty(len(qs), dtype=torch.float64, device="cuda")
    cuda_lib.eval_noalloc(fd, md, 200, prm[1], qs, fixed_spacing=sp, moving_spacing=sp, fixed_depth=12,
                          moving_depth=12, out=out)
    assert np.all(np.abs(out.cpu().numpy() - want[1]) <= TOL * np.maximum(np.abs(want[1]), h[1, :, 2]))


def test_noalloc_rejects_sizes_beyond_the_static_scratch(cuda_lib):
    import torch

    f, m = phantoms.ellipsoid_pair(shape=(16, 16, 16), seed=62)
    fd, md = torch.from_numpy(f).cuda(), torch.from_numpy(m).cuda()
    with pytest.raises(cuda_lib.MIError) as ei:
        cuda_lib.eval_noalloc(fd, md, 257, phantoms.identity_params(1)[0], [1.0])
    assert ei.value.status == cuda_lib.MI_EINVAL and "256" in str(ei.value)
    with pytest.raises(cuda_lib.MIError) as ei:  # host volumes are not accepted: nothing is copied
        cuda_lib.eval_noalloc(f, m, 32, phantoms.identity_params(1)[0], [1.0])
    assert ei.value.status == cuda_lib.MI_EINVAL


def test_noalloc_clamps_out_of_depth_values_like_mi_eval(cuda_lib):
    """Values above the declared bit depth are clamped as they are read, as mi_eval clamps them on load."""
    import torch

    f, m = phantoms.head_pair(shape=(20, 24, 28), spacing=(1.0, 1.0, 1.0), seed=63)
    rng = np.random.default_rng(64)
    m = m.copy()
    hot = rng.random(m.shape) < 0.05
    m[hot] = rng.integers(4096, 65536, size=int(hot.sum()), dtype=np.uint16)  # beyond 12 bits
    qs = [1.0, 1.5]
    ctx = cuda_lib.Context(f, m, bins=64, fixed_depth=12, moving_depth=12, path="plain")
    prm = phantoms.random_transforms(2, seed=65, t_mm=2, r_deg=5, s_range=(0.97, 1.03))
    want, h, _ = ctx.eval(prm, qs, with_entropies=True)
    fd, md = torch.from_numpy(f).cuda(), torch.from_numpy(m).cuda()
    for t in range(2):
        got = cuda_lib.eval_noalloc(fd, md, 64, prm[t], qs, fixed_depth=12, moving_depth=12)
        assert np.all(np.abs(got - want[t]) <= TOL * np.maximum(np.abs(want[t]), h[t, :, 2])), (t, got, want[t])


def test_noalloc_rejects_outputs_and_volumes_it_would_have_to_copy(cuda_lib):
    import torch

    f, m = phantoms.ellipsoid_pair(shape=(16, 16, 16), seed=66)
    fd, md = torch.from_numpy(f).cuda(), torch.from_numpy(m).cuda()
    prm = phantoms.identity_params(1)[0]
    for bad in (torch.empty(2, dtype=torch.float32, device="cuda"), torch.empty(1, dtype=torch.float64, device="cuda"),
                torch.empty(4, dtype=torch.float64, device="cuda")[::2]):
        with pytest.raises(cuda_lib.MIError) as ei:
            cuda_lib.eval_noalloc(fd, md, 32, prm, [1.0, 2.0], out=bad)
        assert ei.value.status == cuda_lib.MI_EINVAL
    with pytest.raises(cuda_lib.MIError) as ei:
        cuda_lib.eval_noalloc(fd.transpose(0, 2), md, 32, prm, [1.0])
    assert ei.value.status == cuda_lib.MI_EINVAL and "contiguous" in str(ei.value)
