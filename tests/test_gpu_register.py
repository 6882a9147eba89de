"""Registration by gradient ascent on the Parzen MI, and the gradient against
finite differences at full size (Eq. 3; the Discussion's mixed entropies).

The analytic gradient is the exact derivative of the piecewise-smooth MI
(trilinear interpolation has a derivative jump wherever a sample crosses a
grid plane of the moving volume).  A central difference of step h is the
mean of that derivative over [theta - h, theta + h], not its value at theta:
a scale step of 1e-3 moves samples 96 mm from the centre by 0.1 mm, and the
pointwise gap then reaches ~100 % of the gradient.  The comparison with
central differences is therefore made against the segment mean of the
analytic gradient.
"""
import numpy as np
import pytest

import oracle

from paper_1909_10690_gb300 import phantoms, register

pytestmark = pytest.mark.gpu

SP = (1.0, 1.0, 1.2)


@pytest.fixture(scope="module")
def head(cuda_lib):
    f, m = phantoms.head_pair(shape=(128, 192, 192), spacing=SP, seed=50, dtype=np.float32)
    return f, m


@pytest.mark.parametrize("q, q_t", [(1.0, None), (1.0, 1.5), (1.0, 2.0)], ids=["shannon", "mixed_t1.5", "mixed_t2"])
def test_registration_recovers_motion(cuda_lib, head, q, q_t):
    f, m = head
    ctx = cuda_lib.Context(f, m, bins=64, kernel="parzen", fixed_spacing=SP, moving_spacing=SP)
    truth = np.array(phantoms.HEAD_MOTION)
    rng = np.random.default_rng(7)
    n = 20
    d = np.concatenate([rng.uniform(-10, 10, (n, 3)), rng.uniform(-15, 15, (n, 3)), rng.uniform(-0.1, 0.1, (n, 3))], 1)
    theta, hist = register.register(ctx, truth[None] + d, q=q, q_translation=q_t, steps=200)
    et, er, es = register.pose_error(theta, truth)
    ok = (et < 1.0) & (er < 1.0) & (es < 0.01)
    assert ok.all(), (et, er, es)
    assert np.all(hist[-1] > hist[0])


def test_central_differences_equal_the_mean_gradient(cuda_lib, head):
    """Central differences at h = 1e-3 on 50 random poses, 9 parameters, 3 q.

    MI is continuous along theta + t e_k when the overlap is constant (a crop
    of the fixed volume keeps every sample inside the moving volume for these
    poses), so (MI(theta + h e_k) - MI(theta - h e_k)) / 2h is exactly the
    mean of dMI/dtheta_k over the segment.  The test forms that mean with an
    n-node midpoint rule of the analytic gradient and requires agreement
    within 1e-4 of the largest gradient component.  The derivative jumps
    wherever samples cross grid planes (its total variation along a scale
    segment is ~20 times its size), so the rule needs n = 8192 nodes on the
    scale parameters (measured gap ~1e-5; 8.7e-5 at n = 4096, 6e-4 at 256)
    and n = 256 on the rest (measured ~2e-5).  For two of the poses the differences are also taken of
    the FP64 oracle's MI, so that the check does not rest on the GPU's MI alone.
    """
    f, m = head
    fc = np.ascontiguousarray(f[24:104, 32:160, 32:160])
    ctx = cuda_lib.Context(fc, m, bins=64, kernel="parzen", fixed_spacing=SP, moving_spacing=SP)
    P = 50
    prm = phantoms.random_transforms(P, seed=53, t_mm=5, r_deg=5, s_range=(0.95, 1.05)).astype(np.float64)
    qs = [1.0, 0.7, 1.3]
    h = 1e-3
    _, g0 = ctx.grad(prm.astype(np.float32), qs)
    assert np.all(np.isfinite(g0))
    scale = np.abs(g0).max(-1)  # per pose and q
    for k in range(9):
        n = 8192 if k >= 6 else 256
        pp = prm.copy()
        pm = prm.copy()
        pp[:, k] += h
        pm[:, k] -= h
        a32, b32 = pm.astype(np.float32), pp.astype(np.float32)
        a, b = a32[:, k].astype(np.float64), b32[:, k].astype(np.float64)
        fd = (ctx.eval(b32, qs) - ctx.eval(a32, qs)) / (b - a)[:, None]
        gsum = np.zeros((P, len(qs)))
        chunk = min(512, n)
        for j0 in range(0, n, chunk):
            nodes = np.repeat(prm[:, None, :], chunk, 1)
            nodes[:, :, k] = a[:, None] + (np.arange(j0, j0 + chunk)[None, :] + 0.5) * ((b - a) / n)[:, None]
            _, gn = ctx.grad(nodes.reshape(-1, 9).astype(np.float32), qs)
            gsum += gn.reshape(P, chunk, len(qs), 9)[:, :, :, k].sum(1)
        gap = np.abs(fd - gsum / n) / scale
        assert gap.max() <= 1e-4, (k, gap.max())
        # and independently of the GPU's MI: differences of the FP64 oracle's MI at the same endpoints
        for t in (0, 25):
            mo = [oracle.parzen(fc, m, oracle.affine(e[t], fc.shape, SP, m.shape, SP), 64, qs)[0] for e in (a32, b32)]
            fd_o = (mo[1] - mo[0]) / (b[t] - a[t])
            assert np.all(np.abs(fd_o - gsum[t] / n) <= 1e-4 * scale[t]), (k, t, fd_o, gsum[t] / n)


@pytest.mark.parametrize("q, q_t", [(1.0, None), (1.0, 1.5)], ids=["shannon", "mixed_t1.5"])
def test_kiefer_wolfowitz_recovers_motion_on_the_hard_metric(cuda_lib, q, q_t):
    """Kiefer-Wolfowitz on the hard-binned MI (Eq. 2; the Introduction's stochastic approximation):
    each iteration is one batched evaluation of 18 perturbations for each of the 16 poses.

    The fixed volume is a centred crop (same centre, so the same transform) that stays inside the
    moving volume near the solution.  Over the whole field of view the overlap shrinks as the
    rotation grows, and with background the largest class plain MI rises as background leaves the
    overlap: its maximum there sits up to ~5 degrees beyond the true angles."""
    f, m = phantoms.head_pair(shape=(128, 192, 192), spacing=SP, seed=50)
    fc = np.ascontiguousarray(f[16:112, 24:168, 24:168])
    ctx = cuda_lib.Context(fc, m, bins=64, fixed_spacing=SP, moving_spacing=SP, fixed_depth=12, moving_depth=12)
    truth = np.array(phantoms.HEAD_MOTION)
    rng = np.random.default_rng(8)
    n = 16
    d = np.concatenate([rng.uniform(-8, 8, (n, 3)), rng.uniform(-10, 10, (n, 3)), rng.uniform(-0.08, 0.08, (n, 3))], 1)
    theta, hist = register.register_kw(ctx, truth[None] + d, q=q, q_translation=q_t, steps=200)
    et, er, es = register.pose_error(theta, truth)
    ok = (et < 0.5) & (er < 0.75) & (es < 0.005)  # measured: 0.19 mm, 0.39 deg, 0.0022
    assert ok.all(), (et, er, es)
    assert np.all(hist[-1] > hist[0])
