"""GPU parity of the general 12-parameter affine [M | t] (the Methodology's 12 degrees of freedom).

The transform builder is host code compiled into the CUDA library; it must
give the oracle's FP64 [A | b] bit for bit, so the 16.16 matrices, the hard
histograms and the overlap counts are exact.  MI is within the hard path's
1e-6 of max(|MI|, H_FM); Parzen MI and the 12-component gradient within the
Parzen tolerances (1e-6 absolute-or-relative MI, 1e-4 of the largest gradient
component).
"""
import numpy as np
import pytest

import oracle
from paper_1909_10690_gb300 import phantoms

pytestmark = pytest.mark.gpu

TOL = 1e-6
G_TOL = 1e-4


def random_affines(n, seed, lin=0.12, t_mm=4.0):
    """[M | t] with M = a random rotation-and-scale motion plus a random skew part, t in mm."""
    rng = np.random.default_rng(seed)
    prm = phantoms.random_transforms(n, seed=seed, t_mm=t_mm, r_deg=12, s_range=(0.9, 1.1))
    out = np.empty((n, 12), np.float32)
    for k in range(n):
        L, t = phantoms.motion_matrix(prm[k].astype(np.float64))
        M = L + rng.uniform(-lin, lin, (3, 3)) * (1 - np.eye(3))
        out[k] = np.hstack([M, t.reshape(3, 1)]).astype(np.float32).ravel()
    return out


def test_affine12_builder_matches_oracle_bit_for_bit(cuda_lib):
    f = np.zeros((20, 24, 30), np.uint16)
    m = np.zeros((22, 28, 26), np.uint16)
    sf, sm = (1.0, 0.875, 1.25), (1.125, 1.0, 1.375)
    ctx = cuda_lib.Context(f, m, bins=16, fixed_spacing=sf, moving_spacing=sm, transform="affine")
    assert ctx.nparams == 12
    T = random_affines(2000, seed=60, lin=0.5, t_mm=30)
    a, q, j = ctx.affine(T)
    assert j.shape == (2000, 12, 12)
    for t in range(len(T)):
        ao, jo = oracle.affine(T[t], f.shape, sf, m.shape, sm, with_jacobian=True, transform="affine")
        np.testing.assert_array_equal(a[t], ao)
        np.testing.assert_array_equal(q[t], oracle.affine_q16(ao))
        np.testing.assert_allclose(j[t], jo, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("path", ["plain", "batched"])
def test_affine12_histograms_and_mi_parity(cuda_lib, path):
    f, m = phantoms.head_pair(shape=(40, 44, 48), spacing=(1, 1, 1.2), seed=61)
    sp = (1, 1, 1.2)
    ctx = cuda_lib.Context(f, m, bins=64, fixed_depth=12, moving_depth=12, fixed_spacing=sp, moving_spacing=sp,
                           transform="affine", path=path)
    T = random_affines(16, seed=62)
    qs = [1.0, 0.5, 1.5]
    mi, h, cnt = ctx.eval(T, qs, with_entropies=True)
    q16 = np.stack([oracle.affine_q16(oracle.affine(p, f.shape, sp, m.shape, sp, transform="affine")) for p in T])
    mi_o, h_o, cnt_o = oracle.mi_eval_q16(f, m, 64, q16, qs, fixed_depth=12, moving_depth=12, nthreads=8)
    np.testing.assert_array_equal(cnt, cnt_o)
    scale = np.maximum(np.abs(mi_o), h_o[..., 2])
    assert np.all(np.abs(mi - mi_o) <= TOL * scale)
    H = ctx.hist(transforms=T[:4], path=cuda_lib.PATH_BATCHED if path == "batched" else cuda_lib.PATH_PLAIN)
    for k in range(4):
        ho, _ = oracle.joint_hist(f, m, q16[k], 64, 12, 12)
        np.testing.assert_array_equal(H[k], ho.astype(np.uint32))


def test_affine12_integer_shear_is_exact_on_gpu(cuda_lib):
    # x' = x + (y - c_y): integer coordinates, so the resampled volume is a row-wise shift of the moving one
    rng = np.random.default_rng(63)
    f = rng.integers(0, 4096, size=(7, 9, 13), dtype=np.uint16)
    m = rng.integers(0, 4096, size=(7, 9, 13), dtype=np.uint16)
    ctx = cuda_lib.Context(f, m, bins=32, fixed_depth=12, moving_depth=12, transform="affine")
    T = np.array([[1, 1, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0]], np.float32)
    _, q, _ = ctx.affine(T)
    out = ctx.resample(q[0], np.uint16)
    cy = 4
    for j in range(9):
        for i in range(13):
            src = i + (j - cy)
            want = m[:, j, src] if 0 <= src < 13 else np.zeros(7, np.uint16)
            np.testing.assert_array_equal(out[:, j, i], want)


def test_affine12_uneven_batch(cuda_lib):
    specs = [((30, 36, 40), np.uint8, 8, 32), ((34, 28, 44), np.uint16, 12, 64), ((26, 40, 31), np.uint16, 12, 128)]
    pairs, vols = [], []
    for i, (shape, dt, depth, bins) in enumerate(specs):
        f, m = phantoms.head_pair(shape=shape, spacing=(1, 1, 1), depth=depth, seed=64 + i, dtype=dt)
        vols.append((f, m, depth, bins))
        pairs.append(dict(fixed=f, moving=m, bins=bins, fixed_depth=depth, moving_depth=depth))
    ctx = cuda_lib.Context(pairs=pairs, transform="affine")
    T = random_affines(30, seed=67)
    pair_of = np.arange(30, dtype=np.int32) % 3
    qs = [1.0, 2.0]
    mi, h, cnt = ctx.batch_eval(pair_of, T, qs, with_entropies=True)
    for p, (f, m, depth, bins) in enumerate(vols):
        sel = np.nonzero(pair_of == p)[0]
        q16 = np.stack([oracle.affine_q16(oracle.affine(T[t], f.shape, (1, 1, 1), m.shape, (1, 1, 1),
                                                        transform="affine")) for t in sel])
        mi_o, h_o, cnt_o = oracle.mi_eval_q16(f, m, bins, q16, qs, fixed_depth=depth, moving_depth=depth, nthreads=8)
        np.testing.assert_array_equal(cnt[sel], cnt_o)
        assert np.all(np.abs(mi[sel] - mi_o) <= TOL * np.maximum(np.abs(mi_o), h_o[..., 2]))


def test_affine12_parzen_gradient(cuda_lib):
    f, m = phantoms.head_pair(shape=(30, 34, 38), spacing=(1, 1, 1), seed=68, dtype=np.float32)
    B = 32
    ctx = cuda_lib.Context(f, m, bins=B, kernel="parzen", transform="affine")
    T = random_affines(4, seed=69, lin=0.08, t_mm=3)
    qs = [1.0, 0.7, 1.3]
    mi, g = ctx.grad(T, qs)
    assert g.shape == (4, 3, 12)
    for t in range(len(T)):
        aff, J = oracle.affine(T[t], f.shape, (1, 1, 1), m.shape, (1, 1, 1), with_jacobian=True, transform="affine")
        mi_o, g_o, n = oracle.parzen(f, m, aff, B, qs, daff=J)
        assert np.all(np.abs(mi[t] - mi_o) <= TOL * np.maximum(np.abs(mi_o), 1.0)), (t, mi[t], mi_o)
        for iq in range(len(qs)):
            assert np.abs(g[t, iq] - g_o[iq]).max() <= G_TOL * np.abs(g_o[iq]).max(), (t, iq, g[t, iq], g_o[iq])


def test_affine12_autograd(cuda_lib):
    import torch

    f, m = phantoms.head_pair(shape=(24, 26, 28), spacing=(1, 1, 1), seed=70, dtype=np.float32)
    ctx = cuda_lib.Context(f, m, bins=32, kernel="parzen", transform="affine")
    MIFunction = cuda_lib.mi_function()
    theta = torch.tensor(random_affines(2, seed=71, lin=0.05, t_mm=2), device="cuda", requires_grad=True)
    mi = MIFunction.apply(theta, ctx, [1.0])
    mi.sum().backward()
    _, g = ctx.grad(theta.detach(), [1.0])
    torch.testing.assert_close(theta.grad.double(), g[:, 0].double(), rtol=1e-6, atol=1e-9)


def test_affine12_singular_and_reflection(cuda_lib):
    rng = np.random.default_rng(72)
    f = rng.integers(0, 4096, size=(21, 23, 25), dtype=np.uint16)
    m = rng.integers(0, 4096, size=(21, 23, 25), dtype=np.uint16)
    T = np.array([[0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0],              # M = 0: every voxel samples the centre
                  [-1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0],             # mirror x
                  [1, 0, 0, 0, 0, -1, 0, 0, 0, 0, -1, 0],            # half turn about x (det +1)
                  [0, 0, 0, 2.5, 0, 1, 0, -1, 0, 0, 1, 0.5]], np.float32)  # rank 2, shifted
    qs = [1.0, 0.5]
    for path in ("plain", "batched"):
        ctx = cuda_lib.Context(f, m, bins=32, fixed_depth=12, moving_depth=12, transform="affine", path=path)
        mi, h, cnt = ctx.eval(T, qs, with_entropies=True)
        q16 = np.stack([oracle.affine_q16(oracle.affine(p, f.shape, (1, 1, 1), m.shape, (1, 1, 1),
                                                        transform="affine")) for p in T])
        mi_o, h_o, cnt_o = oracle.mi_eval_q16(f, m, 32, q16, qs, fixed_depth=12, moving_depth=12)
        np.testing.assert_array_equal(cnt, cnt_o)
        assert np.all(np.abs(mi - mi_o) <= TOL * np.maximum(np.abs(mi_o), h_o[..., 2]))
        H = ctx.hist(transforms=T, path=cuda_lib.PATH_BATCHED if path == "batched" else cuda_lib.PATH_PLAIN)
        for k in range(len(T)):
            ho, _ = oracle.joint_hist(f, m, q16[k], 32, 12, 12)
            np.testing.assert_array_equal(H[k], ho.astype(np.uint32))
    # M = 0: one moving bin, so the moving and joint entropies equal H(F) and H(M) = 0: MI = 0
    np.testing.assert_allclose(mi[0], 0.0, atol=1e-12)
