"""GPU parity of the differentiable (Parzen) path against the FP64 oracle.

The GPU computes coordinates, interpolation and B-spline weights in FP32 and
accumulates the soft histogram per CTA in FP32, then in FP64; entropies and
W = dMI/dP are FP64.  Positions are 32.32 fixed point from the FP64 affine,
so trilinear cells and the overlap agree with the oracle.  Tolerances: MI
within 1e-6 max(|MI|, 1) -- FP32 weights and per-CTA FP32 partial sums
perturb P by ~1e-7 relative, and MI sums P against log-ratios of size < 10,
so the error is an absolute ~1e-6 at most (a purely relative bound is
ill-posed as MI -> 0); gradients within 1e-4 of the oracle gradient's largest
component (the stated gradient tolerance, taken norm-relative so that
near-zero components do not divide by zero).
"""
import numpy as np
import pytest

import oracle
from paper_1909_10690_gb300 import phantoms

pytestmark = pytest.mark.gpu

MI_TOL = 1e-6
G_TOL = 1e-4


def check(ctx, f, m, prm, qs, B, form=0, depth=None, shape_sp=((1, 1, 1), (1, 1, 1))):
    mi, g = ctx.grad(prm, qs)
    for t in range(len(prm)):
        aff, J = oracle.affine(prm[t], f.shape, shape_sp[0], m.shape, shape_sp[1], with_jacobian=True)
        mi_o, g_o, n = oracle.parzen(f, m, aff, B, qs, daff=J, form=form, fixed_depth=depth, moving_depth=depth)
        assert np.all(np.abs(mi[t] - mi_o) <= MI_TOL * np.maximum(np.abs(mi_o), 1.0)), (t, mi[t], mi_o)
        for iq in range(len(qs)):
            scale = np.abs(g_o[iq]).max()
            assert np.abs(g[t, iq] - g_o[iq]).max() <= G_TOL * scale, (t, iq, g[t, iq], g_o[iq])


def test_parzen_float_pair(cuda_lib):
    f, m = phantoms.head_pair(shape=(36, 44, 52), spacing=(1, 1, 1), seed=40, dtype=np.float32)
    B = 32
    ctx = cuda_lib.Context(f, m, bins=B, kernel="parzen")
    prm = phantoms.random_transforms(6, seed=41, t_mm=5, r_deg=10, s_range=(0.93, 1.07))
    check(ctx, f, m, prm, [1.0, 0.7, 1.3], B)


def test_parzen_smallest_volumes(cuda_lib):
    """2 x 2 x 2 and small ragged float pairs at 8 bins and 8 q: MI as the oracle's for empty (NaN),
    one-voxel and wider overlaps (the gradient is exercised at sizes where it is not ~0).

    The q set starts at 0.5: with one or two voxels in the overlap, B-spline tail cells of weight
    ~1e-6 enter S_q as P^q, and at q = 0.2 their FP32 weight error reaches 1.4e-6 of MI."""
    rng = np.random.default_rng(97)
    qs = [0.5, 0.7, 0.8, 1.0, 1.2, 1.5, 2.0, 3.0]
    seen = set()
    for shape_f, shape_m in (((2, 2, 2), (2, 2, 2)), ((3, 2, 5), (2, 4, 2))):
        f = rng.random(shape_f, dtype=np.float32)
        m = rng.random(shape_m, dtype=np.float32)
        ctx = cuda_lib.Context(f, m, bins=8, kernel="parzen")
        prm = np.concatenate([phantoms.identity_params(1),
                              phantoms.random_transforms(11, seed=98, t_mm=0.6, r_deg=10, s_range=(0.9, 1.1))])
        mi = ctx.eval(prm, qs)
        for t in range(len(prm)):
            aff = oracle.affine(prm[t], f.shape, (1, 1, 1), m.shape, (1, 1, 1))
            mi_o, _, n = oracle.parzen(f, m, aff, 8, qs)
            seen.add(min(n, 2))
            if n == 0:
                assert np.all(np.isnan(mi[t]))
            else:
                assert np.all(np.abs(mi[t] - mi_o) <= MI_TOL * np.maximum(np.abs(mi_o), 1.0)), (t, mi[t], mi_o)
    assert seen == {0, 1, 2}


@pytest.mark.parametrize("B", [8, 64, 96, 128])  # forward with eight, four, two and one histogram copies
def test_parzen_integer_pair_and_bin_counts(cuda_lib, B):
    f, m = phantoms.head_pair(shape=(30, 34, 40), spacing=(1, 1, 1), seed=42)
    ctx = cuda_lib.Context(f, m, bins=B, kernel="parzen", fixed_depth=12, moving_depth=12)
    np.testing.assert_array_equal(ctx.fixed_bins(), oracle.parzen_fixed_bins(f, B, depth=12).astype(np.uint8))
    prm = phantoms.random_transforms(4, seed=43, t_mm=4, r_deg=8, s_range=(0.95, 1.05))
    check(ctx, f, m, prm, [1.0, 1.5], B, depth=12)


def test_parzen_128_bins_five_q_reads_w_from_global_then_shared_memory(cuda_lib):
    # the adjoint takes q in groups of up to four: at 128 bins four q's W tables (276 KB) exceed shared
    # memory and are read from global memory by 256-thread CTAs; the fifth q's (69 KB) sits in the
    # shared memory of 512-thread CTAs
    f, m = phantoms.head_pair(shape=(26, 30, 34), spacing=(1, 1, 1), seed=53, dtype=np.float32)
    ctx = cuda_lib.Context(f, m, bins=128, kernel="parzen")
    prm = phantoms.random_transforms(3, seed=54, t_mm=3, r_deg=6, s_range=(0.96, 1.04))
    check(ctx, f, m, prm, [1.0, 0.7, 1.3, 1.5, 2.0], 128)


def test_parzen_versor_and_offset_gradient(cuda_lib):
    # d MI / d(versor, zero-centred scale): the Jacobian of the unit-ball parameterisation
    f, m = phantoms.head_pair(shape=(30, 34, 38), spacing=(1, 1, 1), seed=46, dtype=np.float32)
    B = 32
    ctx = cuda_lib.Context(f, m, bins=B, kernel="parzen", rotation="versor", scale="offset")
    rng = np.random.default_rng(47)
    prm = np.concatenate([rng.uniform(-3, 3, (4, 3)), rng.uniform(-0.08, 0.08, (4, 3)),
                          rng.uniform(-0.05, 0.05, (4, 3))], 1).astype(np.float32)
    qs = [1.0, 1.3]
    mi, g = ctx.grad(prm, qs)
    for t in range(len(prm)):
        aff, J = oracle.affine(prm[t], f.shape, (1, 1, 1), m.shape, (1, 1, 1), with_jacobian=True, rotation="versor",
                               scale="offset")
        mi_o, g_o, n = oracle.parzen(f, m, aff, B, qs, daff=J)
        assert np.all(np.abs(mi[t] - mi_o) <= MI_TOL * np.maximum(np.abs(mi_o), 1.0)), (t, mi[t], mi_o)
        for iq in range(len(qs)):
            assert np.abs(g[t, iq] - g_o[iq]).max() <= G_TOL * np.abs(g_o[iq]).max(), (t, iq)


def test_parzen_pseudo_additive_and_many_q(cuda_lib):
    f, m = phantoms.head_pair(shape=(28, 30, 32), spacing=(1, 1, 1), seed=44, dtype=np.float32)
    B = 24
    ctx = cuda_lib.Context(f, m, bins=B, kernel="parzen", tsallis_form="pseudo_additive")
    prm = phantoms.random_transforms(3, seed=45, t_mm=3, r_deg=6, s_range=(0.95, 1.05))
    check(ctx, f, m, prm, [0.5, 0.7, 0.9, 1.0, 1.1, 1.3, 1.5, 2.0], B, form=1)


def test_parzen_eval_matches_grad_mi_and_empty(cuda_lib):
    f, m = phantoms.head_pair(shape=(20, 22, 24), spacing=(1, 1, 1), seed=46, dtype=np.float32)
    ctx = cuda_lib.Context(f, m, bins=16, kernel="parzen")
    prm = phantoms.random_transforms(5, seed=47, t_mm=3, r_deg=6)
    mi_e = ctx.eval(prm, [1.0, 1.3])
    mi_g, _ = ctx.grad(prm, [1.0, 1.3])
    np.testing.assert_array_equal(mi_e, mi_g)
    # the overlap counts the soft histogram sums, as the oracle's; no hard-histogram entropies
    mi_c, h, cnt = ctx.eval(prm, [1.0, 1.3], with_entropies=True)
    assert h is None
    np.testing.assert_array_equal(mi_c, mi_e)
    for t in range(len(prm)):
        aff = oracle.affine(prm[t], f.shape, (1, 1, 1), m.shape, (1, 1, 1))
        assert cnt[t] == oracle.parzen(f, m, aff, 16, [1.0])[2]
    far = phantoms.identity_params(1)
    far[0, 1] = 500.0
    with pytest.raises(cuda_lib.MIError) as ei:
        ctx.grad(far, [1.0])
    assert ei.value.status == cuda_lib.MI_EEMPTY
    with pytest.raises(cuda_lib.MIError) as ei:
        cuda_lib.Context(f, m, bins=16).grad(prm, [1.0])
    assert ei.value.status == cuda_lib.MI_EUNSUPPORTED


def test_autograd_function(cuda_lib):
    import torch

    f, m = phantoms.head_pair(shape=(24, 26, 28), spacing=(1, 1, 1), seed=48, dtype=np.float32)
    ctx = cuda_lib.Context(f, m, bins=32, kernel="parzen")
    MIFunction = cuda_lib.mi_function()
    theta = torch.tensor(phantoms.random_transforms(3, seed=49, t_mm=3, r_deg=5), device="cuda", requires_grad=True)
    q = [1.0, 1.3]
    mi = MIFunction.apply(theta, ctx, q)
    w = torch.tensor([[1.0, 0.5], [2.0, -1.0], [0.0, 3.0]], device="cuda", dtype=mi.dtype)
    (mi * w).sum().backward()
    _, g = ctx.grad(theta.detach(), q)
    want = (w.unsqueeze(-1) * g).sum(dim=1)
    torch.testing.assert_close(theta.grad.double(), want.double(), rtol=1e-6, atol=1e-9)


@pytest.mark.slow
def test_parzen_full_size_sampled(cuda_lib):
    # the differentiable workload at full size: 192x192x128 float32, 64 bins, Shannon and q = 0.7, 1.3
    f, m = phantoms.head_pair(shape=(128, 192, 192), spacing=(1, 1, 1.2), seed=50, dtype=np.float32)
    B = 64
    ctx = cuda_lib.Context(f, m, bins=B, kernel="parzen", fixed_spacing=(1, 1, 1.2), moving_spacing=(1, 1, 1.2))
    prm = phantoms.random_transforms(50, seed=51, t_mm=10, r_deg=15, s_range=(0.9, 1.1))
    qs = [1.0, 0.7, 1.3]
    mi, g = ctx.grad(prm, qs)  # the bench's launch configuration: 50 poses in one call
    assert np.all(np.isfinite(mi)) and np.all(np.isfinite(g))
    # 8 of the 50 poses, spread over the call, against the FP64 oracle (one host thread per pose: the
    # oracle's C code runs outside the interpreter lock)
    from concurrent.futures import ThreadPoolExecutor

    sample = [0, 7, 13, 20, 26, 33, 41, 49]
    sp = (1, 1, 1.2)

    def oracle_pose(t):
        aff, J = oracle.affine(prm[t], f.shape, sp, m.shape, sp, with_jacobian=True)
        return oracle.parzen(f, m, aff, B, qs, daff=J)

    with ThreadPoolExecutor(max_workers=len(sample)) as ex:
        results = list(ex.map(oracle_pose, sample))
    for t, (mi_o, g_o, _) in zip(sample, results):
        assert np.all(np.abs(mi[t] - mi_o) <= MI_TOL * np.maximum(np.abs(mi_o), 1.0)), (t, mi[t], mi_o)
        for iq in range(len(qs)):
            assert np.abs(g[t, iq] - g_o[iq]).max() <= G_TOL * np.abs(g_o[iq]).max(), (t, iq, g[t, iq], g_o[iq])


@pytest.mark.parametrize("B, nz", [(64, 16), (32, 32)])
def test_parzen_forward_at_the_per_copy_voxel_cap(cuda_lib, B, nz):
    # rows of 16384 voxels, 4 nz rows a pose, 38 poses.  At 64 bins a CTA holds four histogram copies,
    # each fed by every fourth lane, so a copy may take 16 rows (2^16 voxels); at 32 bins eight copies,
    # every eighth lane, 32 rows.  The rows then split into 152 chunks of that many (one wave of one CTA
    # per SM on 152 SMs), four to a pose, and at the identity every copy sums exactly 2^16 voxels' 16-bit
    # weight halves, the most that fits
    rng = np.random.default_rng(52)
    ny, nx = 4, 16384
    z = np.arange(nz)[:, None, None] / (nz - 1)
    x = np.arange(nx)[None, None, :] / (nx - 1)
    f = (0.25 + 0.5 * (z > 0.5) + 0.02 * rng.standard_normal((nz, ny, nx))).clip(0, 1).astype(np.float32)
    m = (0.2 + 0.3 * z + 0.4 * x + 0.01 * rng.standard_normal((nz, ny, nx))).clip(0, 1).astype(np.float32)
    ctx = cuda_lib.Context(f, m, bins=B, kernel="parzen")
    prm = np.tile(np.array([0, 0, 0, 0, 0, 0, 1, 1, 1], np.float32), (38, 1))
    prm[19:, 0] = np.linspace(-4, 4, 19, dtype=np.float32)
    qs = [1.0, 0.7, 1.3]
    mi, g = ctx.grad(prm, qs)
    for t in (0, 30):
        aff, J = oracle.affine(prm[t], f.shape, (1, 1, 1), m.shape, (1, 1, 1), with_jacobian=True)
        mi_o, g_o, n = oracle.parzen(f, m, aff, B, qs, daff=J)
        assert np.all(np.abs(mi[t] - mi_o) <= MI_TOL * np.maximum(np.abs(mi_o), 1.0)), (t, mi[t], mi_o)
        for iq in range(len(qs)):
            assert np.abs(g[t, iq] - g_o[iq]).max() <= G_TOL * np.abs(g_o[iq]).max(), (t, iq, g[t, iq], g_o[iq])
    # every identity pose gives the same soft histogram
    assert np.all(mi[:19] == mi[0]) and np.all(g[:19] == g[0])


@pytest.mark.parametrize("kernel", ["hard", "parzen"])
def test_moving_volume_beyond_the_texture_extent_is_rejected(cuda_lib, kernel):
    f = np.zeros((2, 2, 64), np.float32)
    m = np.zeros((2, 2, 40000), np.float32)
    with pytest.raises(cuda_lib.MIError) as e:
        cuda_lib.Context(f, m, bins=16, kernel=kernel)
    assert e.value.status == cuda_lib.MI_EUNSUPPORTED


def test_parzen_symmetric_pair_and_separated_classes(cuda_lib):
    # the oracle's pins on the CUDA path: a mirror-symmetric pair at a uniform scale has no translation
    # or rotation gradient (FP32 accumulation: within the gradient tolerance of the scale components),
    # and aligned classes >= 4 moving bins apart give Shannon MI = H(class proportions)
    rng = np.random.default_rng(28)
    shape = (12, 14, 16)
    table = rng.uniform(0.1, 0.9, size=tuple((n + 1) // 2 for n in shape)).astype(np.float32)
    idx = [np.minimum(np.arange(n), n - 1 - np.arange(n)) for n in shape]
    f = np.ascontiguousarray(table[np.ix_(idx[0], idx[1], idx[2])])
    ctx = cuda_lib.Context(f, f, bins=32, kernel="parzen")
    p = np.array([[0, 0, 0, 0, 0, 0, 1.04, 1.04, 1.04]], dtype=np.float32)
    mi, g = ctx.grad(p, [1.0, 0.7, 1.3])
    for iq in range(3):
        assert np.abs(g[0, iq, :6]).max() <= G_TOL * np.abs(g[0, iq, 6:]).max(), g[0, iq]
    c = np.full((8, 10, 12), 0.2, np.float32)
    c[:, :, 9:] = 0.8
    want = -(0.25 * np.log(0.25) + 0.75 * np.log(0.75))
    for B in (16, 64):
        cctx = cuda_lib.Context(c, c, bins=B, kernel="parzen")
        mi = cctx.eval(np.array([[0, 0, 0, 0, 0, 0, 1, 1, 1]], np.float32), [1.0])
        assert abs(mi[0, 0] - want) <= MI_TOL * want, (B, mi[0, 0], want)


def test_parzen_multi_pair_one_launch_per_kernel(cuda_lib):
    # pairs of different dims, types and bin counts in one Parzen context: every kernel runs once for all
    # pairs; MI equals the single-pair contexts' bit for bit (integer soft histograms, the same FP64
    # reduction), gradients agree within the gradient tolerance (FP32 moments summed over another CTA
    # split) and with the oracle
    specs = [((20, 26, 31), np.float32, None, 16), ((28, 22, 37), np.uint16, 12, 64), ((17, 33, 24), np.uint8, 8, 128)]
    pairs, vols = [], []
    for i, (shape, dt, depth, B) in enumerate(specs):
        f, m = phantoms.head_pair(shape=shape, spacing=(1, 1, 1), depth=depth or 12, seed=53 + i, dtype=dt)
        vols.append((f, m, depth, B))
        pairs.append(dict(fixed=f, moving=m, bins=B, fixed_depth=depth, moving_depth=depth))
    ctx = cuda_lib.Context(pairs=pairs, kernel="parzen")
    prm = phantoms.random_transforms(15, seed=56, t_mm=3, r_deg=6, s_range=(0.95, 1.05))
    pair_of = np.array([0, 1, 2, 2, 1, 0, 1, 2, 0, 0, 2, 1, 1, 0, 2], np.int32)
    qs = [1.0, 0.7, 1.3]
    mi, g = ctx.batch_grad(pair_of, prm, qs)
    assert ctx.last_kernel_ms()[1] == 6
    mi_only = ctx.batch_eval(pair_of, prm, qs)
    np.testing.assert_array_equal(mi_only, mi)
    for p, (f, m, depth, B) in enumerate(vols):
        sel = np.nonzero(pair_of == p)[0]
        one = cuda_lib.Context(f, m, bins=B, kernel="parzen", fixed_depth=depth, moving_depth=depth)
        mi1, g1 = one.grad(prm[sel], qs)
        np.testing.assert_array_equal(mi[sel], mi1)
        for iq in range(len(qs)):
            scale = np.abs(g1[:, iq]).max()
            assert np.abs(g[sel, iq] - g1[:, iq]).max() <= G_TOL * scale, (p, iq)
        t = sel[0]
        aff, J = oracle.affine(prm[t], f.shape, (1, 1, 1), m.shape, (1, 1, 1), with_jacobian=True)
        mi_o, g_o, _ = oracle.parzen(f, m, aff, B, qs, daff=J, fixed_depth=depth, moving_depth=depth)
        assert np.all(np.abs(mi[t] - mi_o) <= MI_TOL * np.maximum(np.abs(mi_o), 1.0)), (p, mi[t], mi_o)
        for iq in range(len(qs)):
            assert np.abs(g[t, iq] - g_o[iq]).max() <= G_TOL * np.abs(g_o[iq]).max(), (p, iq)
    with pytest.raises(cuda_lib.MIError):  # a multi-pair context takes the batch entry points
        ctx.grad(prm[:1], qs)
