"""GPU parity of the hard-binned path against the CPU oracle.

Joint histograms must match bit for bit; MI and entropies within
|d| <= 1e-6 max(|MI|, H_FM) (both sides sum exact counts in FP64, so the
observed gap is summation order, ~1e-13).
"""

import numpy as np
import pytest

import hand_cases
import oracle
from paper_1909_10690_gb300 import phantoms

pytestmark = pytest.mark.gpu

TOL = 1e-6
VARIANTS = list(range(16))  # MI_HV_U32 .. MI_HV_U16_GATHER
U32_VARIANTS = (0, 1, 4, 5, 11, 14)  # one 32-bit counter per cell: at most 181 bins in shared memory
IDENT = np.array([65536, 0, 0, 0, 0, 65536, 0, 0, 0, 0, 65536, 0], dtype=np.int32)


# absolute floor: where the whole overlap falls in one cell, H_FM = 0 and MI is exactly 0 (Eq. 2);
# both sides then return FP64 rounding of entropies of a few nats (~1e-16)
MI_FLOOR = 1e-12


def assert_mi_close(mi_gpu, mi_ref, h_ref):
    scale = np.maximum(np.abs(mi_ref), h_ref[..., 2])
    bad = np.abs(mi_gpu - mi_ref) > TOL * scale + MI_FLOOR
    assert not np.any(bad), (mi_gpu[bad], mi_ref[bad])


def random_q16(shape_f, shape_m, n, seed, t=4.0, r=15.0, s=(0.9, 1.1)):
    prm = phantoms.random_transforms(n, seed=seed, t_mm=t, r_deg=r, s_range=s)
    return prm, np.stack([oracle.affine_q16(oracle.affine(p, shape_f, (1, 1, 1), shape_m, (1, 1, 1))) for p in prm])


@pytest.fixture(scope="module")
def tiny_pair():
    return phantoms.ellipsoid_pair(shape=(64, 64, 64), seed=1)


def test_fixed_bins_and_resample_bit_exact(cuda_lib):
    f, m = phantoms.head_pair(shape=(33, 45, 67), spacing=(1, 1, 1), seed=3)
    ctx = cuda_lib.Context(f, m, bins=37, fixed_depth=12, moving_depth=12)
    np.testing.assert_array_equal(ctx.fixed_bins(), oracle.bin_volume(f, 37, 12))
    _, q16 = random_q16(f.shape, m.shape, 4, seed=4)
    for q in q16:
        np.testing.assert_array_equal(ctx.resample(q, np.uint16), oracle.resample(m, q, f.shape, depth=12))


def test_affine_builder_matches_oracle_bit_for_bit(cuda_lib):
    f = np.zeros((20, 24, 30), np.uint16)
    m = np.zeros((22, 28, 26), np.uint16)
    sf, sm = (1.0, 0.875, 1.25), (1.125, 1.0, 1.375)
    ctx = cuda_lib.Context(f, m, bins=16, fixed_spacing=sf, moving_spacing=sm)
    prm = phantoms.random_transforms(2000, seed=5, t_mm=30, r_deg=180, s_range=(0.5, 1.5))
    a, q, j = ctx.affine(prm)
    for t in range(len(prm)):
        ao, jo = oracle.affine(prm[t], f.shape, sf, m.shape, sm, with_jacobian=True)
        np.testing.assert_array_equal(a[t], ao)
        np.testing.assert_array_equal(q[t], oracle.affine_q16(ao))
        np.testing.assert_allclose(j[t], jo, rtol=1e-12, atol=1e-12)


def test_versor_and_offset_builder_matches_oracle_bit_for_bit(cuda_lib):
    # the unit-ball rotation (inside and outside the ball) and zero-centred scale parameters
    f = np.zeros((20, 24, 30), np.uint16)
    m = np.zeros((22, 28, 26), np.uint16)
    sf, sm = (1.0, 0.875, 1.25), (1.125, 1.0, 1.375)
    ctx = cuda_lib.Context(f, m, bins=16, fixed_spacing=sf, moving_spacing=sm, rotation="versor", scale="offset")
    rng = np.random.default_rng(8)
    n = 2000
    prm = np.concatenate([rng.uniform(-30, 30, (n, 3)), rng.uniform(-1.2, 1.2, (n, 3)),
                          rng.uniform(-0.5, 0.5, (n, 3))], 1).astype(np.float32)
    a, q, j = ctx.affine(prm)
    for t in range(n):
        ao, jo = oracle.affine(prm[t], f.shape, sf, m.shape, sm, with_jacobian=True, rotation="versor", scale="offset")
        np.testing.assert_array_equal(a[t], ao)
        np.testing.assert_array_equal(q[t], oracle.affine_q16(ao))
        np.testing.assert_allclose(j[t], jo, rtol=1e-12, atol=1e-12)


def test_versor_and_offset_mi_parity(cuda_lib):
    f, m = phantoms.head_pair(shape=(40, 44, 48), spacing=(1, 1, 1), seed=9)
    ctx = cuda_lib.Context(f, m, bins=64, fixed_depth=12, moving_depth=12, rotation="versor", scale="offset")
    rng = np.random.default_rng(10)
    prm = np.concatenate([rng.uniform(-4, 4, (12, 3)), rng.uniform(-0.15, 0.15, (12, 3)),
                          rng.uniform(-0.1, 0.1, (12, 3))], 1).astype(np.float32)
    mi, h, cnt = ctx.eval(prm, [1.0, 1.5], with_entropies=True)
    q16 = np.stack([oracle.affine_q16(oracle.affine(p, f.shape, (1, 1, 1), m.shape, (1, 1, 1), rotation="versor",
                                                    scale="offset")) for p in prm])
    mi_o, h_o, cnt_o = oracle.mi_eval_q16(f, m, 64, q16, [1.0, 1.5], fixed_depth=12, moving_depth=12, nthreads=8)
    np.testing.assert_array_equal(cnt, cnt_o)
    assert_mi_close(mi, mi_o, h_o)


def test_hand_enumerated_cases_on_gpu(cuda_lib):
    vols, cases = hand_cases.load()
    for c in cases:
        bins = hand_cases.bins_of(c)
        ctx = cuda_lib.Context(hand_cases.volume(vols[c["fixed"]]), hand_cases.volume(vols[c["moving"]]), bins=bins)
        want = hand_cases.expected_hist(c, np.uint32)
        for path in (cuda_lib.PATH_PLAIN, cuda_lib.PATH_BATCHED):
            h = ctx.hist(affines=np.array(c["q16"], np.int32), path=path)
            np.testing.assert_array_equal(h[0], want, err_msg=c["name"])
        qs = [float(k) for k in c["mi"]]
        mi = ctx.eval_q16(np.array(c["q16"], np.int32), qs)
        np.testing.assert_allclose(mi[0], [c["mi"][k] for k in c["mi"]], rtol=0, atol=1e-12)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("path", ["plain", "batched"])
def test_tiny_workload_histograms_and_mi(cuda_lib, tiny_pair, variant, path):
    f, m = tiny_pair
    prm = phantoms.tiny_sweep()
    ctx = cuda_lib.Context(f, m, bins=32, hist_variant=variant, path=path)
    qs = [1.0, 0.5, 1.5]
    mi, h, cnt = ctx.eval(prm, qs, with_entropies=True)
    mi_o, h_o, cnt_o = oracle.mi_eval(f, m, 32, prm, qs, nthreads=8)
    np.testing.assert_array_equal(cnt, cnt_o)
    assert_mi_close(mi, mi_o, h_o)
    np.testing.assert_allclose(h, h_o, rtol=1e-9, atol=1e-12)
    H = ctx.hist(transforms=prm, path=cuda_lib.PATH_PLAIN if path == "plain" else cuda_lib.PATH_BATCHED)
    for t in range(len(prm)):
        q16 = oracle.affine_q16(oracle.affine(prm[t], f.shape, (1, 1, 1), m.shape, (1, 1, 1)))
        ho, n = oracle.joint_hist(f, m, q16, 32)
        np.testing.assert_array_equal(H[t], ho.astype(np.uint32))


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("bins", [2, 37, 64, 128, 256])
def test_ragged_sizes_all_variants(cuda_lib, variant, bins):
    # odd dims spanning several row batches and a ragged tail, 12-bit data, random 9-parameter transforms
    f, m = phantoms.head_pair(shape=(29, 41, 75), spacing=(1, 1, 1), seed=6)
    m = np.ascontiguousarray(m[:, :37, :71])
    if bins > 181 and variant in U32_VARIANTS:
        pytest.skip("32-bit counters do not fit shared memory at this bin count")
    prm, q16 = random_q16(f.shape, m.shape, 40, seed=bins)
    for path in (cuda_lib.PATH_PLAIN, cuda_lib.PATH_BATCHED):
        ctx = cuda_lib.Context(f, m, bins=bins, fixed_depth=12, moving_depth=12, hist_variant=variant)
        H = ctx.hist(affines=q16, path=path)
        for t in range(0, len(q16), 3):
            ho, _ = oracle.joint_hist(f, m, q16[t], bins, 12, 12)
            np.testing.assert_array_equal(H[t], ho.astype(np.uint32))
    mi, h, cnt = ctx.eval_q16(q16, [1.0, 2.0], with_entropies=True)
    mi_o, h_o, cnt_o = oracle.mi_eval_q16(f, m, bins, q16, [1.0, 2.0], fixed_depth=12, moving_depth=12, nthreads=8)
    np.testing.assert_array_equal(cnt, cnt_o)
    assert_mi_close(mi, mi_o, h_o)


@pytest.mark.parametrize("variant", [2, 3, 6, 7, 8, 9, 10, 12, 13, 15])
def test_u16_counter_drains_exact(cuda_lib, variant):
    # a large uniform background makes the (0, 0) cell pass 2^14 many times inside one CTA
    f = np.zeros((64, 96, 100), np.uint16)
    m = np.zeros((64, 96, 100), np.uint16)
    f[20:40, 30:60, 30:70] = 3000
    m[22:42, 30:60, 28:68] = 1000
    ctx = cuda_lib.Context(f, m, bins=256, fixed_depth=12, moving_depth=12, hist_variant=variant)
    _, q16 = random_q16(f.shape, m.shape, 6, seed=7, t=2, r=5, s=(0.95, 1.05))
    q16 = np.concatenate([IDENT[None], q16.reshape(-1, 12)])
    for path in (cuda_lib.PATH_PLAIN, cuda_lib.PATH_BATCHED):
        H = ctx.hist(affines=q16, path=path)
        for t in range(len(q16)):
            ho, _ = oracle.joint_hist(f, m, q16[t], 256, 12, 12)
            np.testing.assert_array_equal(H[t], ho.astype(np.uint32))
    assert H[0, 0, 0] > 10 * 2 ** 14


@pytest.mark.parametrize("variant", [10, 11, 12, 13, 14, 15])
@pytest.mark.parametrize("tile_rows", [1, 2, 4, 32])
def test_tile_shapes_bit_exact(cuda_lib, variant, tile_rows):
    # every tile shape (1, 2 or 4 fixed rows per warp step, or the 32-row stream) and slab count on
    # ragged dims whose rows clip to every length mod 8, 16 and 32 (and to nothing at the overlap's
    # edge), both paths; 8-bit and 12-bit moving data
    for depth, dt in ((12, np.uint16), (8, np.uint8)):
        f, m = phantoms.head_pair(shape=(23, 37, 83), spacing=(1, 1, 1), depth=depth, seed=9 + depth, dtype=dt)
        m = np.ascontiguousarray(m[:, :35, :79])
        prm, q16 = random_q16(f.shape, m.shape, 24, seed=tile_rows + 3 * variant, t=6, r=20, s=(0.8, 1.2))
        for slabs in (1, 3, 16):
            ctx = cuda_lib.Context(f, m, bins=100, fixed_depth=depth, moving_depth=depth, hist_variant=variant,
                                   tile_rows=tile_rows, tile_slabs=slabs)
            for path in (cuda_lib.PATH_PLAIN, cuda_lib.PATH_BATCHED):
                H = ctx.hist(affines=q16, path=path)
                for t in range(0, len(q16), 5):
                    ho, _ = oracle.joint_hist(f, m, q16[t], 100, depth, depth)
                    np.testing.assert_array_equal(H[t], ho.astype(np.uint32), err_msg=f"{depth} {slabs} {path} {t}")


@pytest.mark.parametrize("variant", [10, 11, 12])  # MI_HV_ROWS_QUAD, MI_HV_U32_QUAD, MI_HV_U16_QUAD
@pytest.mark.parametrize("dtype, depth", [(np.uint8, 8), (np.uint16, 12), (np.uint16, 16)])
def test_quad_texels_full_range_and_last_column(cuda_lib, variant, dtype, depth):
    # The quad variants read 2 x 2 (y, z) quads at columns ix and ix + 1.  On the moving volume's last
    # x column (reached exactly by the identity and by whole-voxel x shifts, here with y and z fractions
    # too) column nx lies past the volume and is read clamped, where its weight is 0.  Full-range values
    # at every depth the quad texels hold (uchar4, ushort4), histograms bit for bit on both paths.
    rng = np.random.default_rng(40 + depth)
    f = rng.integers(0, 1 << depth, (19, 21, 35)).astype(dtype)
    m = rng.integers(0, 1 << depth, (17, 23, 29)).astype(dtype)
    nx = m.shape[2]
    fixed_q = [IDENT.copy()]
    for bx, by, bz in ((-6, 0, 0), (-6, 0x8000, 0x4000), (3, 0x1234, 0xFF00)):
        q = IDENT.copy()
        q[3], q[7], q[11] = bx * 65536, by, bz
        fixed_q.append(q)
    _, rq = random_q16(f.shape, m.shape, 6, seed=41, t=3.0, r=12.0, s=(0.9, 1.1))
    q16 = np.concatenate([np.stack(fixed_q), rq.reshape(len(rq), 12)]).astype(np.int32)
    want = [oracle.joint_hist(f, m, q, 64, depth, depth)[0].astype(np.uint32) for q in q16]
    assert want[0].sum() == 29 * 21 * 17  # the identity's overlap: moving x 0..28, y 0..20, z 0..16
    for path in (cuda_lib.PATH_PLAIN, cuda_lib.PATH_BATCHED):
        ctx = cuda_lib.Context(f, m, bins=64, fixed_depth=depth, moving_depth=depth, hist_variant=variant)
        H = ctx.hist(affines=q16, path=path)
        for t in range(len(q16)):
            np.testing.assert_array_equal(H[t], want[t], err_msg=f"{path} {t} (nx {nx})")
    mi = ctx.eval_q16(q16, [1.0, 1.5])
    mi_o, h_o, _ = oracle.mi_eval_q16(f, m, 64, q16, [1.0, 1.5], fixed_depth=depth, moving_depth=depth)
    assert_mi_close(mi, mi_o, h_o)


def test_gather_variants_need_depth_12_or_less(cuda_lib):
    # the z-pair atlas packs two values in 20-bit fields: 16-bit data keeps the other fetches
    rng = np.random.default_rng(10)
    f = rng.integers(0, 65536, size=(12, 14, 16), dtype=np.uint16)
    m = rng.integers(0, 65536, size=(12, 14, 16), dtype=np.uint16)
    with pytest.raises(cuda_lib.MIError) as ei:
        cuda_lib.Context(f, m, bins=32, hist_variant=cuda_lib.HV_ROWS_GATHER).eval(phantoms.identity_params(1))
    assert ei.value.status == cuda_lib.MI_EUNSUPPORTED
    ctx = cuda_lib.Context(f, m, bins=32)
    prm = phantoms.random_transforms(4, seed=11, t_mm=2, r_deg=5, s_range=(0.95, 1.05))
    mi, h, cnt = ctx.eval(prm, [1.0], with_entropies=True)
    mi_o, h_o, cnt_o = oracle.mi_eval(f, m, 32, prm, [1.0], nthreads=8)
    np.testing.assert_array_equal(cnt, cnt_o)
    assert_mi_close(mi, mi_o, h_o)


def test_edge_cases(cuda_lib):
    f, m = phantoms.ellipsoid_pair(shape=(16, 18, 20), seed=8)
    ctx = cuda_lib.Context(f, m, bins=16)
    # n = 0 is a no-op
    assert ctx.eval(np.zeros((0, 9), np.float32), [1.0]).shape == (0, 1)
    # empty overlap: NaN for that transform, the others still evaluated, status MI_EEMPTY
    prm = phantoms.identity_params(3)
    prm[1, 0] = 1000.0
    with pytest.raises(cuda_lib.MIError) as ei:
        ctx.eval(prm, [1.0, 2.0], allow_empty=False)
    assert ei.value.status == cuda_lib.MI_EEMPTY
    mi, h, cnt = ctx.eval(prm, [1.0, 2.0], with_entropies=True)
    assert cnt[1] == 0 and np.all(np.isnan(mi[1])) and np.all(np.isfinite(mi[[0, 2]]))
    # identity on u = v: MI = H(F) exactly (up to summation order)
    ctx2 = cuda_lib.Context(f, f, bins=16)
    mi, h, cnt = ctx2.eval(phantoms.identity_params(1), [1.0, 0.5, 2.0], with_entropies=True)
    np.testing.assert_allclose(mi[0], h[0, :, 0], rtol=1e-12)
    assert cnt[0] == f.size
    # invalid arguments
    for bad_q in ([0.0], [-1.0], [1.0000001], [float("nan")], [1.0] * 9):
        with pytest.raises(cuda_lib.MIError) as ei:
            ctx.eval(prm, bad_q)
        assert ei.value.status == cuda_lib.MI_EINVAL
    bad = phantoms.identity_params(1)
    bad[0, 3] = np.nan
    with pytest.raises(cuda_lib.MIError):
        ctx.eval(bad, [1.0])
    huge = phantoms.identity_params(1)
    huge[0, 6] = 1e6
    with pytest.raises(cuda_lib.MIError) as ei:
        ctx.eval(huge, [1.0])
    assert ei.value.status == cuda_lib.MI_ERANGE
    with pytest.raises(cuda_lib.MIError):
        cuda_lib.Context(f, m, bins=1)
    with pytest.raises(cuda_lib.MIError):
        cuda_lib.Context(f, m, bins=257)
    with pytest.raises(cuda_lib.MIError):
        cuda_lib.Context(f[:1], m, bins=16)


@pytest.mark.parametrize("dtype, depth", [(np.uint8, 8), (np.uint16, 12)])
def test_smallest_volumes_extreme_bins_and_eight_q(cuda_lib, dtype, depth):
    """2 x 2 x 2 and small ragged pairs, 2 and 256 bins, the 8 q a call takes, every variant and both
    paths: histograms bit-exact, overlap counts (1 to 8 voxels, or none) and MI as the oracle's."""
    rng = np.random.default_rng(95)
    qs = [0.2, 0.5, 0.8, 1.0, 1.2, 1.5, 2.0, 3.0]
    for shape_f, shape_m in (((2, 2, 2), (2, 2, 2)), ((3, 2, 5), (2, 4, 2))):
        f = rng.integers(0, 1 << depth, shape_f).astype(dtype)
        m = rng.integers(0, 1 << depth, shape_m).astype(dtype)
        prm = phantoms.random_transforms(11, seed=96, t_mm=0.6, r_deg=10, s_range=(0.9, 1.1))
        prm = np.concatenate([phantoms.identity_params(1), prm])
        q16 = np.stack([oracle.affine_q16(oracle.affine(p, shape_f, (1, 1, 1), shape_m, (1, 1, 1))) for p in prm])
        for bins in (2, 256):
            mi_o, h_o, cnt_o = oracle.mi_eval_q16(f, m, bins, q16, qs, fixed_depth=depth, moving_depth=depth)
            want = [oracle.joint_hist(f, m, q, bins, depth, depth)[0].astype(np.uint32) for q in q16]
            assert cnt_o.min() == 0 and 1 in cnt_o and cnt_o.max() >= 3  # empty, one-voxel and wider overlaps
            ran = 0
            for variant in VARIANTS:
                ctx = cuda_lib.Context(f, m, bins=bins, fixed_depth=depth, moving_depth=depth, hist_variant=variant)
                if bins == 256 and variant in U32_VARIANTS:  # 32-bit counters do not fit shared memory
                    with pytest.raises(cuda_lib.MIError) as ei:
                        ctx.hist(affines=q16[:1])
                    assert ei.value.status == cuda_lib.MI_EUNSUPPORTED
                    continue
                for path in (cuda_lib.PATH_PLAIN, cuda_lib.PATH_BATCHED):
                    H = ctx.hist(affines=q16, path=path)
                    for t in range(len(q16)):
                        np.testing.assert_array_equal(H[t], want[t])
                mi, h, cnt = ctx.eval_q16(q16, qs, with_entropies=True)
                np.testing.assert_array_equal(cnt, cnt_o)
                ok = cnt_o > 0
                assert np.all(np.isnan(mi[~ok]))
                assert_mi_close(mi[ok], mi_o[ok], h_o[ok])
                ran += 1
            assert ran == (16 if bins == 2 else 16 - len(U32_VARIANTS))


def test_bit_depth_clamp_and_small_depth(cuda_lib):
    rng = np.random.default_rng(9)
    f = rng.integers(0, 64, (12, 13, 14), dtype=np.uint8)
    m = rng.integers(0, 256, (12, 13, 14), dtype=np.uint8)  # values above 2^6 - 1 are clamped on load
    ctx = cuda_lib.Context(f, m, bins=8, fixed_depth=6, moving_depth=6)
    _, q16 = random_q16(f.shape, m.shape, 8, seed=10)
    H = ctx.hist(affines=q16, path=cuda_lib.PATH_PLAIN)
    for t in range(len(q16)):
        ho, _ = oracle.joint_hist(f, m, q16[t], 8, 6, 6)
        np.testing.assert_array_equal(H[t], ho.astype(np.uint32))


def test_float_volumes_hard_path(cuda_lib):
    f, m = phantoms.head_pair(shape=(20, 24, 28), spacing=(1, 1, 1), seed=11, dtype=np.float32)
    ctx = cuda_lib.Context(f, m, bins=48)
    prm = phantoms.random_transforms(10, seed=12, t_mm=3, r_deg=10, s_range=(0.95, 1.05))
    mi, h, cnt = ctx.eval(prm, [1.0, 1.5], with_entropies=True)
    mi_o, h_o, cnt_o = oracle.mi_eval(f, m, 48, prm, [1.0, 1.5], nthreads=8)
    np.testing.assert_array_equal(cnt, cnt_o)
    assert_mi_close(mi, mi_o, h_o)


def test_options_bits_and_pseudo_additive(cuda_lib, tiny_pair):
    f, m = tiny_pair
    prm = phantoms.tiny_sweep()[:5]
    for form, fname in ((0, "additive"), (1, "pseudo_additive")):
        for bits in (False, True):
            ctx = cuda_lib.Context(f, m, bins=32, tsallis_form=fname, bits=bits)
            mi = ctx.eval(prm, [1.0, 0.5, 2.0])
            mi_o, h_o, _ = oracle.mi_eval(f, m, 32, prm, [1.0, 0.5, 2.0], form=form, bits=bits)
            assert_mi_close(mi, mi_o, h_o)


def test_device_and_host_buffers_agree(cuda_lib, tiny_pair):
    import torch

    f, m = tiny_pair
    prm = phantoms.random_transforms(200, seed=13, t_mm=5, r_deg=8)
    ctx = cuda_lib.Context(torch.from_numpy(f).cuda(), torch.from_numpy(m).cuda(), bins=32)
    a = ctx.eval(prm, [1.0, 1.5])
    b = ctx.eval(torch.from_numpy(prm).cuda(), [1.0, 1.5])
    assert b.is_cuda
    np.testing.assert_array_equal(a, b.cpu().numpy())
    s = torch.cuda.Stream()
    ctx.set_stream(s)
    c = ctx.eval(prm, [1.0, 1.5])
    np.testing.assert_array_equal(a, c)


def test_batched_equals_plain_and_graph_replay(cuda_lib, tiny_pair):
    f, m = tiny_pair
    prm = phantoms.random_transforms(400, seed=14, t_mm=6, r_deg=10)
    qs = [0.5, 1.0, 1.5, 2.0]
    plain = cuda_lib.Context(f, m, bins=32, path="plain").eval(prm, qs, with_entropies=True)
    ctx = cuda_lib.Context(f, m, bins=32, path="batched")
    for _ in range(3):  # capture, then two replays
        got = ctx.eval(prm, qs, with_entropies=True)
        np.testing.assert_array_equal(got[2], plain[2])
        np.testing.assert_allclose(got[0], plain[0], rtol=1e-12, atol=1e-14)
    prm2 = prm.copy()
    prm2[:, 0] += 1.0  # same shapes, new values: the replayed graph must read them
    got2 = ctx.eval(prm2, qs)
    want2 = cuda_lib.Context(f, m, bins=32, path="plain").eval(prm2, qs)
    np.testing.assert_allclose(got2, want2, rtol=1e-12, atol=1e-14)


def test_many_transforms_cross_every_chunk(cuda_lib):
    """5000 transforms at 256 bins: the plain path takes them in chunks of 256 (its global histograms are
    capped at 64 MB), the batched path in one graph-replayed launch; a few have no overlap.  Counts equal
    the oracle's and MI is within tolerance for every transform on both paths."""
    f, m = phantoms.head_pair(shape=(16, 18, 20), spacing=(1, 1, 1), seed=99)
    prm = phantoms.random_transforms(5000, seed=100, t_mm=4, r_deg=15, s_range=(0.9, 1.1))
    prm[::997, 1] = 400.0  # no overlap
    qs = [0.5, 1.0, 2.0]
    mi_o, h_o, cnt_o = oracle.mi_eval(f, m, 256, prm, qs, fixed_depth=12, moving_depth=12, nthreads=8)
    assert np.count_nonzero(cnt_o == 0) == 6
    ok = cnt_o > 0
    for path in ("plain", "batched"):
        ctx = cuda_lib.Context(f, m, bins=256, fixed_depth=12, moving_depth=12, path=path)
        mi, h, cnt = ctx.eval(prm, qs, with_entropies=True)
        np.testing.assert_array_equal(cnt, cnt_o)
        assert np.all(np.isnan(mi[~ok]))
        assert_mi_close(mi[ok], mi_o[ok], h_o[ok])


def test_uneven_batch_small(cuda_lib):
    specs = [((40, 36, 50), np.uint8, 8, 32), ((30, 44, 38), np.uint16, 12, 64), ((50, 30, 33), np.uint8, 8, 128),
             ((24, 52, 47), np.uint16, 12, 64), ((35, 35, 35), np.uint16, 12, 32)]
    pairs = []
    vols = []
    for i, (shape, dt, depth, bins) in enumerate(specs):
        f, m = phantoms.head_pair(shape=shape, spacing=(1, 1, 1), depth=depth, seed=20 + i, dtype=dt)
        vols.append((f, m, depth, bins))
        pairs.append(dict(fixed=f, moving=m, bins=bins, fixed_depth=depth, moving_depth=depth))
    ctx = cuda_lib.Context(pairs=pairs)
    n_per = 12
    prm = phantoms.random_transforms(n_per * len(specs), seed=21, t_mm=4, r_deg=10, s_range=(0.9, 1.1))
    pair_of = np.repeat(np.arange(len(specs), dtype=np.int32), n_per)
    rng = np.random.default_rng(22)
    perm = rng.permutation(len(prm))
    prm, pair_of = prm[perm], pair_of[perm]
    qs = [1.0, 0.5, 1.5]
    mi, h, cnt = ctx.batch_eval(pair_of, prm, qs, with_entropies=True)
    for p, (f, m, depth, bins) in enumerate(vols):
        sel = np.nonzero(pair_of == p)[0]
        mi_o, h_o, cnt_o = oracle.mi_eval(f, m, bins, prm[sel], qs, fixed_depth=depth, moving_depth=depth, nthreads=8)
        np.testing.assert_array_equal(cnt[sel], cnt_o)
        assert_mi_close(mi[sel], mi_o, h_o)
        H = ctx.hist(transforms=prm[sel[:3]], pair=p, path=cuda_lib.PATH_BATCHED)
        for k, t in enumerate(sel[:3]):
            q16 = oracle.affine_q16(oracle.affine(prm[t], f.shape, (1, 1, 1), m.shape, (1, 1, 1)))
            ho, _ = oracle.joint_hist(f, m, q16, bins, depth, depth)
            np.testing.assert_array_equal(H[k], ho.astype(np.uint32))


@pytest.fixture(scope="module")
def pair_256_cubed():
    return phantoms.head_pair(shape=(256, 256, 256), spacing=(1, 1, 1), seed=30)


@pytest.mark.slow
@pytest.mark.parametrize("variant", [2, 3, 6, 7, 8, 9, 12, 13, 15])
def test_full_size_every_variant_that_fits_256_bins(cuda_lib, pair_256_cubed, variant):
    """Each histogram / fetch variant that holds 256 bins (16-bit counters with their drains, match
    aggregation, row-bound rows; pair, texture, quad and gather fetches) on the 256^3 12-bit pair,
    256 transforms in one batched launch: three sampled transforms' counts and MI against the oracle,
    one joint histogram bit for bit."""
    f, m = pair_256_cubed
    prm = phantoms.random_transforms(256, seed=110 + variant)
    qs = [0.5, 1.0, 2.0]
    ctx = cuda_lib.Context(f, m, bins=256, fixed_depth=12, moving_depth=12, path="batched", hist_variant=variant)
    try:
        mi, h, cnt = ctx.eval(prm, qs, with_entropies=True)
    except cuda_lib.MIError as e:  # 16-bit counters are limited by the fixed volume's size
        assert e.status == cuda_lib.MI_EUNSUPPORTED
        pytest.skip(str(e))
    sample = [0, 151, 255]
    mi_o, h_o, cnt_o = oracle.mi_eval(f, m, 256, prm[sample], qs, fixed_depth=12, moving_depth=12, nthreads=3)
    np.testing.assert_array_equal(cnt[sample], cnt_o)
    assert_mi_close(mi[sample], mi_o, h_o)
    q16 = oracle.affine_q16(oracle.affine(prm[151], f.shape, (1, 1, 1), m.shape, (1, 1, 1)))
    H = ctx.hist(affines=q16[None], path=cuda_lib.PATH_BATCHED)
    ho, _ = oracle.joint_hist(f, m, q16, 256, 12, 12)
    np.testing.assert_array_equal(H[0], ho.astype(np.uint32))


@pytest.mark.slow
def test_full_size_batched_256_cubed_sampled(cuda_lib):
    # the batched workload at full size (256^3 12-bit, 256 bins, 4096 transforms x 4 q) in the bench's
    # launch configuration; sampled transforms are checked against the oracle one by one
    f, m = phantoms.head_pair(shape=(256, 256, 256), spacing=(1, 1, 1), seed=30)
    prm = phantoms.random_transforms(4096, seed=31)
    qs = [0.5, 1.0, 1.5, 2.0]
    ctx = cuda_lib.Context(f, m, bins=256, fixed_depth=12, moving_depth=12, path="batched")
    mi, h, cnt = ctx.eval(prm, qs, with_entropies=True)
    # 16 transforms spread over the launch (first and last items, every wave position) against the oracle;
    # the joint histograms of 8 of them bit for bit
    sample = np.array([0, 1, 151, 152, 777, 1023, 1500, 2047, 2048, 2600, 3000, 3333, 3800, 4000, 4094, 4095])
    mi_o, h_o, cnt_o = oracle.mi_eval(f, m, 256, prm[sample], qs, fixed_depth=12, moving_depth=12, nthreads=16)
    np.testing.assert_array_equal(cnt[sample], cnt_o)
    assert_mi_close(mi[sample], mi_o, h_o)
    hsel = sample[::2]
    H = ctx.hist(transforms=prm[hsel], path=cuda_lib.PATH_BATCHED)
    from concurrent.futures import ThreadPoolExecutor

    def oracle_hist(t):
        q16 = oracle.affine_q16(oracle.affine(prm[t], f.shape, (1, 1, 1), m.shape, (1, 1, 1)))
        return oracle.joint_hist(f, m, q16, 256, 12, 12)[0]

    with ThreadPoolExecutor(max_workers=len(hsel)) as ex:
        hos = list(ex.map(oracle_hist, hsel))
    for k, ho in enumerate(hos):
        np.testing.assert_array_equal(H[k], ho.astype(np.uint32), err_msg=str(hsel[k]))


@pytest.mark.slow
def test_512_cubed_pair_both_paths_sampled(cuda_lib):
    """A 512^3 uint16 12-bit pair at 0.5 mm (134 M voxels a volume, a 1.1 GB quad array; fixed bins
    hold far more than 2^16 voxels, so every histogram row takes 32-bit counters), 128 bins: counts, MI
    and one full histogram against the oracle on sampled transforms of a 64-transform batched call,
    and the plain path on the same transforms."""
    from concurrent.futures import ThreadPoolExecutor

    sp = (0.5, 0.5, 0.5)
    f, m = phantoms.head_pair(shape=(512, 512, 512), spacing=sp, seed=101)
    prm = phantoms.random_transforms(64, seed=102, t_mm=8, r_deg=10, s_range=(0.9, 1.1))
    qs = [1.0, 2.0]
    sample = [0, 37, 63]

    def oracle_one(t):
        return oracle.mi_eval(f, m, 128, prm[[t]], qs, fixed_spacing=sp, moving_spacing=sp, fixed_depth=12,
                              moving_depth=12)

    with ThreadPoolExecutor(max_workers=len(sample)) as ex:
        res = list(ex.map(oracle_one, sample))
    mi_o = np.concatenate([r[0] for r in res])
    h_o = np.concatenate([r[1] for r in res])
    cnt_o = np.concatenate([r[2] for r in res])
    for path in ("batched", "plain"):
        ctx = cuda_lib.Context(f, m, bins=128, fixed_depth=12, moving_depth=12, fixed_spacing=sp,
                               moving_spacing=sp, path=path)
        mi, h, cnt = ctx.eval(prm if path == "batched" else prm[sample], qs, with_entropies=True)
        sel = sample if path == "batched" else slice(None)
        np.testing.assert_array_equal(cnt[sel], cnt_o)
        assert_mi_close(mi[sel], mi_o, h_o)
        if path == "batched":
            q16 = oracle.affine_q16(oracle.affine(prm[37], f.shape, sp, m.shape, sp))
            H = ctx.hist(affines=q16[None], path=cuda_lib.PATH_BATCHED)
            ho, _ = oracle.joint_hist(f, m, q16, 128, 12, 12)
            np.testing.assert_array_equal(H[0], ho.astype(np.uint32))
        del ctx


@pytest.mark.parametrize("n_a", [65535, 65536])
def test_row_bound_layout_at_the_16_bit_limit(cuda_lib, n_a):
    # a fixed bin holding exactly 65535 voxels keeps 16-bit counters; one more makes it a 32-bit row;
    # at identity with u = v its diagonal cell reaches the bin's full count
    shape = (40, 50, 70)
    f = np.full(shape, 3000, dtype=np.uint16)
    f.ravel()[:n_a] = 1000
    for variant in (8, 9, 10, 13):
        ctx = cuda_lib.Context(f, f, bins=64, fixed_depth=12, moving_depth=12, hist_variant=variant)
        for path in (cuda_lib.PATH_PLAIN, cuda_lib.PATH_BATCHED):
            H = ctx.hist(affines=IDENT, path=path)
            ho, _ = oracle.joint_hist(f, f, IDENT, 64, 12, 12)
            np.testing.assert_array_equal(H[0], ho.astype(np.uint32))
            assert H[0, 1000 * 64 >> 12, 1000 * 64 >> 12] == n_a


@pytest.mark.slow
@pytest.mark.parametrize("bins", [64, 128])
def test_head_sweeps_full_size(cuda_lib, bins):
    # the multimodal head-like workload: 256x256x160 12-bit, 1 x 1 x 1.2 mm, nine one-parameter sweeps of
    # 81 steps (729 transforms) about the known motion, six q values; sampled transforms against the oracle
    sp = (1.0, 1.0, 1.2)
    f, m = phantoms.head_pair(shape=(160, 256, 256), spacing=sp, seed=60)
    truth = np.asarray(phantoms.HEAD_MOTION, np.float32)
    prm = []
    for k, half in enumerate([20.0] * 3 + [30.0] * 3 + [0.2] * 3):
        prm.append(phantoms.sweep(k, truth[k] - half, truth[k] + half, 81, base=truth))
    prm = np.concatenate(prm)
    qs = [0.2, 0.5, 0.8, 1.0, 1.5, 2.0]
    ctx = cuda_lib.Context(f, m, bins=bins, fixed_depth=12, moving_depth=12, fixed_spacing=sp, moving_spacing=sp)
    mi, h, cnt = ctx.eval(prm, qs, with_entropies=True)
    assert np.all(np.isfinite(mi))
    sample = np.array([0, 40, 121, 283, 364, 500, 688, 728])
    mi_o, h_o, cnt_o = oracle.mi_eval(f, m, bins, prm[sample], qs, fixed_spacing=sp, moving_spacing=sp,
                                      fixed_depth=12, moving_depth=12, nthreads=16)
    np.testing.assert_array_equal(cnt[sample], cnt_o)
    assert_mi_close(mi[sample], mi_o, h_o)
    H = ctx.hist(transforms=prm[sample[:2]])
    for k, t in enumerate(sample[:2]):
        q16 = oracle.affine_q16(oracle.affine(prm[t], f.shape, sp, m.shape, sp))
        ho, _ = oracle.joint_hist(f, m, q16, bins, 12, 12)
        np.testing.assert_array_equal(H[k], ho.astype(np.uint32))
    # Eq. 3: along every sweep the Shannon MI peaks at the known motion (the sweep's centre) within one step
    peak = mi[:, qs.index(1.0)].reshape(9, 81).argmax(1)
    assert np.all(np.abs(peak - 40) <= 1), peak


@pytest.mark.slow
def test_uneven_batch_full_size(cuda_lib):
    # 48 pairs from 96^3 up to 320x320x200, mixed uint8/uint16, bins in {32, 64, 128}, 256 transforms each,
    # all in one persistent launch; two sampled transforms per pair against the oracle
    specs = phantoms.uneven_specs(48, seed=5)
    pairs, vols = [], []
    for s in specs:
        f, m = phantoms.head_pair(shape=s["shape"], spacing=(1, 1, 1), depth=s["depth"], seed=s["seed"], dtype=s["dtype"])
        vols.append((f, m, s["depth"], s["bins"]))
        pairs.append(dict(fixed=f, moving=m, bins=s["bins"], fixed_depth=s["depth"], moving_depth=s["depth"]))
    ctx = cuda_lib.Context(pairs=pairs)
    n_per = 256
    prm = phantoms.random_transforms(n_per * len(specs), seed=61)
    pair_of = np.repeat(np.arange(len(specs), dtype=np.int32), n_per)
    perm = np.random.default_rng(62).permutation(len(prm))
    prm, pair_of = prm[perm], pair_of[perm]
    qs = [1.0, 0.5, 1.5, 2.0]
    mi, h, cnt = ctx.batch_eval(pair_of, prm, qs, with_entropies=True)
    for p, (f, m, depth, bins) in enumerate(vols):
        sel = np.nonzero(pair_of == p)[0]
        assert len(sel) == n_per
        chk = sel[[0, n_per - 1]]
        mi_o, h_o, cnt_o = oracle.mi_eval(f, m, bins, prm[chk], qs, fixed_depth=depth, moving_depth=depth, nthreads=16)
        np.testing.assert_array_equal(cnt[chk], cnt_o)
        ok = cnt_o > 0
        assert_mi_close(mi[chk][ok], mi_o[ok], h_o[ok])
    # the Parzen MI and gradient of the 8 largest pairs, each at its own bin count, 64 transforms each, in
    # one call of a multi-pair Parzen context (one launch per kernel); one transform per pair against the
    # FP64 oracle (one host thread per pair: the oracle's C code runs outside the interpreter lock)
    from concurrent.futures import ThreadPoolExecutor

    big = np.argsort([np.prod(s["shape"]) for s in specs])[-8:]
    pctx = cuda_lib.Context(pairs=[dict(fixed=vols[p][0], moving=vols[p][1], bins=vols[p][3], fixed_depth=vols[p][2],
                                        moving_depth=vols[p][2]) for p in big], kernel="parzen")
    psel = [np.nonzero(pair_of == p)[0][:64] for p in big]
    pof = np.concatenate([np.full(64, k, np.int32) for k in range(len(big))])
    qz = [1.0, 0.7, 1.3]
    mi_p, g_p = pctx.batch_grad(pof, prm[np.concatenate(psel)], qz)
    assert pctx.last_kernel_ms()[1] == 6  # forward, marginals, cells, MI, adjoint, gradient: once each

    def oracle_first(k):
        f, m, depth, bins = vols[big[k]]
        aff, J = oracle.affine(prm[psel[k][0]], f.shape, (1, 1, 1), m.shape, (1, 1, 1), with_jacobian=True)
        return oracle.parzen(f, m, aff, bins, qz, daff=J, fixed_depth=depth, moving_depth=depth)

    with ThreadPoolExecutor(max_workers=len(big)) as ex:
        res = list(ex.map(oracle_first, range(len(big))))
    for k, (mi_o, g_o, _) in enumerate(res):
        row = 64 * k
        assert np.all(np.abs(mi_p[row] - mi_o) <= 1e-6 * np.maximum(np.abs(mi_o), 1.0)), (k, mi_p[row], mi_o)
        for iq in range(3):
            assert np.abs(g_p[row, iq] - g_o[iq]).max() <= 1e-4 * np.abs(g_o[iq]).max(), (k, iq)


def test_versor_on_the_sphere_is_a_half_turn(cuda_lib):
    # |v| = 1 exactly and |v| > 1: the same half turn (the sphere surface of the unit-ball maps)
    f, m = phantoms.head_pair(shape=(30, 30, 30), spacing=(1, 1, 1), seed=12)
    ctx = cuda_lib.Context(f, m, bins=32, fixed_depth=12, moving_depth=12, rotation="versor")
    prm = np.array([[0, 0, 0, 0, 0, 1.0, 1, 1, 1], [0, 0, 0, 0, 0, 3.0, 1, 1, 1],
                    [0, 0, 0, 0.6, 0.8, 0, 1, 1, 1], [0, 0, 0, 1.2, 1.6, 0, 1, 1, 1]], np.float32)
    a, q, _ = ctx.affine(prm)
    np.testing.assert_array_equal(q[0], q[1])
    np.testing.assert_array_equal(q[2], q[3])
    mi = ctx.eval(prm, [1.0])
    assert mi[0, 0] == mi[1, 0] and mi[2, 0] == mi[3, 0]
