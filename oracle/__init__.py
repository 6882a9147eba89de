"""CPU oracle for hard-binned and Parzen mutual information (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``mi_oracle.c`` (plain C,
FP64 entropies, exact integer fixed-point resampling) through ctypes and
shares no code with the CUDA library.

Each wrapper cites the passage of the paper it follows; the readings R1..R17
(binning, transform conventions, fixed point, integer trilinear, overlap-only
counts, natural log, Tsallis forms, Parzen soft histogram and its adjoint,
unit-ball rotation, zero-centred scale, random sampling, general affine) are
stated in ``mi_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mi_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libmi_oracle.so")
_lib = None
_lock = threading.Lock()

U8, U16, F32 = 0, 1, 2
_DTYPES = {np.dtype(np.uint8): U8, np.dtype(np.uint16): U16, np.dtype(np.float32): F32}


def build(force: bool = False) -> str:
    """Compile ``mi_oracle.c`` into ``libmi_oracle.so`` next to it (gcc, OpenMP if available)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", _SRC, "-o", _LIB_PATH + ".tmp"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:] + ["-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-lm"], check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            I = ctypes.c_int
            I64 = ctypes.c_int64
            lib.orc_bin_of.restype = I
            lib.orc_bin_of.argtypes = [ctypes.c_uint32, I, I]
            lib.orc_bin_volume.restype = None
            lib.orc_bin_volume.argtypes = [P, I, I, I64, I, P]
            lib.orc_f32_to_u16.restype = None
            lib.orc_f32_to_u16.argtypes = [P, I64, P]
            lib.orc_affine.restype = None
            lib.orc_affine.argtypes = [P, P, P, P, P, P, P]
            lib.orc_affine_mode.restype = None
            lib.orc_affine_mode.argtypes = [P, P, P, P, P, I, I, P, P]
            lib.orc_affine_q16.restype = I
            lib.orc_affine_q16.argtypes = [P, P]
            lib.orc_resample.restype = None
            lib.orc_resample.argtypes = [P, I, I, P, P, P, P]
            lib.orc_joint_hist.restype = I64
            lib.orc_joint_hist.argtypes = [P, P, P, I, I, P, P, I, P]
            lib.orc_entropies.restype = I
            lib.orc_entropies.argtypes = [P, I, P, I, I, I, P, P]
            lib.orc_mi_eval.restype = I
            lib.orc_mi_eval.argtypes = [P, P, P, P, I, I, P, P, I, P, I, P, I, I, I, I, P, P, P]
            lib.orc_mi_eval_q16.restype = I
            lib.orc_mi_eval_q16.argtypes = [P, P, P, I, I, P, I, P, I, P, I, I, I, I, P, P, P]
            U32 = ctypes.c_uint32
            lib.orc_mi_eval_q16_s.restype = I
            lib.orc_mi_eval_q16_s.argtypes = [P, P, P, I, I, P, I, P, I, P, I, I, I, I, U32, U32, P, P, P]
            lib.orc_joint_hist_s.restype = I64
            lib.orc_joint_hist_s.argtypes = [P, P, P, I, I, P, P, I, U32, U32, P]
            lib.orc_fmix32.restype = U32
            lib.orc_fmix32.argtypes = [U32]
            lib.orc_sampled.restype = I
            lib.orc_sampled.argtypes = [I64, U32, U32]
            lib.orc_sample_threshold.restype = U32
            lib.orc_sample_threshold.argtypes = [ctypes.c_double]
            lib.orc_beta3.restype = ctypes.c_double
            lib.orc_beta3.argtypes = [ctypes.c_double]
            lib.orc_dbeta3.restype = ctypes.c_double
            lib.orc_dbeta3.argtypes = [ctypes.c_double]
            lib.orc_parzen_fixed_bin.restype = I
            lib.orc_parzen_fixed_bin.argtypes = [P, I, I, I64, I]
            lib.orc_parzen.restype = I
            lib.orc_parzen.argtypes = [P, I, I, P, P, I, I, P, P, P, I, I, P, I, I, I, P, P, P, P, P]
            lib.orc_affine_matrix.restype = None
            lib.orc_affine_matrix.argtypes = [P, P, P, P, P, P, P]
            lib.orc_overlap_mask.restype = None
            lib.orc_overlap_mask.argtypes = [P, P, P, P]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dims(vol: np.ndarray) -> np.ndarray:
    """Volumes are numpy arrays indexed [z, y, x] (x fastest); dims are (nx, ny, nz)."""
    assert vol.ndim == 3 and vol.flags["C_CONTIGUOUS"]
    return np.array([vol.shape[2], vol.shape[1], vol.shape[0]], dtype=np.int32)


def _dtype_code(vol: np.ndarray) -> int:
    return _DTYPES[vol.dtype]


def _depth(vol: np.ndarray, depth: int | None) -> int:
    if depth is not None:
        return int(depth)
    return {U8: 8, U16: 16, F32: 16}[_dtype_code(vol)]


def bin_of(v: int, bins: int, depth: int) -> int:
    """R1 binning of one integer value (Discussion: full, all-voxel histogram)."""
    return _load().orc_bin_of(int(v), int(bins), int(depth))


def f32_to_u16(vol: np.ndarray) -> np.ndarray:
    """Hard-mode conversion of a [0, 1] float volume to 16-bit integers."""
    vol = np.ascontiguousarray(vol, dtype=np.float32)
    out = np.empty(vol.shape, dtype=np.uint16)
    _load().orc_f32_to_u16(_p(vol), vol.size, _p(out))
    return out


def _as_int(vol: np.ndarray, depth: int | None):
    """Integer view used by the hard path: float volumes go through f32_to_u16 (depth 16)."""
    vol = np.ascontiguousarray(vol)
    if vol.dtype == np.float32:
        return f32_to_u16(vol), 16
    return vol, _depth(vol, depth)


def bin_volume(vol: np.ndarray, bins: int, depth: int | None = None) -> np.ndarray:
    """R1 binning of a whole volume to uint8 bin indices."""
    iv, d = _as_int(vol, depth)
    out = np.empty(iv.shape, dtype=np.uint8)
    _load().orc_bin_volume(_p(iv), _dtype_code(iv), d, iv.size, int(bins), _p(out))
    return out


def affine(params, fixed_shape, fixed_spacing, moving_shape, moving_spacing, with_jacobian=False,
           rotation="euler", scale="factor", transform="params"):
    """R2 (Fig. 1 Transform block; Introduction's translation/rotation/scale families).

    ``params`` = (tx, ty, tz mm, rx, ry, rz degrees, sx, sy, sz).  Shapes are
    numpy shapes (nz, ny, nx); spacings are (sx, sy, sz) in mm.  Returns the
    3x4 FP64 matrix [A | b] mapping a fixed index (i, j, k) to a moving index,
    and optionally its 12x9 Jacobian with respect to the parameters.
    rotation="versor": the rotation parameters are the unit-ball versor of
    R14 (the Results' rotation maps); scale="offset": zero-centred scale
    parameters s, sigma = 1 + s (R15, the Results' scale maps).
    transform="affine": ``params`` is the general affine [M | t] (12 values,
    row-major; R17, the Methodology's 12 degrees of freedom) and the Jacobian
    is 12 x 12; rotation and scale do not apply.
    """
    lib = _load()
    nf = np.array(fixed_shape[::-1], dtype=np.int32)
    nm = np.array(moving_shape[::-1], dtype=np.int32)
    sf = np.ascontiguousarray(fixed_spacing, dtype=np.float32)
    sm = np.ascontiguousarray(moving_spacing, dtype=np.float32)
    out = np.empty(12, dtype=np.float64)
    if transform == "affine":
        prm = np.ascontiguousarray(params, dtype=np.float32).reshape(12)
        dout = np.empty(12 * 12, dtype=np.float64) if with_jacobian else None
        lib.orc_affine_matrix(_p(prm), _p(nf), _p(sf), _p(nm), _p(sm), _p(out), _p(dout) if with_jacobian else None)
        if with_jacobian:
            return out.reshape(3, 4), dout.reshape(12, 12)
        return out.reshape(3, 4)
    if transform != "params":
        raise ValueError("transform is 'params' or 'affine'")
    prm = np.ascontiguousarray(params, dtype=np.float32).reshape(9)
    dout = np.empty(12 * 9, dtype=np.float64) if with_jacobian else None
    if rotation not in ("euler", "versor") or scale not in ("factor", "offset"):
        raise ValueError("rotation is 'euler' or 'versor', scale is 'factor' or 'offset'")
    lib.orc_affine_mode(_p(prm), _p(nf), _p(sf), _p(nm), _p(sm), int(rotation == "versor"), int(scale == "offset"),
                        _p(out), _p(dout) if with_jacobian else None)
    if with_jacobian:
        return out.reshape(3, 4), dout.reshape(12, 9)
    return out.reshape(3, 4)


def affine_q16(aff) -> np.ndarray:
    """R3: llround(x * 65536) of each of the 12 entries of [A | b]."""
    a = np.ascontiguousarray(aff, dtype=np.float64).reshape(12)
    q = np.empty(12, dtype=np.int32)
    if _load().orc_affine_q16(_p(a), _p(q)) != 0:
        raise OverflowError("affine entry does not fit 16.16 fixed point")
    return q.reshape(3, 4)


def resample(moving: np.ndarray, q16, fixed_shape, depth: int | None = None) -> np.ndarray:
    """v(T(x)) on the fixed grid by R3/R4 integer trilinear resampling (0 outside)."""
    iv, d = _as_int(moving, depth)
    q = np.ascontiguousarray(q16, dtype=np.int32).reshape(12)
    out = np.empty(tuple(fixed_shape), dtype=iv.dtype)
    nf = np.array(tuple(fixed_shape)[::-1], dtype=np.int32)
    _load().orc_resample(_p(iv), _dtype_code(iv), d, _p(_dims(iv)), _p(nf), _p(q), _p(out))
    return out


def joint_hist(fixed: np.ndarray, moving: np.ndarray, q16, bins: int, fixed_depth=None, moving_depth=None,
               sample_fraction=0.0, sample_seed=0):
    """R5 joint histogram (row = fixed bin) over the overlap -- over the randomly
    sampled fixed voxels (R16) when 0 < sample_fraction < 1; returns (hist uint64, N)."""
    fb = bin_volume(fixed, bins, fixed_depth)
    mv, md = _as_int(moving, moving_depth)
    q = np.ascontiguousarray(q16, dtype=np.int32).reshape(12)
    h = np.empty((bins, bins), dtype=np.uint64)
    n = _load().orc_joint_hist_s(_p(fb), _p(_dims(fb)), _p(mv), _dtype_code(mv), md, _p(_dims(mv)), _p(q),
                                 int(bins), int(sample_seed) & 0xFFFFFFFF, sample_threshold(sample_fraction), _p(h))
    return h, int(n)


def entropies(hist, q, form: int = 0, bits: bool = False):
    """Eq. (1) Shannon / Tsallis entropies and Eq. (2) MI from one histogram.

    Returns (mi[nq], h[nq, 3]) with h = (H_F, H_M, H_FM).
    """
    h = np.ascontiguousarray(hist, dtype=np.float64)
    bins = h.shape[0]
    qs = np.ascontiguousarray(np.atleast_1d(q), dtype=np.float64)
    mi = np.empty(len(qs), dtype=np.float64)
    hh = np.empty((len(qs), 3), dtype=np.float64)
    _load().orc_entropies(_p(h), bins, _p(qs), len(qs), int(form), int(bool(bits)), _p(mi), _p(hh))
    return mi, hh


def _q_as_double(q):
    """q values travel as float32 through the library; the oracle uses the same values in FP64."""
    return np.ascontiguousarray(np.atleast_1d(np.asarray(q, dtype=np.float32)), dtype=np.float64)


def mi_eval(fixed, moving, bins, params, q, fixed_spacing=(1, 1, 1), moving_spacing=(1, 1, 1), form=0,
            bits=False, fixed_depth=None, moving_depth=None, nthreads=1):
    """Hard-binned MI for each transform (n x 9 params) and each q.

    Returns (mi[n, nq], h[n, nq, 3], count[n]).
    """
    fb = bin_volume(fixed, bins, fixed_depth)
    mv, md = _as_int(moving, moving_depth)
    prm = np.ascontiguousarray(params, dtype=np.float32).reshape(-1, 9)
    n = prm.shape[0]
    qs = _q_as_double(q)
    nq = len(qs)
    mi = np.empty((n, nq), dtype=np.float64)
    hh = np.empty((n, nq, 3), dtype=np.float64)
    cnt = np.empty(n, dtype=np.int64)
    sf = np.ascontiguousarray(fixed_spacing, dtype=np.float32)
    sm = np.ascontiguousarray(moving_spacing, dtype=np.float32)
    rc = _load().orc_mi_eval(_p(fb), _p(_dims(fb)), _p(sf), _p(mv), _dtype_code(mv), md, _p(_dims(mv)), _p(sm),
                             int(bins), _p(prm), n, _p(qs), nq, int(form), int(bool(bits)), int(nthreads), _p(mi),
                             _p(hh), _p(cnt))
    if rc != 0:
        raise RuntimeError(f"oracle mi_eval failed ({rc})")
    return mi, hh, cnt


def fmix32(k: int) -> int:
    """R16: the MurmurHash3 32-bit finalizer."""
    return int(_load().orc_fmix32(int(k) & 0xFFFFFFFF))


def sample_threshold(fraction: float) -> int:
    """R16: floor(fraction * 2^32) for 0 < fraction < 1, else 0 (every voxel)."""
    return int(_load().orc_sample_threshold(float(fraction)))


def sampled(index: int, seed: int, threshold: int) -> bool:
    """R16: whether the fixed voxel with this linear index takes part."""
    return bool(_load().orc_sampled(int(index), int(seed) & 0xFFFFFFFF, int(threshold)))


def mi_eval_q16(fixed, moving, bins, q16, q, form=0, bits=False, fixed_depth=None, moving_depth=None, nthreads=1,
                sample_fraction=0.0, sample_seed=0):
    """Hard-binned MI from 16.16 affines (n x 12 int32) given directly; with
    0 < sample_fraction < 1, over the randomly sampled fixed voxels (R16)."""
    fb = bin_volume(fixed, bins, fixed_depth)
    mv, md = _as_int(moving, moving_depth)
    qa = np.ascontiguousarray(q16, dtype=np.int32).reshape(-1, 12)
    n = qa.shape[0]
    qs = _q_as_double(q)
    nq = len(qs)
    mi = np.empty((n, nq), dtype=np.float64)
    hh = np.empty((n, nq, 3), dtype=np.float64)
    cnt = np.empty(n, dtype=np.int64)
    thr = sample_threshold(sample_fraction)
    rc = _load().orc_mi_eval_q16_s(_p(fb), _p(_dims(fb)), _p(mv), _dtype_code(mv), md, _p(_dims(mv)), int(bins),
                                   _p(qa), n, _p(qs), nq, int(form), int(bool(bits)), int(nthreads),
                                   int(sample_seed) & 0xFFFFFFFF, thr, _p(mi), _p(hh), _p(cnt))
    if rc != 0:
        raise RuntimeError(f"oracle mi_eval_q16 failed ({rc})")
    return mi, hh, cnt


def beta3(x: float) -> float:
    return _load().orc_beta3(float(x))


def dbeta3(x: float) -> float:
    return _load().orc_dbeta3(float(x))


def parzen_fixed_bins(fixed: np.ndarray, B: int, depth=None) -> np.ndarray:
    """R8 fixed bin of every voxel: floor(f (B - 4)) + 2."""
    lib = _load()
    f = np.ascontiguousarray(fixed)
    d = _depth(f, depth)
    flat = np.empty(f.size, dtype=np.int32)
    for x in range(f.size):
        flat[x] = lib.orc_parzen_fixed_bin(_p(f), _dtype_code(f), d, x, int(B))
    return flat.reshape(f.shape)


def parzen(fixed, moving, aff, B, q, daff=None, form=0, bits=False, mask=None, fixed_depth=None, moving_depth=None,
           want_hist=False):
    """R8/R9 Parzen MI (and gradient if ``daff`` is given) at one FP64 affine.

    ``aff`` is the 3x4 [A | b]; ``daff`` the 12 x npar Jacobian from
    :func:`affine` (npar = 9 parameters, or 12 for the general affine).
    Returns (mi[nq], grad[nq, npar] or None, N[, P]).
    """
    fx = np.ascontiguousarray(fixed)
    mv = np.ascontiguousarray(moving)
    a = np.ascontiguousarray(aff, dtype=np.float64).reshape(12)
    qs = _q_as_double(q)
    nq = len(qs)
    mi = np.empty(nq, dtype=np.float64)
    npar = int(np.asarray(daff).size // 12) if daff is not None else 9
    grad = np.empty((nq, npar), dtype=np.float64) if daff is not None else None
    da = np.ascontiguousarray(daff, dtype=np.float64).reshape(12 * npar) if daff is not None else None
    cnt = np.zeros(1, dtype=np.int64)
    ph = np.empty((B, B), dtype=np.float64) if want_hist else None
    mk = np.ascontiguousarray(mask, dtype=np.uint8) if mask is not None else None
    rc = _load().orc_parzen(_p(fx), _dtype_code(fx), _depth(fx, fixed_depth), _p(_dims(fx)), _p(mv), _dtype_code(mv),
                            _depth(mv, moving_depth), _p(_dims(mv)), _p(a), _p(da) if da is not None else None,
                            npar, int(B), _p(qs), nq, int(form), int(bool(bits)), _p(mk) if mk is not None else None,
                            _p(mi), _p(grad) if grad is not None else None, _p(cnt), _p(ph) if ph is not None else None)
    if rc != 0:
        raise RuntimeError(f"oracle parzen failed ({rc})")
    if want_hist:
        return mi, grad, int(cnt[0]), ph
    return mi, grad, int(cnt[0])


def overlap_mask(fixed_shape, moving_shape, aff) -> np.ndarray:
    """Voxels of the fixed grid whose FP64 moving index lies inside the moving volume."""
    a = np.ascontiguousarray(aff, dtype=np.float64).reshape(12)
    nf = np.array(tuple(fixed_shape)[::-1], dtype=np.int32)
    nm = np.array(tuple(moving_shape)[::-1], dtype=np.int32)
    mask = np.empty(tuple(fixed_shape), dtype=np.uint8)
    _load().orc_overlap_mask(_p(nf), _p(nm), _p(a), _p(mask))
    return mask
