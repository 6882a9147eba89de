"""GB300-native Shannon / Tsallis mutual information for 3D registration.

Python binding of the C ABI in ``include/mi.h`` (argument marshalling only;
every step of the metric runs in the CUDA library).  Volumes are numpy arrays
or torch tensors indexed [z, y, x] (x fastest), of dtype uint8, uint16 or
float32; spacings are (x, y, z) in mm.  Transforms are n x 9 float32
(tx, ty, tz mm; rx, ry, rz degrees; sx, sy, sz scale factors), or n x 12
for a general affine [M | t] (``transform="affine"``).

The metric is the paper's F_m(u(x), v(T(x))) (Fig. 1): Shannon MI of
Eq. (1)-(2), and Tsallis MI for q != 1, from one joint histogram per
transform (Discussion).  ``Context.grad`` and :class:`MIFunction` give the
gradient of the differentiable Parzen form for the optimiser of Eq. (3).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib

MI_OK, MI_EINVAL, MI_ENOMEM, MI_ECUDA, MI_EEMPTY, MI_EUNSUPPORTED, MI_ERANGE = range(7)
HV_AUTO, HV_U32, HV_U32_MATCH, HV_U16, HV_U16_MATCH = -1, 0, 1, 2, 3
HV_U32_TEX, HV_U32_MATCH_TEX, HV_U16_TEX, HV_U16_MATCH_TEX = 4, 5, 6, 7
HV_ROWS, HV_ROWS_TEX = 8, 9
HV_ROWS_QUAD, HV_U32_QUAD, HV_U16_QUAD = 10, 11, 12
HV_ROWS_GATHER, HV_U32_GATHER, HV_U16_GATHER = 13, 14, 15
PATH_AUTO, PATH_PLAIN, PATH_BATCHED = 0, 1, 2
_DT = {np.dtype(np.uint8): 0, np.dtype(np.uint16): 1, np.dtype(np.float32): 2}


class MIError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"[status {status}] {message}")
        self.status = status


def load():
    """Load (building if needed) the CUDA library; raises if it cannot be loaded."""
    return _lib.load()


def build(force: bool = False):
    return _lib.build(force=force)


def version() -> str:
    return load().mi_version().decode()


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _torch():
    import torch

    return torch


class _Arg:
    """Keeps a contiguous buffer alive and exposes its address."""

    def __init__(self, x, dtype=None):
        if x is None:
            self.obj, self.ptr, self.on_gpu = None, None, False
            return
        if _is_torch(x):
            torch = _torch()
            t = x.detach()
            if dtype is not None:
                t = t.to(getattr(torch, np.dtype(dtype).name))
            t = t.contiguous()
            self.obj, self.ptr, self.on_gpu = t, t.data_ptr(), t.is_cuda
        else:
            a = np.ascontiguousarray(x, dtype=dtype)
            self.obj, self.ptr, self.on_gpu = a, a.ctypes.data, False


def _np_dtype(x):
    if _is_torch(x):
        torch = _torch()
        return {torch.uint8: np.dtype(np.uint8), torch.float32: np.dtype(np.float32)}.get(
            x.dtype, np.dtype(np.uint16) if str(x.dtype) == "torch.uint16" else None)
    return np.asarray(x).dtype


def _volume(x, spacing, depth):
    dt = _np_dtype(x)
    if dt not in _DT:
        raise TypeError(f"volume dtype must be uint8, uint16 or float32, got {dt}")
    if len(x.shape) != 3:
        raise ValueError("volumes are 3D arrays indexed [z, y, x]")
    arg = _Arg(x)
    v = _lib.MiVolume()
    v.data = arg.ptr
    v.dtype = _DT[dt]
    v.dims[0], v.dims[1], v.dims[2] = int(x.shape[2]), int(x.shape[1]), int(x.shape[0])
    v.bit_depth = int(depth or 0)
    for a in range(3):
        v.spacing_mm[a] = float(spacing[a])
    return v, arg


def _options(kernel, tsallis_form, bits, hist_variant, path, use_graphs, autotune, device, block_threads=0,
             rotation="euler", scale="factor", sample_fraction=0.0, sample_seed=0, transform="params", tile_rows=0,
             tile_slabs=0):
    o = _lib.MiOptions()
    load().mi_options_default(ctypes.byref(o))
    o.kernel = {"hard": 0, "parzen": 1}[kernel]
    o.tsallis_form = {"additive": 0, "pseudo_additive": 1}[tsallis_form]
    o.log_bits = int(bool(bits))
    o.hist_variant = int(hist_variant)
    o.path = {"auto": 0, "plain": 1, "batched": 2}[path] if isinstance(path, str) else int(path)
    o.use_graphs = int(bool(use_graphs))
    o.autotune = int(bool(autotune))
    o.device = -1 if device is None else int(device)
    o.block_threads = int(block_threads)
    o.rotation = {"euler": 0, "versor": 1}[rotation]
    o.scale = {"factor": 0, "offset": 1}[scale]
    o.sample_fraction = float(sample_fraction)
    o.sample_seed = int(sample_seed) & 0xFFFFFFFF
    o.transform = {"params": 0, "affine": 1}[transform]
    o.tile_rows = int(tile_rows)
    o.tile_slabs = int(tile_slabs)
    return o


def _out(shape, like_gpu, dtype, device=None):
    if like_gpu:
        torch = _torch()
        return torch.empty(shape, dtype=getattr(torch, np.dtype(dtype).name), device=device or "cuda")
    return np.empty(shape, dtype=dtype)


def _ptr(x):
    if x is None:
        return None
    return x.data_ptr() if _is_torch(x) else x.ctypes.data


class Context:
    """One (fixed, moving) pair, or several pairs (``pairs=[...]``) for the uneven batch.

    kernel: "hard" (exact joint histogram, default) or "parzen" (differentiable).
    rotation: "euler" (rx, ry, rz in degrees, default) or "versor" (the unit-ball
    parameterisation of the paper's rotation maps); scale: "factor" (1 =
    identity, default) or "offset" (zero-centred, sigma = 1 + s).
    sample_fraction in (0, 1): the metric (hard or Parzen) over a random subset
    of the fixed voxels of that fraction, fixed by sample_seed (0: every voxel).
    transform: "params" (9 parameters, default) or "affine" (12: the general
    affine [M | t] row-major, M dimensionless, t in mm; gradients per entry).
    ``nparams`` is the count.
    tile_rows (0 = autotuned, or 1, 2, 4): adjacent fixed rows one warp step of
    the hard path covers, or 32: each warp walks its 32 clipped rows as one
    stream of voxels; tile_slabs (0 = 4, or 1..16): slabs per sweep of the
    batched kernel.
    """

    def __init__(self, fixed=None, moving=None, bins=64, fixed_spacing=(1.0, 1.0, 1.0),
                 moving_spacing=(1.0, 1.0, 1.0), fixed_depth=None, moving_depth=None, kernel="hard",
                 tsallis_form="additive", bits=False, hist_variant=HV_AUTO, path="auto", use_graphs=True,
                 autotune=True, device=None, pairs=None, block_threads=0, rotation="euler", scale="factor",
                 sample_fraction=0.0, sample_seed=0, transform="params", tile_rows=0, tile_slabs=0):
        self._lib = load()
        self._h = ctypes.c_void_p()
        self.kernel = kernel
        self.rotation, self.scale, self.transform = rotation, scale, transform
        opt = _options(kernel, tsallis_form, bits, hist_variant, path, use_graphs, autotune, device, block_threads,
                       rotation, scale, sample_fraction, sample_seed, transform, tile_rows, tile_slabs)
        if pairs is None:
            pairs = [dict(fixed=fixed, moving=moving, bins=bins, fixed_spacing=fixed_spacing,
                          moving_spacing=moving_spacing, fixed_depth=fixed_depth, moving_depth=moving_depth)]
            batch = False
        else:
            batch = True
        self.npairs = len(pairs)
        n = len(pairs)
        fx = (_lib.MiVolume * n)()
        mv = (_lib.MiVolume * n)()
        keep = []
        bins_arr = (ctypes.c_int * n)()
        self.shapes = []
        self.bins = []
        for i, p in enumerate(pairs):
            fv, fa = _volume(p["fixed"], p.get("fixed_spacing", (1, 1, 1)), p.get("fixed_depth"))
            mvv, ma = _volume(p["moving"], p.get("moving_spacing", (1, 1, 1)), p.get("moving_depth"))
            fx[i], mv[i] = fv, mvv
            keep += [fa, ma]
            bins_arr[i] = int(p["bins"])
            self.shapes.append(tuple(p["fixed"].shape))
            self.bins.append(int(p["bins"]))
        if batch:
            st = self._lib.mi_batch_create(ctypes.byref(self._h), fx, mv, ctypes.cast(bins_arr, ctypes.c_void_p), n,
                                           ctypes.byref(opt))
        else:
            st = self._lib.mi_create(ctypes.byref(self._h), fx, mv, bins_arr[0], ctypes.byref(opt))
        if st != MI_OK:
            raise MIError(st, self._lib.mi_last_error(None).decode())
        self.nparams = self._lib.mi_transform_size(self._h)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.mi_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, allow_empty=False):
        if st == MI_OK or (allow_empty and st == MI_EEMPTY):
            return st
        raise MIError(st, self._lib.mi_last_error(self._h).decode())

    def set_stream(self, stream):
        """Order later work on a CUDA stream (a torch.cuda.Stream, a raw handle, or None)."""
        h = getattr(stream, "cuda_stream", stream)
        self._check(self._lib.mi_set_stream(self._h, ctypes.c_void_p(h) if h else None))

    def eval(self, transforms, q=(1.0,), with_entropies=False, allow_empty=True):
        """MI (n x nq) for n transforms; with_entropies adds (H_F, H_M, H_FM) per q and the overlap counts
        (for a Parzen context the entropies are None: only the counts)."""
        T = _Arg(transforms, np.float32)
        Q = _Arg(np.atleast_1d(np.asarray(q, dtype=np.float32)))
        n = int(np.prod(T.obj.shape) // self.nparams)
        nq = int(np.asarray(q).size)
        gpu = T.on_gpu
        dev = T.obj.device if gpu else None
        mi = _out((n, nq), gpu, np.float64, dev)
        h = _out((n, nq, 3), gpu, np.float64, dev) if with_entropies and self.kernel != "parzen" else None
        cnt = _out((n,), gpu, np.int64, dev) if with_entropies else None
        st = self._lib.mi_eval(self._h, T.ptr, n, Q.ptr, nq, _ptr(mi), _ptr(h), _ptr(cnt))
        self._check(st, allow_empty)
        return (mi, h, cnt) if with_entropies else mi

    def eval_q16(self, affines, q=(1.0,), with_entropies=False, allow_empty=True):
        A = _Arg(affines, np.int32)
        Q = _Arg(np.atleast_1d(np.asarray(q, dtype=np.float32)))
        n = int(np.prod(A.obj.shape) // 12)
        nq = int(np.asarray(q).size)
        gpu = A.on_gpu
        dev = A.obj.device if gpu else None
        mi = _out((n, nq), gpu, np.float64, dev)
        h = _out((n, nq, 3), gpu, np.float64, dev) if with_entropies else None
        cnt = _out((n,), gpu, np.int64, dev) if with_entropies else None
        st = self._lib.mi_eval_q16(self._h, A.ptr, n, Q.ptr, nq, _ptr(mi), _ptr(h), _ptr(cnt))
        self._check(st, allow_empty)
        return (mi, h, cnt) if with_entropies else mi

    def batch_eval(self, pair_of_transform, transforms, q=(1.0,), with_entropies=False, allow_empty=True):
        P = _Arg(pair_of_transform, np.int32)
        T = _Arg(transforms, np.float32)
        Q = _Arg(np.atleast_1d(np.asarray(q, dtype=np.float32)))
        n = int(np.prod(T.obj.shape) // self.nparams)
        nq = int(np.asarray(q).size)
        gpu = T.on_gpu
        dev = T.obj.device if gpu else None
        mi = _out((n, nq), gpu, np.float64, dev)
        h = _out((n, nq, 3), gpu, np.float64, dev) if with_entropies else None
        cnt = _out((n,), gpu, np.int64, dev) if with_entropies else None
        st = self._lib.mi_batch_eval(self._h, P.ptr, T.ptr, n, Q.ptr, nq, _ptr(mi), _ptr(h), _ptr(cnt))
        self._check(st, allow_empty)
        return (mi, h, cnt) if with_entropies else mi

    def grad(self, transforms, q=(1.0,), allow_empty=False):
        """Parzen MI (n x nq) and dMI/dparam (n x nq x nparams)."""
        T = _Arg(transforms, np.float32)
        Q = _Arg(np.atleast_1d(np.asarray(q, dtype=np.float32)))
        n = int(np.prod(T.obj.shape) // self.nparams)
        nq = int(np.asarray(q).size)
        gpu = T.on_gpu
        dev = T.obj.device if gpu else None
        mi = _out((n, nq), gpu, np.float64, dev)
        g = _out((n, nq, self.nparams), gpu, np.float64, dev)
        st = self._lib.mi_grad(self._h, T.ptr, n, Q.ptr, nq, _ptr(mi), _ptr(g))
        self._check(st, allow_empty)
        return mi, g

    def batch_grad(self, pair_of_transform, transforms, q=(1.0,), allow_empty=False):
        """Parzen MI (n x nq) and dMI/dparam (n x nq x nparams) over the pairs of a multi-pair Parzen
        context: transform t on pair pair_of_transform[t], one launch per kernel for all pairs."""
        P = _Arg(pair_of_transform, np.int32)
        T = _Arg(transforms, np.float32)
        Q = _Arg(np.atleast_1d(np.asarray(q, dtype=np.float32)))
        n = int(np.prod(T.obj.shape) // self.nparams)
        nq = int(np.asarray(q).size)
        gpu = T.on_gpu
        dev = T.obj.device if gpu else None
        mi = _out((n, nq), gpu, np.float64, dev)
        g = _out((n, nq, self.nparams), gpu, np.float64, dev)
        st = self._lib.mi_batch_grad(self._h, P.ptr, T.ptr, n, Q.ptr, nq, _ptr(mi), _ptr(g))
        self._check(st, allow_empty)
        return mi, g

    def hist(self, transforms=None, affines=None, pair=0, path=PATH_PLAIN):
        """Joint histograms (n x bins x bins uint32, row = fixed bin) -- test hook."""
        if (transforms is None) == (affines is None):
            raise ValueError("give exactly one of transforms and affines")
        src = _Arg(transforms, np.float32) if transforms is not None else _Arg(affines, np.int32)
        n = int(np.prod(src.obj.shape) // (self.nparams if transforms is not None else 12))
        B = self.bins[pair]
        out = np.empty((n, B, B), dtype=np.uint32)
        st = self._lib.mi_hist(self._h, pair, src.ptr if transforms is not None else None,
                               src.ptr if affines is not None else None, n, int(path), out.ctypes.data)
        self._check(st)
        return out

    def affine(self, transforms, pair=0):
        """(FP64 [A|b] n x 3 x 4, 16.16 n x 3 x 4, Jacobian n x 12 x nparams) from the library's host builder."""
        T = _Arg(transforms, np.float32)
        n = int(np.prod(T.obj.shape) // self.nparams)
        a = np.empty((n, 3, 4), np.float64)
        q = np.empty((n, 3, 4), np.int32)
        j = np.empty((n, 12, self.nparams), np.float64)
        st = self._lib.mi_affine(self._h, pair, T.ptr, n, a.ctypes.data, q.ctypes.data, j.ctypes.data)
        self._check(st)
        return a, q, j

    def fixed_bins(self, pair=0):
        out = np.empty(self.shapes[pair], dtype=np.uint8)
        self._check(self._lib.mi_fixed_bins(self._h, pair, out.ctypes.data))
        return out

    def resample(self, q16, moving_dtype=np.uint16, pair=0):
        q = np.ascontiguousarray(q16, dtype=np.int32).reshape(12)
        out = np.empty(self.shapes[pair], dtype=moving_dtype)
        self._check(self._lib.mi_resample(self._h, pair, q.ctypes.data, out.ctypes.data))
        return out

    def selected_variant(self, n, pair=0):
        return self._lib.mi_selected_variant(self._h, pair, int(n))

    def selected_config(self, n):
        """The configuration chosen for calls of n transforms: dict of variant, threads, ctas, tile_rows,
        tile_slabs (all -1 before the first such call)."""
        out = (ctypes.c_int * 5)()
        self._check(self._lib.mi_selected_config(self._h, int(n), ctypes.cast(out, ctypes.c_void_p)))
        return dict(zip(("variant", "threads", "ctas", "tile_rows", "tile_slabs"), list(out)))

    def last_kernel_ms(self):
        """(device ms of the main kernels of the last call, number of kernels it launched)."""
        ms = ctypes.c_float()
        nl = ctypes.c_int()
        self._check(self._lib.mi_last_kernel_ms(self._h, ctypes.byref(ms), ctypes.byref(nl)))
        return float(ms.value), int(nl.value)


def autotune_cache(path):
    """Record and replay the batched path's autotuned choices in the text file ``path`` (None: off)."""
    load().mi_autotune_cache(None if path is None else str(path).encode())


def eval_noalloc(fixed, moving, bins, transform, q=(1.0,), fixed_spacing=(1.0, 1.0, 1.0),
                 moving_spacing=(1.0, 1.0, 1.0), fixed_depth=None, moving_depth=None, stream=None, out=None):
    """Hard-binned MI of one transform through ``mi_eval_noalloc``, which allocates no device memory.

    For callers that may not allocate device memory where they evaluate the
    metric: code running inside a framework whose caching allocator owns the
    GPU's memory, services that fix their memory budget up front, loops that
    cannot afford cudaMalloc's implicit synchronisation.  ``fixed`` and
    ``moving`` are contiguous uint8/uint16 CUDA tensors on the current device,
    used in place (a non-contiguous tensor is rejected rather than copied).
    ``out`` may be a contiguous CUDA float64 tensor of at least nq elements on
    that device; otherwise a numpy array is returned.  ``stream`` defaults to
    torch's current stream.  All calls share one static device array: calls
    that overlap on the GPU race, so serialise them.
    """
    lib = load()
    torch = _torch()
    for name, v in (("fixed", fixed), ("moving", moving)):
        if not (_is_torch(v) and v.is_cuda):
            raise MIError(MI_EINVAL, f"{name} must be a CUDA tensor (mi_eval_noalloc makes no copy)")
        if not v.is_contiguous():
            raise MIError(MI_EINVAL, f"{name} must be contiguous (a copy would allocate)")
    dev = fixed.device
    if moving.device != dev:
        raise MIError(MI_EINVAL, "fixed and moving must be on the same device")
    fv, fa = _volume(fixed, fixed_spacing, fixed_depth)
    mv, ma = _volume(moving, moving_spacing, moving_depth)
    T = np.ascontiguousarray(np.asarray(transform, dtype=np.float32).reshape(9))
    Q = np.ascontiguousarray(np.atleast_1d(np.asarray(q, dtype=np.float32)))
    if out is not None:
        if not (_is_torch(out) and out.is_cuda and out.device == dev):
            raise MIError(MI_EINVAL, "out must be a CUDA tensor on the volumes' device")
        if out.dtype != torch.float64 or out.numel() < Q.size or not out.is_contiguous():
            raise MIError(MI_EINVAL, f"out must be a contiguous float64 tensor of at least {Q.size} elements")
        res = out
    else:
        res = np.empty(Q.size, dtype=np.float64)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    h = getattr(stream, "cuda_stream", stream)
    with torch.cuda.device(dev):
        st = lib.mi_eval_noalloc(ctypes.byref(fv), ctypes.byref(mv), int(bins), T.ctypes.data, Q.ctypes.data,
                                 int(Q.size), _ptr(res), ctypes.c_void_p(h) if h else None)
    if st not in (MI_OK, MI_EEMPTY):
        raise MIError(st, lib.mi_last_error(None).decode())
    return res


def mi_function():
    """torch.autograd.Function over the Parzen MI: ``MIFunction.apply(theta, ctx, q)``."""
    torch = _torch()

    class MIFunction(torch.autograd.Function):
        @staticmethod
        def forward(fctx, theta, ctx, q):
            mi, g = ctx.grad(theta.detach().to(torch.float32).contiguous(), q)
            fctx.save_for_backward(g if _is_torch(g) else torch.from_numpy(g))
            mi = mi if _is_torch(mi) else torch.from_numpy(mi)
            return mi.to(theta.device)

        @staticmethod
        def backward(fctx, grad_out):
            (g,) = fctx.saved_tensors
            g = g.to(grad_out.device)
            # (n, nq) x (n, nq, P) -> (n, P)
            gt = (grad_out.to(g.dtype).unsqueeze(-1) * g).sum(dim=1)
            return gt, None, None

    return MIFunction


__all__ = ["Context", "MIError", "load", "build", "version", "mi_function", "autotune_cache", "phantoms"]
