"""Build and load the CUDA library (``libmi_gb300.so``) and declare its C ABI for ctypes.

The library is compiled in-tree for sm_103a with nvcc.  Loading fails loudly
if it is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
ROOT = os.path.dirname(PKG)
INCLUDE = os.path.join(ROOT, "include")
LIB_PATH = os.path.join(PKG, "libmi_gb300.so")
BUILD_DIR = os.path.join(PKG, "_build")
SOURCES = ["mi_api.cu", "mi_hard.cu", "mi_parzen.cu", "mi_noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

_lib = None
_lock = threading.Lock()


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _stale() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "mi.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every .cu source in parallel and link ``libmi_gb300.so`` (sm_103a)."""
    if not force and not _stale():
        return LIB_PATH
    nvcc = _nvcc()
    os.makedirs(BUILD_DIR, exist_ok=True)
    flags = ["-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
             "-I", INCLUDE, "-I", CSRC]
    extra = os.environ.get("MI_NVCC_FLAGS")
    if extra:
        flags += extra.split()

    def compile_one(src):
        obj = os.path.join(BUILD_DIR, src.replace(".cu", ".o"))
        cmd = [nvcc, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB_PATH + ".tmp"
    r = subprocess.run([nvcc, "-shared", *ARCH, "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"linking libmi_gb300.so failed:\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class MiVolume(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("dtype", ctypes.c_int), ("dims", ctypes.c_int * 3),
                ("bit_depth", ctypes.c_int), ("spacing_mm", ctypes.c_float * 3)]


class MiOptions(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("tsallis_form", ctypes.c_int), ("log_bits", ctypes.c_int),
                ("hist_variant", ctypes.c_int), ("path", ctypes.c_int), ("use_graphs", ctypes.c_int),
                ("autotune", ctypes.c_int), ("device", ctypes.c_int), ("block_threads", ctypes.c_int),
                ("rotation", ctypes.c_int), ("scale", ctypes.c_int), ("sample_fraction", ctypes.c_float),
                ("sample_seed", ctypes.c_uint), ("transform", ctypes.c_int), ("tile_rows", ctypes.c_int),
                ("tile_slabs", ctypes.c_int)]


# Symbols declared in include/mi.h, with their ctypes signatures.
_P = ctypes.c_void_p
_I = ctypes.c_int
SIGNATURES = {
    "mi_options_default": (None, [ctypes.POINTER(MiOptions)]),
    "mi_version": (ctypes.c_char_p, []),
    "mi_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(MiVolume), ctypes.POINTER(MiVolume), _I,
                       ctypes.POINTER(MiOptions)]),
    "mi_batch_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(MiVolume), ctypes.POINTER(MiVolume), _P, _I,
                             ctypes.POINTER(MiOptions)]),
    "mi_destroy": (None, [_P]),
    "mi_transform_size": (_I, [_P]),
    "mi_fault_alloc": (None, [_I]),
    "mi_fault_drain_cap": (_I, [_I]),
    "mi_last_error": (ctypes.c_char_p, [_P]),
    "mi_set_stream": (_I, [_P, _P]),
    "mi_eval": (_I, [_P, _P, _I, _P, _I, _P, _P, _P]),
    "mi_eval_q16": (_I, [_P, _P, _I, _P, _I, _P, _P, _P]),
    "mi_batch_eval": (_I, [_P, _P, _P, _I, _P, _I, _P, _P, _P]),
    "mi_grad": (_I, [_P, _P, _I, _P, _I, _P, _P]),
    "mi_batch_grad": (_I, [_P, _P, _P, _I, _P, _I, _P, _P]),
    "mi_hist": (_I, [_P, _I, _P, _P, _I, _I, _P]),
    "mi_affine": (_I, [_P, _I, _P, _I, _P, _P, _P]),
    "mi_fixed_bins": (_I, [_P, _I, _P]),
    "mi_resample": (_I, [_P, _I, _P, _P]),
    "mi_selected_variant": (_I, [_P, _I, _I]),
    "mi_selected_config": (_I, [_P, _I, _P]),
    "mi_autotune_cache": (None, [ctypes.c_char_p]),
    "mi_last_kernel_ms": (_I, [_P, _P, _P]),
    "mi_eval_noalloc": (_I, [ctypes.POINTER(MiVolume), ctypes.POINTER(MiVolume), _I, _P, _P, _I, _P, _P]),
}


def load(build_if_missing: bool = True):
    """Load the compiled library (building it first if needed) and return the ctypes handle."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing and _stale():
                build()
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library missing: {LIB_PATH} (run build())")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib
