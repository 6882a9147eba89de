"""The C-ABI library builds, loads and exports every entry point include/mi.h declares (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mi.h")


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mi_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("mi_create", "mi_eval", "mi_grad", "mi_batch_create", "mi_batch_eval", "mi_destroy",
                 "mi_last_error", "mi_set_stream", "mi_hist"):
        assert must in names


def test_library_loads_and_exports_every_declared_symbol():
    import shutil

    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("nvcc not available")
    from paper_1909_10690_gb300 import _lib

    lib = _lib.load()
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert set(declared_symbols()) <= set(_lib.SIGNATURES)
    assert b"sm_103a" in lib.mi_version()


def test_options_default_and_error_without_device():
    import ctypes

    from paper_1909_10690_gb300 import _lib

    lib = _lib.load()
    o = _lib.MiOptions()
    lib.mi_options_default(ctypes.byref(o))
    assert (o.kernel, o.tsallis_form, o.log_bits, o.hist_variant, o.path, o.use_graphs, o.autotune, o.device,
            o.block_threads, o.rotation, o.scale, o.sample_fraction, o.sample_seed,
            o.transform, o.tile_rows, o.tile_slabs) == (0, 0, 0, -1, 0, 1, 1, -1, 0, 0, 0, 0.0, 0, 0, 0, 0)
    assert lib.mi_transform_size(None) == -1
    # invalid arguments are rejected before any device work
    h = ctypes.c_void_p()
    st = lib.mi_create(ctypes.byref(h), None, None, 32, None)
    assert st != 0 and not h.value
    assert lib.mi_last_error(None)
