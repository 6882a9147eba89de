"""Separate contexts on separate host threads.

A context is not thread-safe, but separate contexts are independent: each owns
its device buffers and a non-blocking stream, the library's shared state (the
autotune cache, its file) is behind a mutex, and error messages are per thread.
Here four threads each create their own contexts (so two autotune at once) and
call them repeatedly while the others run; every call must give what the same
kind of context gives when called alone (the library calls release the
interpreter lock, so the threads' kernels overlap on the device).
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from paper_1909_10690_gb300 import phantoms

pytestmark = pytest.mark.gpu

QS = [0.5, 1.0, 2.0]


def _make(cuda_lib, kind, f, m):
    if kind == "parzen":
        return cuda_lib.Context(f, m, bins=32, kernel="parzen", fixed_depth=12, moving_depth=12)
    return cuda_lib.Context(f, m, bins=64, fixed_depth=12, moving_depth=12, path=kind)


def _call(ctx, kind, prm):
    if kind == "parzen":
        mi, g = ctx.grad(prm, QS, allow_empty=True)
        return np.concatenate([mi.ravel(), g.ravel()])
    mi, h, cnt = ctx.eval(prm, QS, with_entropies=True)
    return np.concatenate([mi.ravel(), h.ravel(), cnt.ravel().astype(np.float64)])


def test_contexts_on_separate_threads_agree_with_single_threaded_calls(cuda_lib):
    f, m = phantoms.head_pair(shape=(40, 48, 56), spacing=(1, 1, 1), seed=70)
    prm = phantoms.random_transforms(300, seed=71, t_mm=5, r_deg=10, s_range=(0.93, 1.07))
    prm[::50, 0] = 500.0  # some transforms without overlap
    kinds = ["batched", "batched", "plain", "parzen"]
    want = {k: _call(_make(cuda_lib, k, f, m), k, prm) for k in set(kinds)}

    def worker(kind):
        ctx = _make(cuda_lib, kind, f, m)  # created in the thread: the two batched ones autotune concurrently
        return kind, [_call(ctx, kind, prm) for _ in range(4)]

    with ThreadPoolExecutor(max_workers=len(kinds)) as ex:
        results = list(ex.map(worker, kinds))
    for kind, outs in results:
        for out in outs:
            np.testing.assert_array_equal(out, outs[0])  # repeated calls of one context: bit for bit
            # against a context called alone: histograms are exact, and the FP64 reductions run in one
            # order whatever variant the autotuner picked
            np.testing.assert_allclose(out, want[kind], rtol=1e-12, atol=1e-14, equal_nan=True)
