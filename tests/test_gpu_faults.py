"""Failure handling without a GPU fault: simulated allocation failures through the mi_fault_alloc hook.

Every k-th device allocation of context creation and of the first calls on a
context is made to fail in turn; each must surface as MI_ENOMEM with a
message, leave no half-built context behind, and leave an existing context
giving the same results as before.  The hook is host-side: no kernel faults.
"""
import numpy as np
import pytest

import oracle
from paper_1909_10690_gb300 import phantoms

pytestmark = pytest.mark.gpu


@pytest.fixture
def fault(cuda_lib):
    lib = cuda_lib.load()
    yield lib.mi_fault_alloc
    lib.mi_fault_alloc(-1)


@pytest.mark.parametrize("kernel", ["hard", "parzen"])
def test_create_fails_cleanly_at_every_allocation(cuda_lib, fault, kernel):
    dt = np.float32 if kernel == "parzen" else np.uint16
    f, m = phantoms.head_pair(shape=(20, 22, 24), spacing=(1, 1, 1), seed=80, dtype=dt)
    kw = dict(bins=32, kernel=kernel) if kernel == "parzen" else dict(bins=32, fixed_depth=12, moving_depth=12)
    failures = 0
    for k in range(64):
        fault(k)
        try:
            ctx = cuda_lib.Context(f, m, **kw)
        except cuda_lib.MIError as e:
            assert e.status == cuda_lib.MI_ENOMEM, (k, e)
            failures += 1
            continue
        finally:
            fault(-1)
        ctx.close()
        break  # creation needed fewer than k + 1 allocations: every one of them has been failed once
    assert failures >= 3


def test_calls_fail_cleanly_and_the_context_stays_usable(cuda_lib, fault):
    f, m = phantoms.head_pair(shape=(24, 26, 28), spacing=(1, 1, 1), seed=81)
    ctx = cuda_lib.Context(f, m, bins=64, fixed_depth=12, moving_depth=12)
    prm = phantoms.random_transforms(40, seed=82, t_mm=3, r_deg=8, s_range=(0.95, 1.05))
    qs = [1.0, 1.5]
    want = oracle.mi_eval(f, m, 64, prm, qs, fixed_depth=12, moving_depth=12, nthreads=8)[0]
    tol = 1e-6 * np.maximum(np.abs(want), 1.0)
    for n in (1, 7, 40):  # each size grows the call's scratch buffers
        fault(0)
        with pytest.raises(cuda_lib.MIError) as e:
            ctx.eval(prm[:n], qs)
        assert e.value.status == cuda_lib.MI_ENOMEM
        fault(-1)
        assert np.all(np.abs(ctx.eval(prm[:n], qs) - want[:n]) <= tol[:n])
    pz = cuda_lib.Context(f.astype(np.float32) / 4095, m.astype(np.float32) / 4095, bins=32, kernel="parzen")
    mi0, g0 = pz.grad(prm[:3], qs)
    fault(0)
    with pytest.raises(cuda_lib.MIError) as e:
        pz.grad(prm[:20], qs)
    assert e.value.status == cuda_lib.MI_ENOMEM
    fault(-1)
    mi1, g1 = pz.grad(prm[:3], qs)
    np.testing.assert_array_equal(mi0, mi1)
    np.testing.assert_array_equal(g0, g1)


def test_drain_give_up_is_reported_and_the_context_recovers(cuda_lib):
    # 16-bit counters (MI_HV_U16) drain into the overflow table at 2^14 by a bounded compare-and-swap
    # loop; with its cap at 0 every drain gives up, the kernel flags it and finishes, and the call
    # reports MI_ECUDA.  A constant pair puts all 64000 voxels in one cell, so drains happen.
    lib = cuda_lib.load()
    f = np.full((40, 40, 40), 1000, np.uint16)
    ctx = cuda_lib.Context(f, f, bins=16, fixed_depth=12, moving_depth=12, hist_variant=cuda_lib.HV_U16,
                           path="batched")
    T = phantoms.identity_params(2)
    ok = ctx.eval(T, [1.0, 2.0])
    np.testing.assert_allclose(ok, 0.0, atol=1e-12)  # one cell: every entropy is 0
    try:
        assert lib.mi_fault_drain_cap(0) == cuda_lib.MI_OK
        with pytest.raises(cuda_lib.MIError) as e:
            ctx.eval(T, [1.0, 2.0])
        assert e.value.status == cuda_lib.MI_ECUDA and "drain" in str(e.value)
    finally:
        lib.mi_fault_drain_cap(1 << 16)
    np.testing.assert_array_equal(ctx.eval(T, [1.0, 2.0]), ok)
    assert lib.mi_fault_drain_cap(-1) == cuda_lib.MI_EINVAL
