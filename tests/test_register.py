"""Host logic of the registration loop (Adam ascent, mixed-entropy gradients) on an analytic metric.

A stand-in context returns, per q, a concave quadratic with a known maximum
and its exact gradient, so the loop's bookkeeping (parameter count, which
columns follow which q, ascent direction) is checked without a GPU.  The
CUDA metric itself is exercised by tests/test_gpu_register.py.
"""
import numpy as np
import pytest

from paper_1909_10690_gb300 import maps, register


class QuadraticContext:
    """'MI' for exponent q: -sum_k w_k (theta_k - target_q[k])^2."""

    def __init__(self, nparams, targets, w):
        self.nparams = nparams
        self.targets = {float(q): np.asarray(t, np.float64) for q, t in targets.items()}
        self.w = np.asarray(w, np.float64)
        self.calls = 0

    def grad(self, theta, qs, allow_empty=False):
        self.calls += 1
        th = np.asarray(theta, np.float64)
        mi = np.stack([-(self.w * (th - self.targets[float(q)]) ** 2).sum(1) for q in qs], 1)
        g = np.stack([-2.0 * self.w * (th - self.targets[float(q)]) for q in qs], 1)
        return mi, g


def _problem(P):
    if P == 9:
        shannon = np.array([1.0, -2.0, 0.5, 3.0, -4.0, 2.0, 1.03, 0.97, 1.01])
        w = np.array([1, 1, 1, 1, 1, 1, 1e4, 1e4, 1e4], np.float64)
        tol = np.array([0.6] * 6 + [0.006] * 3)
    else:
        shannon = np.array([1.02, 0.03, -0.01, 1.0, -0.02, 0.98, 0.04, -2.0, 0.01, 0.0, 1.03, 0.5])
        w = np.array([1e4, 1e4, 1e4, 1] * 3, np.float64)
        tol = np.array([0.006, 0.006, 0.006, 0.6] * 3)
    return shannon, w, tol


@pytest.mark.parametrize("P", [9, 12])
def test_ascent_reaches_the_maximum(P):
    target, w, tol = _problem(P)
    ctx = QuadraticContext(P, {1.0: target}, w)
    rng = np.random.default_rng(90)
    starts = target + rng.uniform(-1, 1, (6, P)) * np.where(w > 1, 0.05, 6.0)
    theta, hist = register.register(ctx, starts, q=1.0, steps=300)
    assert theta.shape == (6, P) and hist.shape == (300, 6) and ctx.calls == 300
    assert np.all(np.abs(theta - target) <= tol)
    assert np.all(hist[-1] > hist[0])  # ascent: the metric grew


@pytest.mark.parametrize("P", [9, 12])
def test_translation_follows_the_q_translation_gradient(P):
    # two optima: the translation columns must converge to the q_translation one, the rest to q's
    target, w, tol = _problem(P)
    other = target.copy()
    tcols = register.TRANSLATION[P]
    other[tcols] = [-3.0, 2.5, 4.0]
    ctx = QuadraticContext(P, {1.0: target, 1.5: other}, w)
    theta, _ = register.register(ctx, np.tile(target, (3, 1)), q=1.0, q_translation=1.5, steps=300)
    want = target.copy()
    want[tcols] = other[tcols]
    assert np.all(np.abs(theta - want) <= tol)


def test_parameter_maps_need_the_9_parameter_form():
    with pytest.raises(ValueError):
        maps.param_map(QuadraticContext(12, {1.0: np.zeros(12)}, np.ones(12)), "translation", -1, 1, 3)
