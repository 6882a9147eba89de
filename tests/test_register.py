"""Host logic of the registration loops (Adam ascent on gradients, Kiefer-Wolfowitz
on differences) on an analytic metric, and Kiefer-Wolfowitz on the oracle's hard MI.

A stand-in context returns, per q, a concave quadratic with a known maximum
and its exact gradient, so the loops' bookkeeping (parameter count, which
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

    def eval(self, theta, qs, **_):
        self.calls += 1
        th = np.asarray(theta, np.float64).reshape(-1, self.nparams)
        return np.stack([-(self.w * (th - self.targets[float(q)]) ** 2).sum(1) for q in qs], 1)


class StaircaseContext(QuadraticContext):
    """The quadratic rounded to steps of 1e-3: piecewise constant like a binned MI in theta."""

    def eval(self, theta, qs, **_):
        return np.round(super().eval(theta, qs) * 1e3) / 1e3


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


@pytest.mark.parametrize("P", [9, 12])
def test_kiefer_wolfowitz_reaches_the_maximum(P):
    target, w, tol = _problem(P)
    ctx = QuadraticContext(P, {1.0: target}, w)
    rng = np.random.default_rng(91)
    starts = target + rng.uniform(-1, 1, (5, P)) * np.where(w > 1, 0.05, 6.0)
    theta, hist = register.register_kw(ctx, starts, q=1.0, steps=300)
    # one batched evaluation of 2 P perturbations per pose per iteration
    assert theta.shape == (5, P) and hist.shape == (300, 5) and ctx.calls == 300
    assert np.all(np.abs(theta - target) <= tol)
    assert np.all(hist[-1] > hist[0])


def test_kiefer_wolfowitz_translation_follows_q_translation():
    target, w, tol = _problem(9)
    other = target.copy()
    other[:3] = [-3.0, 2.5, 4.0]
    ctx = QuadraticContext(9, {1.0: target, 1.5: other}, w)
    theta, _ = register.register_kw(ctx, np.tile(target, (3, 1)), q=1.0, q_translation=1.5, steps=300)
    want = target.copy()
    want[:3] = other[:3]
    assert np.all(np.abs(theta - want) <= tol)


def test_kiefer_wolfowitz_climbs_a_piecewise_constant_metric():
    """Differences of a staircase vanish inside a step; the perturbation c_k spans several steps
    early on and the Adam normalisation keeps the ascent moving where single differences are 0."""
    target, w, tol = _problem(9)
    ctx = StaircaseContext(9, {1.0: target}, w)
    rng = np.random.default_rng(92)
    starts = target + rng.uniform(-1, 1, (4, 9)) * np.where(w > 1, 0.04, 4.0)
    theta, _ = register.register_kw(ctx, starts, steps=300)
    assert np.all(np.abs(theta - target) <= tol)


def test_kiefer_wolfowitz_registers_on_the_oracle_hard_mi():
    """The hard-binned MI of the oracle (Eq. 2, no gradient) drives Kiefer-Wolfowitz back to the
    known motion of a small ellipsoid pair."""
    import oracle
    from paper_1909_10690_gb300 import phantoms

    f, m = phantoms.ellipsoid_pair(shape=(40, 40, 40), seed=1)

    class OracleHard:
        nparams = 9

        def eval(self, T, qs):
            return oracle.mi_eval(f, m, 32, T, qs, nthreads=4)[0]

    truth = np.array(phantoms.TINY_MOTION, np.float64)
    rng = np.random.default_rng(93)
    d = np.concatenate([rng.uniform(-2, 2, (3, 3)), rng.uniform(-4, 4, (3, 3)), rng.uniform(-0.02, 0.02, (3, 3))], 1)
    theta, hist = register.register_kw(OracleHard(), truth[None] + d, steps=50)
    et, er, es = register.pose_error(theta, truth)
    assert np.all(et < 0.5) and np.all(er < 1.5) and np.all(es < 0.02), (et, er, es)
    assert np.all(hist[-1] > hist[0])
