"""Registration: ascent on the MI (Eq. 3: T^ = argmax_T F_m(u(x), v(T(x)))).

The paper's registration loop (Fig. 1) feeds the metric's gradient to a
gradient-descent optimiser (Introduction) and, in its Discussion, proposes
mixing entropies from one histogram: the Tsallis gradient for the translation
parameters and the Shannon gradient for rotation and scale.  This module is
that loop: every iteration evaluates MI and dMI/dtheta for all starting poses
in one ``mi_grad`` call (the CUDA path) and takes an Adam step per pose on the
host.  ``register_kw`` is the Introduction's other optimiser, Kiefer-Wolfowitz
stochastic approximation, on the hard-binned metric itself, which has no
analytic gradient: central differences of shrinking step from one batched
evaluation of all poses' perturbations per iteration.  Parameters are (tx, ty,
tz mm; rx, ry, rz degrees; sx, sy, sz factors), or, for a context with
``transform="affine"``, the 12 entries of [M | t] (row-major, t in mm).
"""
from __future__ import annotations

import numpy as np

# default step sizes per parameter: 0.25 mm, 0.25 degree, 0.25 % scale
DEFAULT_LR = np.array([0.25, 0.25, 0.25, 0.25, 0.25, 0.25, 0.0025, 0.0025, 0.0025])
# for the general affine [M | t]: 0.0025 per matrix entry, 0.25 mm per translation
AFFINE_LR = np.array([0.0025, 0.0025, 0.0025, 0.25] * 3)
# columns of the translation parameters
TRANSLATION = {9: [0, 1, 2], 12: [3, 7, 11]}


def register(ctx, starts, q=1.0, q_translation=None, steps=150, lr=None, betas=(0.9, 0.999), eps=1e-12):
    """Gradient ascent on the Parzen MI from n starting poses at once.

    ctx: a Context created with kernel="parzen" (9 parameters, or 12 with transform="affine").
    starts: n x P starting parameters, P = ctx.nparams.
    q: exponent whose gradient drives all parameters (1 = Shannon), or, with
       ``q_translation`` set, all but the translation parameters; the
       translation parameters then follow the q_translation gradient.  Both
       come from one soft histogram per pose (one ``mi_grad`` call).
    lr: step sizes per parameter (default DEFAULT_LR, or AFFINE_LR for 12 parameters).
    Returns (final params n x P, MI history steps x n for q).
    """
    P = int(getattr(ctx, "nparams", 9))
    if P not in TRANSLATION:
        raise ValueError(f"unsupported parameter count {P}")
    theta = np.array(starts, dtype=np.float64).reshape(-1, P)
    qs = [float(q)] if q_translation is None else [float(q), float(q_translation)]
    lr = np.asarray((DEFAULT_LR if P == 9 else AFFINE_LR) if lr is None else lr, dtype=np.float64)
    tcols = TRANSLATION[P]
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    history = []
    for it in range(1, steps + 1):
        mi, g = ctx.grad(theta.astype(np.float32), qs, allow_empty=True)
        mi = np.asarray(mi)
        g = np.asarray(g)
        grad = g[:, 0, :].copy()
        if q_translation is not None:
            grad[:, tcols] = g[:, 1, tcols]
        grad = np.nan_to_num(grad)
        history.append(mi[:, 0].copy())
        m = betas[0] * m + (1 - betas[0]) * grad
        v = betas[1] * v + (1 - betas[1]) * grad * grad
        mhat = m / (1 - betas[0] ** it)
        vhat = v / (1 - betas[1] ** it)
        theta = theta + lr * mhat / (np.sqrt(vhat) + eps)  # ascent: MI is maximised
    return theta, np.array(history)


# Kiefer-Wolfowitz perturbations per parameter at the first iteration: 0.5 mm, 0.5 degree, 0.5 % scale
KW_C = np.array([0.5, 0.5, 0.5, 0.5, 0.5, 0.5, 0.005, 0.005, 0.005])
KW_C_AFFINE = np.array([0.005, 0.005, 0.005, 0.5] * 3)


def register_kw(ctx, starts, q=1.0, q_translation=None, steps=100, c=None, gamma=1.0 / 3.0, lr=None,
                betas=(0.9, 0.999), eps=1e-12):
    """Kiefer-Wolfowitz stochastic approximation on the hard-binned MI from n starting poses at once.

    Iteration k estimates dMI/dtheta_p of every pose by the central difference
    (F(theta + c_k e_p) - F(theta - c_k e_p)) / (2 c_k,p), c_k = c / k^gamma per
    parameter (the Kiefer-Wolfowitz gains: the difference step shrinks, so the
    estimate's bias vanishes), from one batched ``ctx.eval`` of the 2 P n
    perturbed transforms (every q from each transform's one histogram), and
    steps along it with the Adam update of ``register`` (lr per parameter).
    q / q_translation: as in ``register`` (the translation columns may follow
    another q's estimate).  ctx: a hard-path Context (or any object with
    ``nparams`` and ``eval(transforms, q)``).  A perturbed transform with no
    overlap counts as MI 0.  Returns (final params n x P, MI history steps x n
    for q: each pose's mean over its 2 P perturbed evaluations).
    """
    P = int(getattr(ctx, "nparams", 9))
    if P not in TRANSLATION:
        raise ValueError(f"unsupported parameter count {P}")
    theta = np.array(starts, dtype=np.float64).reshape(-1, P)
    n = theta.shape[0]
    qs = [float(q)] if q_translation is None else [float(q), float(q_translation)]
    c = np.asarray((KW_C if P == 9 else KW_C_AFFINE) if c is None else c, dtype=np.float64)
    lr = np.asarray((DEFAULT_LR if P == 9 else AFFINE_LR) if lr is None else lr, dtype=np.float64)
    tcols = TRANSLATION[P]
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    history = []
    eye = np.eye(P)
    for it in range(1, steps + 1):
        ck = c / it ** gamma
        # rows: pose i, parameter p, sign s (+ then -) -> index (i * P + p) * 2 + s
        T = theta[:, None, None, :] + np.stack([eye * ck, -eye * ck], 1)[None]  # n x P x 2 x P
        mi = np.asarray(ctx.eval(T.reshape(-1, P).astype(np.float32), qs)).reshape(n, P, 2, len(qs))
        mi = np.nan_to_num(mi)
        est = (mi[:, :, 0, :] - mi[:, :, 1, :]) / (2.0 * ck[None, :, None])  # n x P x nq
        grad = est[:, :, 0].copy()
        if q_translation is not None:
            grad[:, tcols] = est[:, tcols, 1]
        history.append(mi[:, :, :, 0].mean(axis=(1, 2)))
        m = betas[0] * m + (1 - betas[0]) * grad
        v = betas[1] * v + (1 - betas[1]) * grad * grad
        mhat = m / (1 - betas[0] ** it)
        vhat = v / (1 - betas[1] ** it)
        theta = theta + lr * mhat / (np.sqrt(vhat) + eps)  # ascent: MI is maximised
    return theta, np.array(history)


def pose_error(theta, truth):
    """Per pose: max |translation error| (mm), max |rotation error| (deg), max |scale error|."""
    d = np.abs(np.asarray(theta) - np.asarray(truth)[None, :])
    return d[:, 0:3].max(1), d[:, 3:6].max(1), d[:, 6:9].max(1)
