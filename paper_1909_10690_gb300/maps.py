"""Parameter-space maps of the metric and the ascent paths on them.

The paper's Methodology maps the metric over one transform family at a time
(translation, rotation or scale: three parameters, so the map is a 3D image,
e.g. 51^3 = 132651 evaluations of translations from -25 to 25 mm), and its
Results trace the paths a gradient method follows on those maps and the
regions that converge to the centre.  ``param_map`` evaluates such a grid
through the batched CUDA path; ``ascent_sinks`` follows discrete steepest
ascent from every grid point (host-side post-processing of the map).
"""
from __future__ import annotations

import numpy as np

FAMILIES = {"translation": (0, 1, 2), "rotation": (3, 4, 5), "scale": (6, 7, 8)}


def identity(scale: str = "factor") -> np.ndarray:
    """The identity transform's 9 parameters (scale factors 1, or zero-centred offsets 0)."""
    p = np.zeros(9, np.float32)
    if scale == "factor":
        p[6:] = 1.0
    return p


def axis_values(lo: float, hi: float, steps: int) -> np.ndarray:
    return np.linspace(lo, hi, steps, dtype=np.float64)


def grid(family: str, lo: float, hi: float, steps: int, base=None, scale: str = "factor") -> np.ndarray:
    """steps^3 x 9 transforms: the family's three parameters on a regular grid from lo to hi
    (inclusive, the same range on each axis), the others from ``base`` (identity by default).
    Row order is C order over (p0, p1, p2), p0 slowest."""
    idx = FAMILIES[family]
    b = identity(scale) if base is None else np.asarray(base, np.float32).reshape(9)
    v = axis_values(lo, hi, steps)
    g0, g1, g2 = np.meshgrid(v, v, v, indexing="ij")
    out = np.repeat(b[None], steps ** 3, axis=0)
    out[:, idx[0]] = g0.ravel()
    out[:, idx[1]] = g1.ravel()
    out[:, idx[2]] = g2.ravel()
    return out.astype(np.float32)


def param_map(ctx, family: str, lo: float, hi: float, steps: int, q=(1.0,), base=None, chunk: int = 32768):
    """The metric over the grid: an array (steps, steps, steps, nq) indexed like ``grid``.

    ctx is a hard-path Context; its own rotation / scale conventions apply to
    the parameters (the unit-ball rotation maps use ``rotation="versor"``,
    the zero-centred scale maps ``scale="offset"``).
    """
    if getattr(ctx, "nparams", 9) != 9:
        raise ValueError("parameter maps are over the families of the 9-parameter form (transform='params')")
    T = grid(family, lo, hi, steps, base, getattr(ctx, "scale", "factor"))
    out = np.empty((len(T), len(q)), np.float64)
    for s in range(0, len(T), chunk):
        out[s:s + chunk] = np.asarray(ctx.eval(T[s:s + chunk], list(q)))
    return out.reshape(steps, steps, steps, len(q))


def _neighbour_offsets():
    return [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]


def ascent_next(mi_map: np.ndarray, maximize: bool = True) -> np.ndarray:
    """For every grid point, the flat index of the point a discrete steepest-ascent step goes to:
    the best of its 26 neighbours if that is strictly better, else itself (a sink).  Ties between
    neighbours go to the first in (-1, -1, -1) ... (1, 1, 1) order; NaN counts as worst."""
    m = np.asarray(mi_map, np.float64)
    if m.ndim != 3:
        raise ValueError("expects one 3D map (select a q first)")
    v = np.where(np.isnan(m), -np.inf, m if maximize else -m)
    n0, n1, n2 = v.shape
    pad = np.pad(v, 1, constant_values=-np.inf)
    flat = np.arange(v.size).reshape(v.shape)
    best_val = v.copy()
    best_idx = flat.copy()
    for a, b, c in _neighbour_offsets():
        if (a, b, c) == (0, 0, 0):
            continue
        nv = pad[1 + a:1 + a + n0, 1 + b:1 + b + n1, 1 + c:1 + c + n2]
        better = nv > best_val
        if not better.any():
            continue
        i0 = np.clip(np.arange(n0) + a, 0, n0 - 1)[:, None, None]
        i1 = np.clip(np.arange(n1) + b, 0, n1 - 1)[None, :, None]
        i2 = np.clip(np.arange(n2) + c, 0, n2 - 1)[None, None, :]
        nidx = (i0 * n1 + i1) * n2 + i2
        best_val = np.where(better, nv, best_val)
        best_idx = np.where(better, nidx, best_idx)
    return best_idx.ravel()


def ascent_sinks(mi_map: np.ndarray, maximize: bool = True):
    """Follow discrete steepest ascent from every grid point to where it stops.

    Returns (sink, maxima): ``sink`` has the map's shape and holds the flat
    index of the local maximum each point's path ends at; ``maxima`` are the
    distinct sinks, sorted."""
    nxt = ascent_next(mi_map, maximize)
    s = nxt.copy()
    while True:  # pointer jumping: every round doubles the path length followed
        s2 = s[s]
        if np.array_equal(s2, s):
            break
        s = s2
    return s.reshape(np.shape(mi_map)), np.unique(s)


def capture_fraction(mi_map: np.ndarray, target, maximize: bool = True) -> float:
    """Fraction of grid points whose ascent path ends at ``target`` (a grid index triple)."""
    sink, _ = ascent_sinks(mi_map, maximize)
    t = np.ravel_multi_index(tuple(target), np.shape(mi_map))
    return float(np.mean(sink == t))


def ascent_path(mi_map: np.ndarray, start, maximize: bool = True) -> list:
    """The grid points (index triples) of the discrete ascent path from ``start`` to its sink."""
    nxt = ascent_next(mi_map, maximize)
    p = int(np.ravel_multi_index(tuple(start), np.shape(mi_map)))
    out = [p]
    while nxt[p] != p:
        p = int(nxt[p])
        out.append(p)
    return [tuple(int(x) for x in np.unravel_index(i, np.shape(mi_map))) for i in out]
