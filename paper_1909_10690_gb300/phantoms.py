"""Seeded synthetic volumes and transform sets (inputs only).

The paper measures on Human Connectome Project 3T structural brain images
(Methodology), which are not available here; these phantoms stand in for
them.  This module draws inputs only: it renders analytic ellipsoid
geometry, adds noise and draws transform parameters.  It holds none of the
method's arithmetic (no resampling, binning, histogram or entropy), so the
oracle and the CUDA path can both consume its outputs.

Conventions shared with the method's transform (so that a moving phantom
rendered under a known motion is recovered by that motion's parameters):
parameters are (tx, ty, tz mm; rx, ry, rz degrees; sx, sy, sz factors); the
motion maps a fixed physical point p to R diag(s) (p - c_f) + c_m + t with
R = Rz Ry Rx and c the volume centres.  Volumes are numpy arrays indexed
[z, y, x]; spacings are given as (x, y, z) in mm.
"""
from __future__ import annotations

import numpy as np


def _rot(rx: float, ry: float, rz: float) -> np.ndarray:
    a, b, c = np.deg2rad([rx, ry, rz])
    Rx = np.array([[1, 0, 0], [0, np.cos(a), -np.sin(a)], [0, np.sin(a), np.cos(a)]])
    Ry = np.array([[np.cos(b), 0, np.sin(b)], [0, 1, 0], [-np.sin(b), 0, np.cos(b)]])
    Rz = np.array([[np.cos(c), -np.sin(c), 0], [np.sin(c), np.cos(c), 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def motion_matrix(params) -> tuple[np.ndarray, np.ndarray]:
    """Linear part L = R diag(s) and translation t (mm) of a 9-parameter motion."""
    p = np.asarray(params, dtype=np.float64)
    return _rot(*p[3:6]) @ np.diag(p[6:9]), p[0:3]


class Ellipsoid:
    """Solid ellipsoid {x : (x - c)^T Q (x - c) <= 1} in physical mm (x, y, z order)."""

    def __init__(self, centre, semi_axes, rotation=None):
        R = np.eye(3) if rotation is None else np.asarray(rotation, dtype=np.float64)
        D = np.diag(1.0 / np.asarray(semi_axes, dtype=np.float64) ** 2)
        self.c = np.asarray(centre, dtype=np.float64)
        self.Q = R @ D @ R.T

    def moved(self, L, t, c_from, c_to) -> "Ellipsoid":
        """Image of the ellipsoid under y = L (x - c_from) + c_to + t."""
        e = Ellipsoid.__new__(Ellipsoid)
        e.c = L @ (self.c - c_from) + c_to + t
        Li = np.linalg.inv(L)
        e.Q = Li.T @ self.Q @ Li
        return e

    def scaled(self, f: float) -> "Ellipsoid":
        e = Ellipsoid.__new__(Ellipsoid)
        e.c = self.c.copy()
        e.Q = self.Q / (f * f)
        return e


def _paint(label: np.ndarray, ell: Ellipsoid, value: int, spacing) -> None:
    """label[inside ell] = value, evaluated over the ellipsoid's bounding box, slab by slab."""
    nz, ny, nx = label.shape
    half = np.sqrt(np.diag(np.linalg.inv(ell.Q)))  # half-extent of the bounding box along x, y, z (mm)
    lo = np.floor((ell.c - half) / np.asarray(spacing)).astype(int) - 1
    hi = np.ceil((ell.c + half) / np.asarray(spacing)).astype(int) + 2
    x0, y0, z0 = (max(0, v) for v in lo)
    x1, y1, z1 = min(nx, hi[0]), min(ny, hi[1]), min(nz, hi[2])
    if x0 >= x1 or y0 >= y1 or z0 >= z1:
        return
    Q = ell.Q.astype(np.float32)
    dx = (np.arange(x0, x1, dtype=np.float32) * np.float32(spacing[0]) - np.float32(ell.c[0]))[None, None, :]
    dy = (np.arange(y0, y1, dtype=np.float32) * np.float32(spacing[1]) - np.float32(ell.c[1]))[None, :, None]
    for zs in range(z0, z1, 16):
        ze = min(z1, zs + 16)
        dz = (np.arange(zs, ze, dtype=np.float32) * np.float32(spacing[2]) - np.float32(ell.c[2]))[:, None, None]
        f = (Q[0, 0] * dx * dx + Q[1, 1] * dy * dy + Q[2, 2] * dz * dz
             + 2 * Q[0, 1] * dx * dy + 2 * Q[0, 2] * dx * dz + 2 * Q[1, 2] * dy * dz)
        label[zs:ze, y0:y1, x0:x1][f <= 1.0] = value


def _centre(shape, spacing) -> np.ndarray:
    nz, ny, nx = shape
    return np.array([(nx - 1) / 2 * spacing[0], (ny - 1) / 2 * spacing[1], (nz - 1) / 2 * spacing[2]])


def _random_rotation(rng) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


# ---------------------------------------------------------------------------
# Tiny ellipsoid phantom (64^3 uint8)
# ---------------------------------------------------------------------------

TINY_MOTION = (3.0, -2.0, 1.0, 0.0, 0.0, 5.0, 1.0, 1.0, 1.0)


def ellipsoid_pair(shape=(64, 64, 64), seed=1, motion=TINY_MOTION, noise_sigma=4.0):
    """Fixed and moving uint8 phantoms: five random ellipsoids painted in order
    with intensities 40/90/140/190/240 on a 0 background plus N(0, sigma^2)
    noise (round half-even, clipped to 0..255).  The moving phantom shows the
    same ellipsoids moved by ``motion`` (spacing 1 mm, so mm = voxels) with an
    independent noise draw.  Returns (fixed, moving) indexed [z, y, x].
    """
    rng = np.random.default_rng(seed)
    spacing = (1.0, 1.0, 1.0)
    n = np.array(shape[::-1], dtype=np.float64)
    ells = []
    for _ in range(5):
        c = (0.2 + 0.6 * rng.random(3)) * (n - 1)
        ax = rng.uniform(6, 20, size=3)
        ells.append(Ellipsoid(c, ax, _random_rotation(rng)))
    L, t = motion_matrix(motion)
    cen = _centre(shape, spacing)
    out = []
    for which in range(2):
        label = np.zeros(shape, dtype=np.uint8)
        for e, v in zip(ells, (40, 90, 140, 190, 240)):
            _paint(label, e if which == 0 else e.moved(L, t, cen, cen), v, spacing)
        vol = label.astype(np.float64) + rng.normal(0.0, noise_sigma, size=shape)
        out.append(np.clip(np.rint(vol), 0, 255).astype(np.uint8))
    return out[0], out[1]


# ---------------------------------------------------------------------------
# Head-like multimodal pair (layered ellipsoids, Rician noise)
# ---------------------------------------------------------------------------

BACKGROUND, SKULL, CSF, GM, WM = 0, 1, 2, 3, 4
HEAD_MOTION = (6.0, -4.0, 3.0, 4.0, -3.0, 6.0, 1.04, 0.97, 1.02)


def _head_labels(shape, spacing, rng, motion=None):
    """Label volume of a layered-ellipsoid head (skull / CSF / GM / WM plus
    ventricles), optionally moved by ``motion`` about the volume centre."""
    cen = _centre(shape, spacing)
    ext = np.array(shape[::-1], dtype=np.float64) * np.asarray(spacing)
    head = Ellipsoid(cen + rng.uniform(-0.02, 0.02, 3) * ext, ext * np.array([0.36, 0.42, 0.40]),
                     _rot(*rng.uniform(-6, 6, 3)))
    layers = [(head, SKULL), (head.scaled(0.90), CSF), (head.scaled(0.86), GM), (head.scaled(0.70), WM)]
    for _ in range(3):
        c = head.c + rng.uniform(-0.12, 0.12, 3) * ext
        layers.append((Ellipsoid(c, rng.uniform(0.03, 0.08, 3) * ext, _random_rotation(rng)), CSF))
    for _ in range(4):
        c = head.c + rng.uniform(-0.2, 0.2, 3) * ext
        layers.append((Ellipsoid(c, rng.uniform(0.03, 0.06, 3) * ext, _random_rotation(rng)), GM))
    label = np.zeros(shape, dtype=np.uint8)
    if motion is not None:
        L, t = motion_matrix(motion)
    for e, v in layers:
        _paint(label, e if motion is None else e.moved(L, t, cen, cen), v, spacing)
    return label


def _rician(mean: np.ndarray, sigma: float, rng) -> np.ndarray:
    """Magnitude of a complex Gaussian around ``mean`` (float32 draws)."""
    s = np.float32(sigma)
    a = rng.standard_normal(size=mean.shape, dtype=np.float32)
    a *= s
    a += mean.astype(np.float32, copy=False)
    b = rng.standard_normal(size=mean.shape, dtype=np.float32)
    b *= s
    a *= a
    b *= b
    a += b
    return np.sqrt(a, out=a)


def head_pair(shape=(160, 256, 256), spacing=(1.0, 1.0, 1.2), depth=12, seed=2, motion=HEAD_MOTION,
              noise=0.02, dtype=np.uint16):
    """Multimodal head-like pair.

    Fixed: T1-like class means (WM brightest) drawn per class; moving: a
    non-monotonic T2-like remap (CSF brightest, WM darkest, skull dark) of the
    same anatomy moved by ``motion``.  Rician noise of ``noise`` x full scale.
    Values are integers of bit depth ``depth`` in ``dtype`` (or float32 in
    [0, 1] when dtype is float32).  Returns (fixed, moving).
    """
    rng = np.random.default_rng(seed)
    full = float((1 << depth) - 1) if dtype != np.float32 else 4095.0
    lab_f = _head_labels(shape, spacing, np.random.default_rng(seed + 1000))
    lab_m = _head_labels(shape, spacing, np.random.default_rng(seed + 1000), motion=motion)
    t1 = np.array([0.0, rng.uniform(0.08, 0.15), rng.uniform(0.15, 0.25), rng.uniform(0.45, 0.55),
                   rng.uniform(0.70, 0.80)]) * full
    t2 = np.array([0.0, rng.uniform(0.05, 0.10), rng.uniform(0.80, 0.90), rng.uniform(0.50, 0.60),
                   rng.uniform(0.30, 0.38)]) * full
    out = []
    for lab, means in ((lab_f, t1), (lab_m, t2)):
        vol = _rician(means.astype(np.float32)[lab], noise * full, rng)
        if dtype == np.float32:
            out.append(np.clip(vol / full, 0.0, 1.0).astype(np.float32))
        else:
            out.append(np.clip(np.rint(vol), 0, full).astype(dtype))
    return out[0], out[1]


# ---------------------------------------------------------------------------
# Transform sets
# ---------------------------------------------------------------------------

def identity_params(n: int = 1) -> np.ndarray:
    p = np.zeros((n, 9), dtype=np.float32)
    p[:, 6:9] = 1.0
    return p


def random_transforms(n: int, seed: int = 3, t_mm: float = 15.0, r_deg: float = 20.0,
                      s_range=(0.85, 1.15)) -> np.ndarray:
    """n x 9 float32: translation U(+-t_mm), rotation U(+-r_deg), scale U(s_range)."""
    rng = np.random.default_rng(seed)
    p = np.empty((n, 9), dtype=np.float32)
    p[:, 0:3] = rng.uniform(-t_mm, t_mm, (n, 3))
    p[:, 3:6] = rng.uniform(-r_deg, r_deg, (n, 3))
    p[:, 6:9] = rng.uniform(s_range[0], s_range[1], (n, 3))
    return p


def sweep(param: int, lo: float, hi: float, steps: int, base=None) -> np.ndarray:
    """steps x 9 transforms varying one parameter linearly from lo to hi."""
    p = np.repeat(identity_params(1) if base is None else np.asarray(base, np.float32)[None], steps, axis=0)
    p[:, param] = np.linspace(lo, hi, steps, dtype=np.float64).astype(np.float32)
    return p


def head_sweeps(steps: int = 81) -> np.ndarray:
    """One-parameter sweeps on each of the 9 parameters: translation +-20 mm,
    rotation +-30 degrees, scale 0.8..1.2 (9 x steps transforms)."""
    out = []
    for a in range(3):
        out.append(sweep(a, -20.0, 20.0, steps))
    for a in range(3):
        out.append(sweep(3 + a, -30.0, 30.0, steps))
    for a in range(3):
        out.append(sweep(6 + a, 0.8, 1.2, steps))
    return np.concatenate(out)


def tiny_sweep() -> np.ndarray:
    """The tiny workload's transforms: the true motion plus a 21-point x sweep (-10..10 voxels)."""
    return np.concatenate([np.asarray(TINY_MOTION, np.float32)[None], sweep(0, -10.0, 10.0, 21)])


def uneven_specs(n_pairs: int = 48, seed: int = 5):
    """Size, type and bin count of each pair of the uneven batch: dims per axis
    U[96, 320] x U[96, 320] x U[96, 200] with 96^3 and 320x320x200 forced in,
    half uint8 and half uint16 12-bit, bins from {32, 64, 128}."""
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(n_pairs):
        if i == 0:
            nx, ny, nz = 96, 96, 96
        elif i == 1:
            nx, ny, nz = 320, 320, 200
        else:
            nx, ny, nz = int(rng.integers(96, 321)), int(rng.integers(96, 321)), int(rng.integers(96, 201))
        u8 = (i % 2 == 0)
        specs.append({"shape": (nz, ny, nx), "dtype": np.uint8 if u8 else np.uint16, "depth": 8 if u8 else 12,
                      "bins": int(rng.choice([32, 64, 128])), "seed": 100 + i})
    return specs
