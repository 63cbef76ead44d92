"""Seeded synthetic detectors, light-response truth and scintillation events.

This module feeds BOTH the FP64 oracle and the CUDA library with identical
inputs.  It holds none of the reconstruction arithmetic (no B-splines, no
likelihood, no search): it only lays out sensor arrays, evaluates the closed-
form light response used as the synthetic detector's truth, and draws events.

The paper (arXiv:1602.07247) publishes no dataset for this path; the gamma
camera and workbench data it mentions (Sec. 9) are not available, so every
workload is synthetic with the shapes of Sec. 5-6:
  * Anger-camera sensor arrays: hexagonal PMT arrays and square SiPM arrays
    (Sec. 3.3 array types);
  * a point source emitting E photons isotropically; the mean signal of
    sensor i is E * eta_i(x) (Sec. 6: an LRF is the mean signal versus source
    position); counts are Poisson, optionally with a normal single
    photo-electron response (Sec. 4.2.5).
The truth LRF is eta(r) = A / (1 + (r/r0)^2)^1.5 in the sensor plane and
A r0^2 d / (d^2 + r^2)^1.5 with d = r0 + z out of it.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

A_DEFAULT = 0.04
R0_DEFAULT = 40.0


# --------------------------------------------------------------------------
# sensor arrays
# --------------------------------------------------------------------------


def hex_array(rings: int, pitch: float) -> np.ndarray:
    """Hexagonal array: axial coordinates (i, j) with |i|, |j|, |i+j| <= rings.
    rings = 2, 3, 4, 5, 6 give 19, 37, 61, 91, 127 sensors."""
    pts = []
    for j in range(-rings, rings + 1):
        for i in range(-rings, rings + 1):
            if abs(i) <= rings and abs(j) <= rings and abs(i + j) <= rings:
                pts.append((pitch * (i + 0.5 * j), pitch * (np.sqrt(3.0) / 2.0) * j))
    return np.asarray(pts, dtype=np.float64)


def square_array(n: int, pitch: float) -> np.ndarray:
    """n x n square array centred on the origin, row-major (y outer)."""
    c = (np.arange(n) - (n - 1) / 2.0) * pitch
    yy, xx = np.meshgrid(c, c, indexing="ij")
    return np.stack([xx.ravel(), yy.ravel()], axis=1).astype(np.float64)


def sensor_gains(n: int, sigma: float, seed: int) -> np.ndarray:
    """Per-sensor relative gains g_i ~ N(1, sigma^2)."""
    if sigma == 0.0:
        return np.ones(n)
    return np.random.default_rng(seed).normal(1.0, sigma, size=n)


# --------------------------------------------------------------------------
# closed-form light response used as the synthetic truth
# --------------------------------------------------------------------------


def eta_axial(r, A: float = A_DEFAULT, r0: float = R0_DEFAULT):
    r = np.asarray(r, dtype=np.float64)
    return A / (1.0 + (r / r0) ** 2) ** 1.5


def eta_3d(r, z, A: float = A_DEFAULT, r0: float = R0_DEFAULT):
    r = np.asarray(r, dtype=np.float64)
    d = r0 + np.asarray(z, dtype=np.float64)
    return A * r0 * r0 * d / (d * d + r * r) ** 1.5


def truth_eta(sensor_xy: np.ndarray, gains: np.ndarray, pts: np.ndarray, A=A_DEFAULT, r0=R0_DEFAULT):
    """g_i * eta(|p_xy - X_i|, p_z) for every point p and sensor i: [n_pts, n_s]."""
    pts = np.asarray(pts, dtype=np.float64)
    dx = pts[:, None, 0] - sensor_xy[None, :, 0]
    dy = pts[:, None, 1] - sensor_xy[None, :, 1]
    r = np.sqrt(dx * dx + dy * dy)
    if pts.shape[1] > 2:
        v = eta_3d(r, pts[:, None, 2], A, r0)
    else:
        v = eta_axial(r, A, r0)
    return v * gains[None, :]


def grid_samples(n_int, lo, hi, per_interval: int = 4) -> np.ndarray:
    """Tensor grid with per_interval points per knot interval per axis,
    domain edges included: [n_pts, dim] (x fastest)."""
    axes = [np.linspace(lo[a], hi[a], per_interval * n_int[a] + 1) for a in range(len(n_int))]
    mesh = np.meshgrid(*axes[::-1], indexing="ij")
    return np.stack([m.ravel() for m in mesh[::-1]], axis=1)


# --------------------------------------------------------------------------
# events
# --------------------------------------------------------------------------


@dataclass
class Events:
    signals: np.ndarray  # [n, n_s] float32
    xyz: np.ndarray      # [n, 3] float64 true source positions
    energy: np.ndarray   # [n] float64 true photon numbers


def draw_events(sensor_xy, gains, n: int, seed: int, *, region: str, extent: float,
                e0: float, e_spread: float = 0.05, z_range=None, spe_sigma: float = 0.0,
                A=A_DEFAULT, r0=R0_DEFAULT, chunk: int = 1 << 18) -> Events:
    """n point-source events.  region 'disk' (radius extent) or 'square'
    (|x|, |y| <= extent); E ~ e0 * U(1 - e_spread, 1 + e_spread); z uniform in
    z_range when given.  Counts n_i ~ Poisson(E eta_i); with spe_sigma > 0
    each photo-electron contributes N(1, spe_sigma^2), drawn as the exact sum
    n + spe_sigma sqrt(n) z, clamped at 0."""
    rng = np.random.default_rng(seed)
    if region == "disk":
        rad = extent * np.sqrt(rng.random(n))
        ang = 2.0 * np.pi * rng.random(n)
        x, y = rad * np.cos(ang), rad * np.sin(ang)
    elif region == "square":
        x = rng.uniform(-extent, extent, n)
        y = rng.uniform(-extent, extent, n)
    else:
        raise ValueError(region)
    z = rng.uniform(z_range[0], z_range[1], n) if z_range is not None else np.zeros(n)
    E = e0 * rng.uniform(1.0 - e_spread, 1.0 + e_spread, n)
    xyz = np.stack([x, y, z], axis=1)
    n_s = sensor_xy.shape[0]
    sig = np.empty((n, n_s), dtype=np.float32)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        pts = xyz[a:b] if z_range is not None else xyz[a:b, :2]
        mu = E[a:b, None] * truth_eta(sensor_xy, gains, pts, A, r0)
        cnt = rng.poisson(mu).astype(np.float64)
        if spe_sigma > 0.0:
            cnt = np.maximum(cnt + spe_sigma * np.sqrt(cnt) * rng.standard_normal(cnt.shape), 0.0)
        sig[a:b] = cnt.astype(np.float32)
    return Events(signals=sig, xyz=xyz, energy=E)
