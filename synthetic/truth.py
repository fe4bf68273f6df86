"""Ground truth of the synthetic phantoms, for scoring reconstructions.

The attenuation of a phantom (sum of the attenuations of the ellipsoids
that contain a point, centres c0 + v t, semi-axes a0 (1 + growth t)) on a
regular grid of cell centres over [-1, 1]^3, and the mask of cells inside the
field of view (the cylinder x^2 + y^2 <= 1, |z| <= 1) where the data
constrain the reconstruction. This is the data generator's own field, not
part of the reconstruction method.
"""
from __future__ import annotations

import numpy as np


def grid_axis(n: int) -> np.ndarray:
    """Cell centres of n equal cells over [-1, 1]."""
    return -1.0 + (np.arange(n) + 0.5) * (2.0 / n)


def attenuation_grid(ph, t: float, n: int = 64) -> np.ndarray:
    """Phantom attenuation at time t on the n^3 grid, indexed [z, y, x]."""
    ax = grid_axis(n)
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    P = np.stack([X, Y, Z], axis=-1).reshape(-1, 3)
    out = np.zeros(len(P))
    for c0, a0, rho, v in zip(ph.centre, ph.axes, ph.rho, ph.vel):
        c = c0 + v * t
        a = a0 * (1.0 + ph.growth * t)
        q = (P - c) / a
        out += rho * ((q * q).sum(-1) <= 1.0)
    return out.reshape(n, n, n)


def fov_mask(n: int = 64) -> np.ndarray:
    """Cells of the n^3 grid inside the cylindrical field of view."""
    ax = grid_axis(n)
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    return X * X + Y * Y <= 1.0


def scores(rec: np.ndarray, truth: np.ndarray, mask: np.ndarray) -> dict:
    """Relative L2 error and PSNR (peak = the truth's maximum) over the mask."""
    r, g = rec[mask], truth[mask]
    mse = float(np.mean((r - g) ** 2))
    return {"rel_l2": float(np.linalg.norm(r - g) / np.linalg.norm(g)),
            "psnr_db": float(10.0 * np.log10(g.max() ** 2 / mse)) if mse > 0 else float("inf")}
