"""Acquisition geometry of the forward model, in FP64.

Sec. III: a projection index i in [0, MN) decodes to view m = floor(i/N) and
pixel n = i mod N; every pixel of view m is measured at time T_m and angle
theta_m. Rotating the object by theta is the same as rotating the
source-detector pair by -theta about the z axis (Sec. III). Appendix A: rays
run from the source to the pixel (parallel or cone beam) and are sampled at
equal spacing inside the cylindrical field of view; Appendix B item 1: the
sample coordinates are normalised to [-1, 1] with the min/max of that
cylinder.

Readings where the paper is silent: one ray per pixel (D = 1) through the
pixel centre; S samples per ray at the midpoints of S equal sub-intervals of
the FOV chord; at theta = 0 rays travel along +y, detector u runs along +x,
detector rows along +z; the cone source sits at (0, -SOD, 0) and the
detector plane at distance SDD from it. A ray that misses the FOV has
chord length 0 and starts at s0 = 0.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np


def decode(i, n_pixels: int, det_cols: int):
    """Sec. III: i = m*N + n with m = floor(i/N), n = i mod N; pixel n is
    (row, col) = (n div cols, n mod cols). Returns (m, row, col)."""
    i = np.asarray(i, dtype=np.int64)
    m = i // n_pixels
    n = i % n_pixels
    return m, n // det_cols, n % det_cols


def pixel_uv(geom, row, col):
    """Detector coordinates of pixel centres."""
    u = geom.det_off_u + (np.asarray(col, np.float64) + 0.5) * geom.det_pitch_u
    v = geom.det_off_v + (np.asarray(row, np.float64) + 0.5) * geom.det_pitch_v
    return u, v


def rotate_xy(vec, theta):
    """Rotate vectors [..., 3] by -theta about z: the source/detector frame
    of an object that has been rotated by +theta (Sec. III)."""
    c, s = np.cos(theta), np.sin(theta)
    a, b = vec[..., 0], vec[..., 1]
    out = np.empty_like(vec)
    out[..., 0] = a * c + b * s
    out[..., 1] = -a * s + b * c
    out[..., 2] = vec[..., 2]
    return out


def fov_chord(geom, o, d):
    """Interval [s0, s1] of o + s*d inside the cylindrical FOV
    (x^2 + y^2 <= R^2 and z0 <= z <= z1). Returns (s0, l) with l = s1 - s0,
    and (0, 0) for rays that miss."""
    R = geom.fov_r
    a = d[:, 0] ** 2 + d[:, 1] ** 2
    b = 2.0 * (o[:, 0] * d[:, 0] + o[:, 1] * d[:, 1])
    c = o[:, 0] ** 2 + o[:, 1] ** 2 - R * R
    disc = b * b - 4.0 * a * c
    ok = (disc > 0.0) & (a > 0.0)
    sq = np.sqrt(np.where(ok, disc, 0.0))
    a_safe = np.where(a > 0.0, a, 1.0)
    lo = (-b - sq) / (2.0 * a_safe)
    hi = (-b + sq) / (2.0 * a_safe)
    dz = d[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        za = (geom.fov_z0 - o[:, 2]) / dz
        zb = (geom.fov_z1 - o[:, 2]) / dz
    flat = dz == 0.0
    inside = (o[:, 2] >= geom.fov_z0) & (o[:, 2] <= geom.fov_z1)
    zlo = np.where(flat, np.where(inside, -np.inf, np.inf), np.minimum(za, zb))
    zhi = np.where(flat, np.where(inside, np.inf, -np.inf), np.maximum(za, zb))
    s0 = np.maximum(lo, zlo)
    s1 = np.minimum(hi, zhi)
    hit = ok & (s1 > s0)
    return np.where(hit, s0, 0.0), np.where(hit, s1 - s0, 0.0)


def rays_at(geom, theta, u, v):
    """Ray origin and unit direction for detector points (u, v) of a view at
    angle theta, in object coordinates."""
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    theta = np.broadcast_to(np.asarray(theta, np.float64), u.shape)
    o = np.zeros(u.shape + (3,))
    d = np.zeros(u.shape + (3,))
    if geom.beam == "parallel":
        o[..., 0] = u
        o[..., 2] = v
        d[..., 1] = 1.0
    elif geom.beam == "cone":
        o[..., 1] = -geom.sod
        dx, dy, dz = u, np.full_like(u, geom.sdd), v
        norm = np.sqrt(dx * dx + dy * dy + dz * dz)
        d[..., 0] = dx / norm
        d[..., 1] = dy / norm
        d[..., 2] = dz / norm
    else:
        raise ValueError(geom.beam)
    return rotate_xy(o, theta), rotate_xy(d, theta)


def rays(geom, idx):
    """Per projection index: origin o, direction d, chord start s0, chord
    length l, and time t. All FP64."""
    m, row, col = decode(idx, geom.n_pixels, geom.det_cols)
    u, v = pixel_uv(geom, row, col)
    o, d = rays_at(geom, geom.view_angle[m], u, v)
    s0, l = fov_chord(geom, o.reshape(-1, 3), d.reshape(-1, 3))
    return o.reshape(-1, 3), d.reshape(-1, 3), s0, l, geom.view_time[m].reshape(-1)


def sample_points(o, d, s0, l, S: int):
    """Appendix A: equally spaced samples on the chord; sample j sits at
    s0 + (j + 1/2) * l / S. Returns points [n, S, 3]."""
    j = (np.arange(S, dtype=np.float64) + 0.5) / S
    s = s0[:, None] + j[None, :] * l[:, None]
    return o[:, None, :] + s[..., None] * d[:, None, :]


def normalize(geom, P, t):
    """Appendix B item 1: map (t, z, y, x) to [-1, 1] with the min/max of
    the cylinder (x, y in [-R, R], z in [z0, z1]) and of the time range.
    P: [..., 3] as (x, y, z); t broadcastable to P[..., 0].
    Returns [..., 4] ordered (t, z, y, x)."""
    R = geom.fov_r
    out = np.empty(P.shape[:-1] + (4,))
    out[..., 0] = 2.0 * (np.broadcast_to(t, P.shape[:-1]) - geom.t0) / (geom.t1 - geom.t0) - 1.0
    out[..., 1] = 2.0 * (P[..., 2] - geom.fov_z0) / (geom.fov_z1 - geom.fov_z0) - 1.0
    out[..., 2] = 2.0 * (P[..., 1] + R) / (2.0 * R) - 1.0
    out[..., 3] = 2.0 * (P[..., 0] + R) / (2.0 * R) - 1.0
    return out


def voxel_pitch(det_pitch: float, sod: float, sdd: float) -> float:
    """Sec. V (Discussion): the reconstruction voxel is the detector pixel
    divided by the geometric magnification SDD/SOD."""
    return det_pitch / (sdd / sod)


# ------------------------------------------------- App. A forward model

def sample_spacing(geom) -> float:
    """App. A: the spacing of samples along a ray is the pixel size
    back-projected onto the object (through the rotation axis: times
    SOD/SDD for a cone beam) divided by the sub-pixel factor D."""
    pitch = min(geom.det_pitch_u, geom.det_pitch_v)
    if geom.beam == "cone":
        pitch *= geom.sod / geom.sdd
    return pitch / geom.subpixels


def subpixel_rays(geom, idx):
    """App. A: D x D rays per pixel, to the centres of its D x D sub-pixels;
    ray k of pixel p is sub-pixel (a, b) = (k div D, k mod D), a along the
    detector rows (v), b along the columns (u). Returns o, d, s0, l, t per
    ray, pixel-major ([n * D * D])."""
    D = geom.subpixels
    m, row, col = decode(idx, geom.n_pixels, geom.det_cols)
    a = (np.arange(D)[:, None] * np.ones((1, D))).reshape(-1)     # row sub-index
    b = (np.ones((D, 1)) * np.arange(D)[None, :]).reshape(-1)     # column sub-index
    u = geom.det_off_u + (col[:, None] + (b[None, :] + 0.5) / D) * geom.det_pitch_u
    v = geom.det_off_v + (row[:, None] + (a[None, :] + 0.5) / D) * geom.det_pitch_v
    theta = np.repeat(np.asarray(geom.view_angle)[m][:, None], D * D, axis=1)
    o, d = rays_at(geom, theta, u, v)
    o, d = o.reshape(-1, 3), d.reshape(-1, 3)
    s0, l = fov_chord(geom, o, d)
    t = np.repeat(np.asarray(geom.view_time)[m], D * D)
    return o, d, s0, l, t


def subpixel_counts(geom, l):
    """Samples per ray: the fewest equal sub-intervals of the chord no
    longer than the spacing, ceil(l / spacing); 0 for an empty chord."""
    n = np.ceil(np.asarray(l, np.float64) / sample_spacing(geom))
    return np.where(np.asarray(l) > 0, np.maximum(n, 1), 0).astype(np.int64)


def subpixel_samples(o, d, s0, l, n):
    """Midpoints of n[k] equal sub-intervals of each chord, concatenated ray
    by ray. Returns points [sum n, 3] and the ray of each sample."""
    ray = np.repeat(np.arange(len(n)), n)
    first = np.concatenate([[0], np.cumsum(n)[:-1]])
    j = np.arange(ray.size) - first[ray]
    s = s0[ray] + (j + 0.5) * l[ray] / n[ray]
    return o[ray] + s[:, None] * d[ray], ray
