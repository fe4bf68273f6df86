"""Closed-form line integrals used to generate measurements and to pin the
ray geometry, in FP64.

The measured projection of a ray is the line integral of the object's
attenuation over the part of the ray inside the cylindrical FOV (Sec. III:
only coordinates inside the FOV contribute). For an ellipsoid of constant
attenuation rho the integral is rho times the length of the intersection of
two intervals: the ray's chord through the ellipsoid (roots of a quadratic)
and the ray's chord through the FOV. Overlapping ellipsoids add.

A phantom ellipsoid k at time t has centre c_k + v_k t and semi-axes
a_k (1 + g t) (readings of the synthetic workloads: linear growth by 50 %
over t in [0, 1] and constant velocity).

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import math

import numpy as np

from . import geometry


def ellipsoids_at(ph, t):
    """Centres and semi-axes at times t [n]: arrays [n, k, 3]."""
    t = np.asarray(t, np.float64)[:, None, None]
    c = ph.centre[None] + ph.vel[None] * t
    a = ph.axes[None] * (1.0 + ph.growth * t)
    return c, a


def ellipsoid_intervals(ph, t, o, d):
    """Per ray and ellipsoid, the interval [e0, e1] of s where o + s d is
    inside the ellipsoid; empty intervals have e1 <= e0."""
    c, a = ellipsoids_at(ph, t)
    q = (o[:, None, :] - c) / a
    r = d[:, None, :] / a
    A = (r * r).sum(-1)
    B = 2.0 * (q * r).sum(-1)
    C = (q * q).sum(-1) - 1.0
    disc = B * B - 4.0 * A * C
    sq = np.sqrt(np.maximum(disc, 0.0))
    e0 = np.where(disc > 0.0, (-B - sq) / (2.0 * A), 0.0)
    e1 = np.where(disc > 0.0, (-B + sq) / (2.0 * A), 0.0)
    return e0, e1


def line_integrals(ph, t, o, d, s0, l):
    """Exact integral over [s0, s0 + l] of the phantom along o + s d."""
    e0, e1 = ellipsoid_intervals(ph, t, o, d)
    lo = np.maximum(e0, s0[:, None])
    hi = np.minimum(e1, (s0 + l)[:, None])
    return (ph.rho[None, :] * np.maximum(hi - lo, 0.0)).sum(axis=1)


def projections(ph, geom, idx):
    """Noise-free measured projections p_i of the phantom for indices idx,
    each ray at its view's time."""
    o, d, s0, l, t = geometry.rays(geom, idx)
    return line_integrals(ph, t, o, d, s0, l)


def density(ph, P, t):
    """Attenuation of the phantom at points P [n, S, 3] and times t [n]."""
    c, a = ellipsoids_at(ph, t)
    q = (P[:, :, None, :] - c[:, None]) / a[:, None]
    inside = (q * q).sum(-1) <= 1.0
    return (inside * ph.rho[None, None, :]).sum(-1)


def project_field(field, geom, idx, S):
    """Midpoint rule (l/S) sum_j f(P_j, t) over each ray's FOV chord, with an
    analytic field f(P [n,S,3], t [n]) -> [n, S] in place of the network."""
    o, d, s0, l, t = geometry.rays(geom, idx)
    P = geometry.sample_points(o, d, s0, l, S)
    return (l / S) * field(P, t).sum(axis=1)


def gaussian_blob_line(centre, sigma, o, d, s0, l):
    """Closed-form integral of exp(-|P - c|^2 / (2 sigma^2)) over
    [s0, s0 + l] along o + s d (d a unit vector):
    exp(-h^2/(2 sigma^2)) * sigma * sqrt(pi/2) * [erf(b) - erf(a)] where s*
    is the foot of the perpendicular from c and h its distance."""
    rel = np.asarray(centre)[None, :] - o
    s_star = (rel * d).sum(-1)
    h2 = (rel * rel).sum(-1) - s_star ** 2
    k = math.sqrt(2.0) * sigma
    erf = np.vectorize(math.erf)
    a = (s0 - s_star) / k
    b = (s0 + l - s_star) / k
    return np.exp(-h2 / (2 * sigma * sigma)) * sigma * math.sqrt(math.pi / 2) * (erf(b) - erf(a))
