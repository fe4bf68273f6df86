"""Pins of the oracle's App. A forward model (D x D sub-pixel rays per
pixel, samples about Delta/D apart): sub-ray placement, sample counts from
the closed-form chord, the uniform-field projection, the ellipsoid phantom
against exact chord integrals, and central differences of the loss."""
from dataclasses import replace

import numpy as np

from oracle import geometry, network, phantom as oph, step
from synthetic import workloads as wl


def _w():
    return wl.workload(9)


def test_subray_placement_and_counts():
    """At theta = 0 (view 0) a parallel ray enters at x = u, z = v: the
    sub-pixel centres; its chord is 2 sqrt(R^2 - u^2) and it carries
    ceil(l / (pitch / D)) samples."""
    w = _w()
    g = w.geom
    D = g.subpixels
    rows, cols = np.array([0, 5, 17, 31]), np.array([3, 16, 0, 31])
    idx = rows * g.det_cols + cols                      # view 0
    o, d, s0, l, t = geometry.subpixel_rays(g, idx)
    k = np.arange(len(idx) * D * D)
    pix, a, b = k // (D * D), (k % (D * D)) // D, k % D
    u = g.det_off_u + (cols[pix] + (b + 0.5) / D) * g.det_pitch_u
    v = g.det_off_v + (rows[pix] + (a + 0.5) / D) * g.det_pitch_v
    assert np.allclose(o[:, 0], u, atol=1e-14) and np.allclose(o[:, 2], v, atol=1e-14)
    assert np.allclose(l, 2 * np.sqrt(np.maximum(1 - u * u, 0)), atol=1e-12)
    n = geometry.subpixel_counts(g, l)
    delta = g.det_pitch_u / D
    assert geometry.sample_spacing(g) == delta
    assert np.array_equal(n, np.where(l > 0, np.maximum(np.ceil(l / delta), 1), 0))
    assert (l / np.maximum(n, 1) <= delta + 1e-15).all()


def test_uniform_field_projection():
    """M = 1 everywhere: p_bar_i = mu0 sum_k n_k l_k / sum_k n_k over the
    pixel's sub-rays (Eq. 1 with w = mu0 l)."""
    w = _w()
    g = replace(w.geom, mu0=0.7)
    idx = wl.ray_subset(g.n_proj, 40, 3)
    e, wt, pix, n_pix = step.subpixel_model(g, w.net, idx)
    p = step.forward_model_subpixel(np.ones(len(wt)), wt, pix, n_pix)
    _, _, _, l, _ = geometry.subpixel_rays(g, idx)
    n = geometry.subpixel_counts(g, l)
    D2 = g.subpixels ** 2
    want = 0.7 * (n * l).reshape(-1, D2).sum(1) / np.maximum(n.reshape(-1, D2).sum(1), 1)
    assert np.allclose(p, want, rtol=1e-13, atol=1e-15)


def test_ellipsoid_phantom_vs_exact_chords():
    """The phantom's density summed at the samples (spacing l/n) against the
    exact chord integrals of each sub-ray with the same weights: per ray
    the midpoint sum errs by at most one spacing per boundary crossing."""
    w = wl.workload(2)
    g = replace(w.geom, subpixels=2)
    ph = wl.phantom(w)
    idx = wl.ray_subset(g.n_proj, 60, 4)
    o, d, s0, l, t = geometry.subpixel_rays(g, idx)
    n = geometry.subpixel_counts(g, l)
    P, ray = geometry.subpixel_samples(o, d, s0, l, n)
    dens = oph.density(ph, P[:, None, :], t[ray])[:, 0]
    approx = np.bincount(ray, weights=dens * (l / np.maximum(n, 1))[ray], minlength=len(l))
    exact = oph.line_integrals(ph, t, o, d, s0, l)
    bound = (2 * ph.rho.sum() + 1e-12) * l / np.maximum(n, 1)
    assert (np.abs(exact - approx) <= bound + 1e-12).all()
    assert np.abs(exact - approx).max() < 0.1 * np.abs(exact).max()


def test_subpixel_loss_central_differences():
    w = _w()
    g, net = w.geom, replace(w.net, grff_c=8, width=16, hidden_layers=2)
    theta = wl.he_init(net, 5)
    idx = wl.ray_subset(g.n_proj, 6, 8)
    proj = np.random.default_rng(2).uniform(0, 1, g.n_proj)
    out = step.loss_and_grad(theta, g, net, idx, proj)
    ks = np.random.default_rng(9).choice(theta.size, 16, replace=False)
    for k in ks:
        fd = step.fd_grad(theta, g, net, idx, proj, k, h=1e-5)
        assert abs(fd - out["grad"][k]) <= 1e-7 * max(1e-3, np.abs(out["grad"]).max()), k


def test_cone_subrays_by_brute_force():
    """Cone beam, view 0 (theta = 0): each sub-ray starts at the source
    (0, -SOD, 0) and points at its sub-pixel centre (u, SDD - SOD, v); its
    chord length matches a brute-force count of points inside the FOV
    (x^2 + y^2 <= 1, |z| <= 1) along the line, and its sample count is the
    fewest equal parts no longer than the spacing, the pixel pitch scaled to
    the rotation axis (SOD / SDD) over D."""
    k = np.arange(16.0)
    g = replace(wl.cone_geometry(16, 32, 32, 2 * np.pi * k / 16, k / 16, 32), subpixels=2)
    D = g.subpixels
    rows, cols = np.array([2, 15, 16, 29, 0]), np.array([4, 15, 17, 27, 31])
    idx = rows * g.det_cols + cols                      # view 0
    o, d, s0, l, t = geometry.subpixel_rays(g, idx)
    kk = np.arange(len(idx) * D * D)
    pix, a, b = kk // (D * D), (kk % (D * D)) // D, kk % D
    u = g.det_off_u + (cols[pix] + (b + 0.5) / D) * g.det_pitch_u
    v = g.det_off_v + (rows[pix] + (a + 0.5) / D) * g.det_pitch_v
    target = np.stack([u, np.full_like(u, g.sdd - g.sod), v], 1)
    assert np.allclose(o, [0.0, -g.sod, 0.0], atol=1e-14)
    want_d = target - o
    want_d /= np.linalg.norm(want_d, axis=1, keepdims=True)
    assert np.allclose(d, want_d, atol=1e-14)
    h = 2e-5
    s = np.arange(0.0, g.sod + 2.0, h) + h / 2
    for r in range(len(l)):
        P = o[r] + s[:, None] * d[r]
        inside = (P[:, 0] ** 2 + P[:, 1] ** 2 <= 1.0) & (np.abs(P[:, 2]) <= 1.0)
        assert abs(inside.sum() * h - l[r]) <= 2 * h
    delta = min(g.det_pitch_u, g.det_pitch_v) * g.sod / g.sdd / D
    assert abs(geometry.sample_spacing(g) - delta) <= 1e-15
    n = geometry.subpixel_counts(g, l)
    full = l > 0
    assert (l[full] / n[full] <= delta * (1 + 1e-12)).all()
    assert (l[full] / np.maximum(n[full] - 1, 1e-300) > delta).all()
    assert (n[~full] == 0).all()
