"""CPU pins of the oracle's geometry, sampler and phantom integrals against
closed forms, hand-derived special cases and brute force."""
import math
import os

import numpy as np
import pytest

from oracle import geometry, phantom, sampler, step
from synthetic import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- decode (Sec. III)

def test_decode_exhaustive_workload1():
    g = wl.workload(1).geom
    i = np.arange(g.n_proj)
    m, row, col = geometry.decode(i, g.n_pixels, g.det_cols)
    assert m.min() == 0 and m.max() == g.n_views - 1
    assert row.min() == 0 and row.max() == g.det_rows - 1
    assert col.min() == 0 and col.max() == g.det_cols - 1
    # the decode is a bijection onto (view, row, col) that reassembles i
    assert np.array_equal(m * g.n_pixels + row * g.det_cols + col, i)
    assert len(set(zip(m.tolist(), row.tolist(), col.tolist()))) == g.n_proj


def test_decode_edges_cone():
    g = wl.workload(3).geom            # 1024 views of 512 x 512
    N = 512 * 512
    cases = {0: (0, 0, 0), N - 1: (0, 511, 511), N: (1, 0, 0),
             N + 513: (1, 1, 1), 1024 * N - 1: (1023, 511, 511)}
    for i, want in cases.items():
        got = tuple(int(x[0]) for x in geometry.decode(np.array([i]), N, 512))
        assert got == want, (i, got, want)


# ------------------------------------------------------ FOV chord (Sec. III, App. A)

def test_parallel_chord_is_circle_chord():
    g = wl.workload(1).geom
    idx = np.arange(g.n_proj)[::7]
    o, d, s0, l, t = geometry.rays(g, idx)
    _, _, col = geometry.decode(idx, g.n_pixels, g.det_cols)
    u = -1.0 + (col + 0.5) * (2.0 / 32)
    # chord of the unit circle at distance |u| from the centre
    assert np.allclose(l, 2.0 * np.sqrt(1.0 - u * u), rtol=0, atol=1e-13)
    # a uniform unit field integrates to the chord length
    one = phantom.project_field(lambda P, t: np.ones(P.shape[:2]), g, idx, 32)
    assert np.allclose(one, l, rtol=0, atol=1e-13)


@pytest.mark.parametrize("w", [3])
def test_cone_chord_brute_force(w):
    g = wl.workload(w).geom
    rng = np.random.default_rng(7)
    idx = rng.integers(0, g.n_proj, 64)
    # include the corner pixels, whose rays miss the FOV
    idx = np.concatenate([idx, [0, 511, 512 * 511, 512 * 512 - 1]])
    o, d, s0, l, t = geometry.rays(g, idx)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-14)
    s = np.linspace(0.0, 12.0, 240001)
    ds = s[1] - s[0]
    for k in range(len(idx)):
        P = o[k][None, :] + s[:, None] * d[k][None, :]
        inside = (P[:, 0] ** 2 + P[:, 1] ** 2 <= 1.0) & (np.abs(P[:, 2]) <= 1.0)
        assert abs(inside.sum() * ds - l[k]) < 2 * ds
        if l[k] > 0:
            for e in (s0[k] + 1e-9, s0[k] + l[k] - 1e-9):
                q = o[k] + e * d[k]
                assert q[0] ** 2 + q[1] ** 2 <= 1.0 + 1e-8 and abs(q[2]) <= 1.0 + 1e-8
            for e in (s0[k] - 1e-6, s0[k] + l[k] + 1e-6):
                q = o[k] + e * d[k]
                assert q[0] ** 2 + q[1] ** 2 > 1.0 or abs(q[2]) > 1.0
    assert (l[-4:] == 0).all()


# -------------------------------------- rotation sign and ray placement (Sec. III)

def _blob(c, sigma):
    c = np.asarray(c, np.float64)
    return lambda P, t: np.exp(-((P - c) ** 2).sum(-1) / (2 * sigma * sigma))


def _pixels_of(g, view, rows, cols):
    return view * g.n_pixels + np.asarray(rows) * g.det_cols + np.asarray(cols)


def test_parallel_rotation_hand_derived():
    """An object rotated by +theta is seen by a source/detector rotated by
    -theta. At theta = 0 rays run along +y with u along +x; at theta = pi/2
    the ray of detector point (u, v) is the line y = -u, z = v along +x; at
    theta = pi it is x = -u, z = v. A narrow blob at (0, 0.5, 0) therefore
    integrates to sigma*sqrt(2 pi)*exp(-h^2/2sigma^2) with h the distance
    to that line."""
    g = wl.parallel_geometry(4, 32, 32, [0.0, math.pi / 2, math.pi, 0.0], [0, 0, 0, 0], 4096)
    sigma, c = 0.05, (0.0, 0.5, 0.0)
    rows, cols = np.meshgrid(np.arange(32), np.arange(32), indexing="ij")
    rows, cols = rows.ravel(), cols.ravel()
    u = -1.0 + (cols + 0.5) / 16.0
    v = -1.0 + (rows + 0.5) / 16.0
    lines = {0: (u - c[0]) ** 2 + v ** 2,            # x = u
             1: (-u - c[1]) ** 2 + v ** 2,           # y = -u
             2: (-u - c[0]) ** 2 + v ** 2}           # x = -u
    for view, h2 in lines.items():
        got = phantom.project_field(_blob(c, sigma), g, _pixels_of(g, view, rows, cols), 4096)
        want = sigma * math.sqrt(2 * math.pi) * np.exp(-h2 / (2 * sigma ** 2))
        assert np.abs(got - want).max() < 1e-7, view


def test_cone_ray_hand_derived():
    """Cone beam at theta = 0: source (0, -SOD, 0), detector point (u, v) at
    y = SDD - SOD. A blob at the origin lies at distance
    SOD * sqrt(u^2 + v^2) / sqrt(u^2 + SDD^2 + v^2) from that ray.
    At theta = pi/2 the source sits at (-SOD, 0, 0) and a blob at
    (0, -0.3, 0) is met by the ray of u = 0.3 * SDD / SOD (magnification)."""
    g = wl.cone_geometry(2, 64, 64, [0.0, math.pi / 2], [0.0, 0.0], 4096)
    sigma = 0.05
    rows, cols = np.meshgrid(np.arange(64), np.arange(64), indexing="ij")
    rows, cols = rows.ravel(), cols.ravel()
    u = -2.7 + (cols + 0.5) * 5.4 / 64
    v = -2.7 + (rows + 0.5) * 5.4 / 64
    h2 = 16.0 * (u * u + v * v) / (u * u + 64.0 + v * v)
    got = phantom.project_field(_blob((0, 0, 0), sigma), g, _pixels_of(g, 0, rows, cols), 4096)
    want = sigma * math.sqrt(2 * math.pi) * np.exp(-h2 / (2 * sigma ** 2))
    assert np.abs(got - want).max() < 1e-7
    got = phantom.project_field(_blob((0, -0.3, 0), sigma), g, _pixels_of(g, 1, rows, cols), 4096)
    peak = cols[np.argmax(got)]
    assert abs((-2.7 + (peak + 0.5) * 5.4 / 64) - 0.6) <= 5.4 / 64


def test_blob_closed_form_general_angles():
    """Midpoint sampling of arbitrary rays converges to the closed-form
    segment integral (App. A ray sampling; O((l/S)^2) error)."""
    for w in (2, 3):
        g = wl.workload(w).geom
        idx = wl.ray_subset(g.n_proj, 200, 11)
        o, d, s0, l, t = geometry.rays(g, idx)
        c, sigma = np.array([0.2, -0.1, 0.05]), 0.3
        want = phantom.gaussian_blob_line(c, sigma, o, d, s0, l)
        errs = []
        for S in (64, 128, 256):
            got = phantom.project_field(_blob(c, sigma), g, idx, S)
            errs.append(np.abs(got - want).max())
        assert errs[-1] < 1e-5
        assert errs[0] / errs[-1] > 12      # second-order convergence


# --------------------------------------------- ellipsoid phantom (measurements)

def test_sphere_chord_textbook():
    """Parallel rays at theta = 0 through a static sphere of radius r at the
    origin: line integral rho * 2 sqrt(r^2 - u^2 - v^2)."""
    g = wl.parallel_geometry(1, 32, 32, [0.0], [0.0], 32)
    ph = wl.Phantom(np.zeros((1, 3)), np.full((1, 3), 0.4), np.array([0.7]), np.zeros((1, 3)), 0.0)
    idx = np.arange(g.n_proj)
    _, row, col = geometry.decode(idx, g.n_pixels, g.det_cols)
    u = -1 + (col + 0.5) / 16
    v = -1 + (row + 0.5) / 16
    want = 0.7 * 2 * np.sqrt(np.maximum(0.16 - u * u - v * v, 0))
    assert np.allclose(phantom.projections(ph, g, idx), want, atol=1e-13)


@pytest.mark.parametrize("w", [1, 2, 3])
def test_ellipsoid_closed_form_vs_midpoint(w):
    """Exact chord integrals of the (moving, growing, FOV-clipped) phantom
    against midpoint sums of its indicator; the midpoint sum of a piecewise
    constant function errs by at most one spacing per boundary crossing."""
    wk = wl.workload(w)
    g, ph = wk.geom, wl.phantom(wk)
    idx = wl.ray_subset(g.n_proj, 256, 21)
    exact = phantom.projections(ph, g, idx)
    o, d, s0, l, t = geometry.rays(g, idx)
    S = 8192
    approx = phantom.project_field(lambda P, tt: phantom.density(ph, P, tt), g, idx, S)
    bound = (2 * ph.rho.sum() + 1e-12) * l / S
    assert (np.abs(exact - approx) <= bound + 1e-12).all()
    assert exact.max() > 0.1           # the phantom is actually seen


def test_phantom_motion_and_growth():
    wk = wl.workload(2)
    ph = wl.phantom(wk)
    c, a = phantom.ellipsoids_at(ph, np.array([0.0, 1.0]))
    assert np.allclose(a[1], 1.5 * a[0])
    speed = np.linalg.norm(c[1] - c[0], axis=1)
    assert (speed <= 0.3 + 1e-12).all() and speed.max() > 0.05


# ---------------------------------------------------------- sampler (Sec. III)

@pytest.mark.parametrize("n", [1, 2, 3, 5, 17, 100, 1000, 4097])
def test_sampler_bijection(n):
    for e in range(3):
        perm = [sampler.permute(x, n, 3001, e) for x in range(n)]
        assert sorted(perm) == list(range(n))


def test_sampler_epoch_covers_all_pixels():
    n, B = 1000, 64
    spe = -(-n // B)
    seen = np.concatenate([sampler.minibatch(s, B, n, 7) for s in range(spe)])
    assert set(seen.tolist()) == set(range(n))
    nxt = np.concatenate([sampler.minibatch(s, B, n, 7) for s in range(spe, 2 * spe)])
    assert set(nxt.tolist()) == set(range(n))
    assert not np.array_equal(seen[:B], nxt[:B])        # a new permutation


def test_sampler_uniformity():
    n, B = 65536, 1024
    idx = sampler.minibatch(0, B, n, 3001)
    assert len(np.unique(idx)) == B
    hist = np.bincount(idx // (n // 16), minlength=16)
    assert hist.min() > 30 and hist.max() < 100           # ~64 per bin


# --------------------------------------------------- Table I / Sec. V pins

def test_voxel_pitch_table1():
    with open(os.path.join(GOLDEN, "table1_magnification.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    for _, pix, sod, sdd, vox in rows:
        assert abs(geometry.voxel_pitch(float(pix), float(sod), float(sdd)) - float(vox)) < 0.006


def test_normalize_maps_fov_box_to_unit_cube():
    g = wl.workload(2).geom
    P = np.array([[[-1.0, -1.0, -1.0], [1.0, 1.0, 1.0], [0.0, 0.5, -0.5]]])
    r = geometry.normalize(g, P, np.array([[0.0, 1.0, 0.25]]))
    assert np.allclose(r[0, 0], [-1, -1, -1, -1])
    assert np.allclose(r[0, 1], [1, 1, 1, 1])
    assert np.allclose(r[0, 2], [-0.5, -0.5, 0.5, 0.0])


def test_project_view_matches_training_rays():
    """A re-projection on the acquisition detector at a view's angle and
    time equals the forward model of the training rays of that view."""
    wk = wl.workload(1)
    g, net = wk.geom, wk.net
    theta = wl.he_init(net, 2001)
    view = 5
    img = step.project_view(theta, g, net, g.view_angle[view], g.view_time[view],
                            g.det_rows, g.det_cols, g.samples_per_ray)
    idx = view * g.n_pixels + np.arange(g.n_pixels)
    out = step.loss_and_grad(theta, g, net, idx, np.zeros(g.n_proj))
    assert np.allclose(img.ravel(), out["p_bar"], rtol=0, atol=1e-12)
