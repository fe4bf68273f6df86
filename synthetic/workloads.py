"""Seeded synthetic workloads for the DINR training step and query server.

Everything here is an *input*: acquisition geometry (view angles and times,
detector layout), analytic ellipsoid phantoms, He-initialised network
weights, random ray subsets and query streams. The paper's data sets are not
available, so these stand in for them with the shapes of its experiments
(parallel-beam simulated 4D data of its Sec. IV-B, cone-beam experimental
scans of its Table I). No step of the reconstruction method is computed
here; the measured projections of a phantom are computed separately by the
oracle (tests) and by the CUDA library (benchmark).

Seeds per workload c (1-based): phantom 1000+c, weights 2000+c, minibatch
sampler 3000+c, noise 4000+c, query stream 5000.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
import math

import numpy as np

from . import rng


@dataclass(frozen=True)
class Geometry:
    """Acquisition geometry in object units.

    Pixel centres: u = det_off_u + (col + 0.5) * det_pitch_u,
    v = det_off_v + (row + 0.5) * det_pitch_v (rows run along +z).
    The field of view is the cylinder x^2 + y^2 <= fov_r^2,
    fov_z0 <= z <= fov_z1, and times lie in [t0, t1].
    """
    beam: str                     # "parallel" or "cone"
    n_views: int
    det_rows: int
    det_cols: int
    view_angle: np.ndarray        # radians, per view
    view_time: np.ndarray         # per view
    det_pitch_u: float
    det_pitch_v: float
    det_off_u: float
    det_off_v: float
    sod: float = 0.0              # source to rotation axis (cone)
    sdd: float = 0.0              # source to detector (cone)
    fov_r: float = 1.0
    fov_z0: float = -1.0
    fov_z1: float = 1.0
    t0: float = 0.0
    t1: float = 1.0
    samples_per_ray: int = 32
    mu0: float = 1.0
    subpixels: int = 0            # App. A model: D x D rays per pixel (0: one ray, S samples)

    @property
    def n_pixels(self) -> int:
        return self.det_rows * self.det_cols

    @property
    def n_proj(self) -> int:
        return self.n_views * self.n_pixels


@dataclass(frozen=True)
class Net:
    n_freq: int
    hidden_layers: int
    width: int
    act: str = "relu"             # "relu" or "swish"
    out_act: str = "identity"     # "identity" or "softplus"
    encoding: str = "octave"      # "octave" or "grff" (Gaussian random Fourier features)
    grff_c: int = 0               # C frequencies (2C features) of the GRFF encoding
    sigma_t: float = 0.1          # std of B's time column
    sigma_s: float = 0.5          # std of B's three spatial columns
    grff_seed: int = 0

    @property
    def d_in(self) -> int:
        return 2 * self.grff_c if self.encoding == "grff" else 4 + 8 * self.n_freq

    @property
    def grff_B(self) -> np.ndarray:
        """The frozen GRFF matrix B [C][4] (columns t, z, y, x): normals of
        the stream grff_seed, column 0 scaled by sigma_t and columns 1-3 by
        sigma_s, rounded to FP32 once so both sides use the same values."""
        z = rng.normal(self.grff_seed, 4 * self.grff_c).reshape(self.grff_c, 4)
        sig = np.array([self.sigma_t, self.sigma_s, self.sigma_s, self.sigma_s])
        return (z * sig).astype(np.float32).astype(np.float64)

    def layer_shapes(self):
        """(fan_out, fan_in) of each linear layer, output layer last."""
        shapes = [(self.width, self.d_in)]
        shapes += [(self.width, self.width)] * (self.hidden_layers - 1)
        shapes.append((1, self.width))
        return shapes

    @property
    def n_params(self) -> int:
        return sum(o * i + o for o, i in self.layer_shapes())


@dataclass(frozen=True)
class Train:
    batch_rays: int
    lr: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    lr_decay_per_epoch: float = 1.0


@dataclass(frozen=True)
class Phantom:
    """Ellipsoids with centre c0 + vel*t, semi-axes a0*(1 + growth*t),
    attenuation rho. Overlapping ellipsoids add."""
    centre: np.ndarray            # [n, 3] (x, y, z)
    axes: np.ndarray              # [n, 3]
    rho: np.ndarray               # [n]
    vel: np.ndarray               # [n, 3]
    growth: float = 0.5


@dataclass(frozen=True)
class Workload:
    index: int
    name: str
    geom: Geometry
    net: Net
    train: Train
    n_ellipsoids: int
    moving: bool = False
    noise_rel: float = 0.0

    @property
    def seeds(self):
        c = self.index
        return dict(phantom=1000 + c, weights=2000 + c, sampler=3000 + c,
                    noise=4000 + c)


def parallel_geometry(n_views, rows, cols, angles, times, S, mu0=1.0):
    R, z0, z1 = 1.0, -1.0, 1.0
    return Geometry("parallel", n_views, rows, cols,
                    np.asarray(angles, np.float64), np.asarray(times, np.float64),
                    det_pitch_u=2 * R / cols, det_pitch_v=(z1 - z0) / rows,
                    det_off_u=-R, det_off_v=z0, samples_per_ray=S, mu0=mu0)


def cone_geometry(n_views, rows, cols, angles, times, S, sod=4.0, sdd=8.0,
                  half_extent=2.7, mu0=1.0):
    return Geometry("cone", n_views, rows, cols,
                    np.asarray(angles, np.float64), np.asarray(times, np.float64),
                    det_pitch_u=2 * half_extent / cols,
                    det_pitch_v=2 * half_extent / rows,
                    det_off_u=-half_extent, det_off_v=-half_extent,
                    sod=sod, sdd=sdd, samples_per_ray=S, mu0=mu0)


def _views(n, rotations):
    k = np.arange(n, dtype=np.float64)
    return 2.0 * math.pi * rotations * k / n, k / n


def workload(c: int) -> Workload:
    """The workloads: 1 parity, 2 parallel-beam perf, 3 cone-beam, 4 wide
    network at scale, 5 serving (network of 3), 6 the paper's own network
    (GRFF encoding 2C = 256 with sigma_s = 0.5, sigma_t = 0.1, five Swish
    layers of 2C, linear output) on the geometry of 2, 7 the same network
    at parity size (geometry of 1, 2C = 64, three layers), 8 and 9 the
    networks of 6 and 7 with the paper's forward model (App. A: 2 x 2
    sub-pixel rays per pixel, samples about half a pixel apart)."""
    if c == 1:
        k = np.arange(64, dtype=np.float64)
        g = parallel_geometry(64, 32, 32, math.pi * k / 64, k / 64, 32)
        return Workload(1, "parallel-beam 64 views 32x32, S=32, MLP 3x64 softplus, B=1024",
                        g, Net(6, 3, 64, "relu", "softplus"), Train(1024), 3)
    if c == 2:
        a, t = _views(512, 4)
        g = parallel_geometry(512, 128, 128, a, t, 128)
        return Workload(2, "parallel-beam 512 views 128x128, S=128, MLP 5x256, B=65536",
                        g, Net(10, 5, 256), Train(65536), 16, moving=True)
    if c == 3:
        a, t = _views(1024, 2)
        g = cone_geometry(1024, 512, 512, a, t, 256)
        return Workload(3, "cone-beam SOD 4 SDD 8, 1024 views 512x512, S=256, MLP 6x256, B=65536",
                        g, Net(10, 6, 256), Train(65536), 64, noise_rel=0.01)
    if c == 4:
        a, t = _views(1024, 2)
        g = cone_geometry(1024, 512, 512, a, t, 256)
        return Workload(4, "cone-beam SOD 4 SDD 8, 1024 views 512x512, S=256, MLP 8x512 F=12, B=65536",
                        g, Net(12, 8, 512), Train(65536), 64, noise_rel=0.01)
    if c == 5:
        w = workload(3)
        return replace(w, index=5, name="serving: trained 6x256 cone-beam network")
    if c == 6:
        w = workload(2)
        net = Net(0, 5, 256, "swish", "identity", "grff", 128, 0.1, 0.5, 6006)
        return replace(w, index=6, net=net,
                       name="parallel-beam 512 views 128x128, S=128, GRFF 2C=256 + 5x256 Swish, "
                            "B=65536")
    if c == 8:
        w = workload(6)
        return replace(w, index=8, geom=replace(w.geom, subpixels=2),
                       name="parallel-beam 512 views 128x128, App. A forward model (2x2 "
                            "sub-pixel rays, spacing pixel/2), GRFF 2C=256 + 5x256 Swish, B=65536")
    if c == 9:
        w = workload(7)
        return replace(w, index=9, geom=replace(w.geom, subpixels=2),
                       name="parallel-beam 64 views 32x32, App. A forward model (2x2 sub-pixel "
                            "rays), GRFF 2C=64 + 3x64 Swish, B=1024")
    if c == 7:
        w = workload(1)
        net = Net(0, 3, 64, "swish", "identity", "grff", 32, 0.1, 0.5, 6007)
        return replace(w, index=7, net=net,
                       name="parallel-beam 64 views 32x32, S=32, GRFF 2C=64 + 3x64 Swish, B=1024")
    raise ValueError(f"no workload {c}")


def phantom(w: Workload) -> Phantom:
    """Seeded ellipsoids: 10 uniforms per ellipsoid from the phantom stream
    (centre x3, semi-axes x3, attenuation, direction x2, speed)."""
    n = w.n_ellipsoids
    u = rng.uniform(w.seeds["phantom"], 10 * n).reshape(n, 10)
    centre = u[:, 0:3] - 0.5
    axes = 0.1 + 0.2 * u[:, 3:6]
    rho = 0.5 + 0.5 * u[:, 6]
    vel = np.zeros((n, 3))
    if w.moving:
        cz = 2.0 * u[:, 7] - 1.0
        phi = 2.0 * math.pi * u[:, 8]
        sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
        speed = 0.3 * u[:, 9]
        vel = speed[:, None] * np.stack([sz * np.cos(phi), sz * np.sin(phi), cz], axis=1)
    return Phantom(centre, axes, rho, vel)


def he_init(net: Net, seed: int) -> np.ndarray:
    """Flat FP64 parameters, layout [W_1 (fan_out x fan_in, row-major), b_1,
    ..., W_H, b_H, w_out, b_out]. Weights ~ N(0, 2/fan_in), biases 0.
    Weight entries take consecutive normals of the stream in layout order."""
    shapes = net.layer_shapes()
    nw = sum(o * i for o, i in shapes)
    z = rng.normal(seed, nw)
    out = np.zeros(net.n_params)
    p = q = 0
    for o, i in shapes:
        out[p:p + o * i] = z[q:q + o * i] * math.sqrt(2.0 / i)
        p += o * i + o
        q += o * i
    return out


def ray_subset(n_proj: int, n: int, seed: int) -> np.ndarray:
    """n distinct projection indices in [0, n_proj), in draw order."""
    if n > n_proj:
        raise ValueError("subset larger than the projection stack")
    got = np.empty(0, dtype=np.int64)
    off = 0
    while got.size < n:
        m = 2 * (n - got.size) + 16
        cand = (rng.u64(seed, m, off) % np.uint64(n_proj)).astype(np.int64)
        off += m
        allc = np.concatenate([got, cand])
        _, first = np.unique(allc, return_index=True)
        got = allc[np.sort(first)]
    return got[:n]


def noise(w: Workload, n: int, offset: int = 0) -> np.ndarray:
    """Standard normals of the noise stream (scaled by the caller)."""
    return rng.normal(w.seeds["noise"], n, offset)


@dataclass(frozen=True)
class Query:
    arrival: float                # seconds
    kind: str                     # "slice", "subvolume" or "reprojection"
    size: int                     # slice side, sub-volume side or detector side
    t: float
    theta: float = 0.0
    box_lo: tuple = (0.0, 0.0, 0.0)
    box_hi: tuple = (0.0, 0.0, 0.0)
    z: float = 0.0

    @property
    def n_outputs(self) -> int:
        if self.kind == "slice":
            return self.size * self.size
        if self.kind == "subvolume":
            return self.size ** 3
        return self.size * self.size


def query_stream(n: int, rate: float = 200.0, seed: int = 5000,
                 reproj_side: int = 256) -> list:
    """Poisson arrivals (exponential gaps of mean 1/rate), kinds uniform over
    {slice, subvolume, reprojection}; slice sides 128..1024 and sub-volume
    sides 32..256 uniform over powers of two; t ~ U(0,1), theta ~ U(0, 2pi);
    sub-volume boxes uniform inside [-1,1]^3; slices are axial (fixed z)."""
    u = rng.uniform(seed, 12 * n).reshape(n, 12)
    out, clock = [], 0.0
    for q in range(n):
        clock += -math.log(1.0 - u[q, 0]) / rate
        kind = ("slice", "subvolume", "reprojection")[min(2, int(3 * u[q, 1]))]
        t = float(u[q, 2])
        if kind == "slice":
            side = 128 << min(3, int(4 * u[q, 3]))
            out.append(Query(clock, kind, side, t, z=float(2 * u[q, 4] - 1)))
        elif kind == "subvolume":
            side = 32 << min(3, int(4 * u[q, 3]))
            ext = 2.0 * side / 256.0          # a 256^3 box spans the whole cube
            lo = [-1.0 + (2.0 - ext) * float(u[q, 5 + d]) for d in range(3)]
            hi = [l + ext for l in lo]
            out.append(Query(clock, kind, side, t, box_lo=tuple(lo), box_hi=tuple(hi)))
        else:
            out.append(Query(clock, kind, reproj_side, t,
                             theta=float(2 * math.pi * u[q, 8])))
    return out
