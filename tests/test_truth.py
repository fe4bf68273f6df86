"""The scoring ground truth (synthetic.truth) is the field the measurements
are projections of: it equals the oracle's phantom density at the grid
points, and the scores are exact on known errors."""
import numpy as np

from oracle import phantom as oph
from synthetic import truth, workloads as wl


def test_grid_matches_phantom_density():
    w = wl.workload(2)
    ph = wl.phantom(w)
    n, t = 16, 0.7
    g = truth.attenuation_grid(ph, t, n)
    ax = truth.grid_axis(n)
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    P = np.stack([X, Y, Z], -1).reshape(1, -1, 3)
    want = oph.density(ph, P, np.array([t]))[0].reshape(n, n, n)
    assert np.max(np.abs(g - want)) <= 1e-12           # same field, another summation order


def test_scores_on_known_error():
    truth_v = np.ones((4, 4, 4))
    mask = np.ones_like(truth_v, bool)
    s = truth.scores(truth_v * 1.1, truth_v, mask)
    assert abs(s["rel_l2"] - 0.1) < 1e-12
    assert abs(s["psnr_db"] - 20.0) < 1e-9            # 10 log10(1 / 0.01)
    m = truth.fov_mask(8)
    # centres +-0.125, +-0.375, +-0.625, +-0.875: per pair of x values the
    # y values with x^2 + y^2 <= 1 number 8, 8, 6, 4 -> 2 (8 + 8 + 6 + 4) = 52
    # cells per z-layer, 8 layers
    assert m.sum() == 8 * 52
