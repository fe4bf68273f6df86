"""GPU parity of the paper's forward model (App. A: D x D sub-pixel rays per
pixel, a variable number of samples per ray, p_bar over all of a pixel's
samples) against the FP64 oracle: the FP32 path (1e-5), the BF16 unfused
path and the fused chains (2e-2; with ReLU against the plain oracle and
the one with BF16-taken ReLU decisions), predictions of pixels whose rays
all miss the field of view, and the full-size paper network on a subset of
pixels."""
from dataclasses import replace

import numpy as np
import pytest

from oracle import geometry
from synthetic import workloads as wl

from gpu_util import (assert_close, check_step, make_model, oracle_refs, plain_gate,
                      require_gpu)

pytestmark = pytest.mark.gpu
TOL = {"fp32": 1e-5, "bf16": 2e-2}


def _check(m, w, geom, net, theta, idx, proj, prec, label):
    check_step(m, replace(w, geom=geom), net, theta, idx, proj, prec, label=label)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_subpixel_model_parity_size(prec):
    require_gpu()
    w = wl.workload(9)
    idx = wl.ray_subset(w.geom.n_proj, 512, w.seeds["sampler"])
    m, theta, proj = make_model(w, prec, idx=idx, batch=512, chunk=200)   # three passes
    _check(m, w, w.geom, w.net, theta, idx, proj, prec, "App. A parity size")
    m.close()


@pytest.mark.parametrize("act,out_act,C,F", [("swish", "identity", 128, 0),
                                             ("relu", "softplus", 0, 6)])
def test_subpixel_model_fused_chains(act, out_act, C, F):
    require_gpu()
    w = wl.workload(9)
    enc = "grff" if C else "octave"
    net = replace(w.net, act=act, out_act=out_act, encoding=enc, grff_c=C, n_freq=F, width=128)
    idx = wl.ray_subset(w.geom.n_proj, 384, 91)
    m, theta, proj = make_model(w, "bf16", idx=idx, net=net, batch=384,
                                params=wl.he_init(net, w.seeds["weights"]))
    m.profile(True)
    _check(m, w, w.geom, net, theta, idx, proj, "bf16", f"App. A chains {act}")
    m.profile(False)
    assert "tc_fwd_chain" in m.profile_report()
    m.close()


def test_subpixel_pixels_outside_the_fov():
    require_gpu()
    w = wl.workload(3)
    g = replace(w.geom, subpixels=2)
    N = g.det_rows * g.det_cols
    idx = np.array([m * N + r * g.det_cols + c for m in (0, 511) for r in (0, g.det_rows - 1)
                    for c in (0, g.det_cols - 1)], np.int64)
    assert (geometry.subpixel_rays(g, idx)[3] == 0).all()
    full = wl.ray_subset(g.n_proj, 8, 5)
    both = np.concatenate([idx, full])
    m, theta, proj = make_model(w, "bf16", idx=both, geom=g, batch=64)
    p = m.predict(both).cpu().numpy()
    assert (p[:len(idx)] == 0).all()
    plain, decided = oracle_refs(theta, g, w.net, both, proj, "bf16")
    assert_close(p, decided["p_bar"], TOL["bf16"], "p_bar (BF16-decided oracle)")
    plain_gate("App. A outside the FOV", "p_bar", p, plain["p_bar"], TOL["bf16"], decided["p_bar"])
    m.close()


@pytest.mark.parametrize("prec,n", [("fp32", 6), ("bf16", 48)])
def test_subpixel_paper_network_full_size_subset(prec, n):
    require_gpu()
    w = wl.workload(8)
    idx = wl.ray_subset(w.geom.n_proj, n, 808)
    m, theta, proj = make_model(w, prec, idx=idx, batch=64)
    _check(m, w, w.geom, w.net, theta, idx, proj, prec, "App. A workload 8 subset")
    m.close()


@pytest.mark.parametrize("prec,act,C,F", [("fp32", "swish", 32, 0), ("bf16", "swish", 32, 0),
                                          ("bf16", "relu", 0, 6)])
def test_subpixel_cone_beam(prec, act, C, F):
    """App. A on a cone-beam geometry (source-to-object 4, source-to-
    detector 8): sub-rays from the source to the sub-pixel centres, spacing
    scaled to the rotation axis; the paper's network (FP32 path, BF16
    unfused) and an octave ReLU network through the fused chains."""
    require_gpu()
    w9 = wl.workload(9)
    k = np.arange(64.0)
    geom = replace(wl.cone_geometry(64, 32, 32, 2 * np.pi * k / 64, k / 64, 32), subpixels=2)
    w = replace(w9, geom=geom)
    enc = "grff" if C else "octave"
    net = replace(w9.net, act=act, encoding=enc, grff_c=C, n_freq=F,
                  width=128 if act == "relu" else w9.net.width)
    idx = wl.ray_subset(geom.n_proj, 256, 17)
    m, theta, proj = make_model(w, prec, idx=idx, net=net, batch=256,
                                params=wl.he_init(net, w.seeds["weights"]))
    try:
        _check(m, w, geom, net, theta, idx, proj, prec, f"App. A cone {act}")
    finally:
        m.close()
