"""The paper's own network (App. B): Gaussian random Fourier features of the
normalised coordinates, Swish hidden layers, linear output. Parity of the
FP32 path (1e-5) and the BF16 tensor-core path (2e-2) with the FP64 oracle
at parity size and on a subset of the full network (2C = 256, five layers);
GRFF with ReLU through the fused chains (ReLU decisions in BF16 on both
sides), including queries."""
from dataclasses import replace

import numpy as np
import pytest

from oracle import step as ostep
from synthetic import workloads as wl

from gpu_util import assert_close, check_step, make_model, require_gpu

pytestmark = pytest.mark.gpu
TOL = {"fp32": 1e-5, "bf16": 2e-2}


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_paper_network_parity_size(prec):
    require_gpu()
    w = wl.workload(7)
    idx = wl.ray_subset(w.geom.n_proj, 1024, w.seeds["sampler"])
    m, theta, proj = make_model(w, prec, idx=idx)
    check_step(m, w, w.net, theta, idx, proj, prec)
    m.close()


def test_grff_relu_fused_chain():
    require_gpu()
    w = wl.workload(7)
    net = replace(w.net, act="relu", out_act="softplus", grff_c=128, width=128)
    idx = wl.ray_subset(w.geom.n_proj, 512, 77)
    m, theta, proj = make_model(w, "bf16", idx=idx, net=net,
                                params=wl.he_init(net, w.seeds["weights"]))
    m.profile(True)
    check_step(m, w, net, theta, idx, proj, "bf16", label="GRFF relu")
    m.profile(False)
    assert "tc_fwd_chain" in m.profile_report()
    pts = np.random.default_rng(3).uniform(-0.9, 0.9, (300, 4))
    pts[:, 0] = np.random.default_rng(4).uniform(0, 1, 300)
    got = m.query(pts.astype(np.float32)).cpu().numpy()
    want = ostep.query(theta, w.geom, net, pts.astype(np.float32).astype(np.float64))
    assert_close(got, want, TOL["bf16"], "query")
    m.close()


@pytest.mark.parametrize("prec,n", [("fp32", 16), ("bf16", 128)])
def test_paper_network_full_size_subset(prec, n):
    require_gpu()
    w = wl.workload(6)
    idx = wl.ray_subset(w.geom.n_proj, n, 606)
    m, theta, proj = make_model(w, prec, idx=idx, batch=256)
    check_step(m, w, w.net, theta, idx, proj, prec)
    m.close()


def test_swish_fused_chains_and_serving():
    """GRFF (C = 128) with Swish through the fused forward and backward
    chains (the forward stores the Swish derivative for the backward), and
    the same network answering point queries through the query server."""
    require_gpu()
    w = wl.workload(7)
    net = replace(w.net, grff_c=128, width=128)
    idx = wl.ray_subset(w.geom.n_proj, 512, 78)
    m, theta, proj = make_model(w, "bf16", idx=idx, net=net,
                                params=wl.he_init(net, w.seeds["weights"]))
    m.profile(True)
    check_step(m, w, net, theta, idx, proj, "bf16")
    m.profile(False)
    rep = m.profile_report()
    assert "tc_fwd_chain" in rep and "tc_bwd_chain" in rep
    pts = np.random.default_rng(5).uniform(-0.9, 0.9, (700, 4))
    pts[:, 0] = np.random.default_rng(6).uniform(0, 1, 700)
    pts = pts.astype(np.float32)
    want = ostep.query(theta, w.geom, net, pts.astype(np.float64))
    assert_close(m.query(pts).cpu().numpy(), want, TOL["bf16"], "query")
    import torch
    out = torch.empty(len(pts), device="cuda")
    rid = m.serve_submit("points", out, coords=pts)
    while not m.serve_poll(rid):
        m.serve_step()
    torch.cuda.synchronize()
    assert_close(out.cpu().numpy(), want, TOL["bf16"], "served")
    m.close()
