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

from gpu_util import assert_close, make_model, require_gpu, split_grad

pytestmark = pytest.mark.gpu
TOL = {"fp32": 1e-5, "bf16": 2e-2}


def _check(m, w, net, theta, idx, proj, prec, decide=None):
    ref = ostep.loss_and_grad(theta, w.geom, net, idx, proj.astype(np.float64), decide=decide)
    assert_close(m.predict(idx).cpu().numpy(), ref["p_bar"], TOL[prec], "p_bar")
    loss, grad = m.loss_grad(idx)
    assert abs(loss.item() - ref["loss"]) <= TOL[prec] * ref["loss"]
    g = grad.cpu().numpy()
    for L, ((gw, gb), (ow, ob)) in enumerate(zip(split_grad(g, net), split_grad(ref["grad"], net))):
        assert_close(gw, ow, TOL[prec], f"dW layer {L}")
        assert_close(gb, ob, TOL[prec], f"db layer {L}")


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_paper_network_parity_size(prec):
    require_gpu()
    w = wl.workload(7)
    idx = wl.ray_subset(w.geom.n_proj, 1024, w.seeds["sampler"])
    m, theta, proj = make_model(w, prec, idx=idx)
    _check(m, w, w.net, theta, idx, proj, prec)
    m.close()


def test_grff_relu_fused_chain():
    require_gpu()
    w = wl.workload(7)
    net = replace(w.net, act="relu", out_act="softplus", grff_c=128, width=128)
    idx = wl.ray_subset(w.geom.n_proj, 512, 77)
    m, theta, proj = make_model(w, "bf16", idx=idx, net=net,
                                params=wl.he_init(net, w.seeds["weights"]))
    m.profile(True)
    _check(m, w, net, theta, idx, proj, "bf16", decide="bf16")
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
    _check(m, w, w.net, theta, idx, proj, prec)
    m.close()
