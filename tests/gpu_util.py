"""Helpers shared by the GPU parity tests: build a library context for a
workload with the oracle's inputs, and the comparison measures."""
import numpy as np
import pytest
import torch

from oracle import phantom as ophantom
from oracle import step as ostep
from synthetic import workloads as wl


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def rel_err(got, want):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    return float(np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-300))


def assert_close(got, want, tol, what=""):
    """Norm-wise relative error <= tol and every element within
    tol * max|want| (the measure the tolerances are stated in)."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    assert got.shape == want.shape, (what, got.shape, want.shape)
    r = rel_err(got, want)
    m = float(np.abs(got - want).max()) / max(float(np.abs(want).max()), 1e-300)
    assert r <= tol and m <= tol, f"{what}: norm-wise {r:.3e}, element-wise {m:.3e} > {tol}"


def split_grad(g, net):
    """Per-layer (W, b) views of a flat gradient, output layer last."""
    out, p = [], 0
    for o, i in net.layer_shapes():
        out.append((g[p:p + o * i], g[p + o * i:p + o * i + o]))
        p += o * i + o
    return out


def projections_for(w, idx):
    """A full projection stack with the oracle's exact phantom projections
    at the indices used (zeros elsewhere)."""
    g = w.geom
    p = np.zeros(g.n_proj, np.float32)
    p[idx] = ophantom.projections(wl.phantom(w), g, idx)
    return p


def make_model(w, prec, idx=None, proj=None, net=None, geom=None, batch=None, chunk=0,
               params=None, recompute=0):
    from paper_2404_19075_b300 import Dinr
    net = net or w.net
    geom = geom or w.geom
    if params is None:
        params = wl.he_init(net, w.seeds["weights"])
    if proj is None:
        proj = projections_for(w, idx) if idx is not None else np.zeros(geom.n_proj, np.float32)
    train = wl.Train(batch or w.train.batch_rays)
    m = Dinr(geom, net, train, proj, prec=prec, init_params=params.astype(np.float32),
             sampler_seed=w.seeds["sampler"], chunk_rays=chunk, recompute=recompute)
    return m, params.astype(np.float32).astype(np.float64), proj


TOL = {"fp32": 1e-5, "bf16": 2e-2}


def check_step(m, w, net, theta, idx, proj, prec, decide=None, tol=None):
    """p_bar, loss and every layer's weight and bias gradients within the
    path's tolerance (or `tol`). The output layer's bias gradient is one
    number, a sum of signed residuals p_bar - p over the batch in which
    cancellation magnifies the rounding of p_bar; it is checked together
    with the output weights' gradient as one tensor (norm-wise and
    element-wise)."""
    t = TOL[prec] if tol is None else tol
    ref = ostep.loss_and_grad(theta, w.geom, net, idx, proj.astype(np.float64), decide=decide)
    assert_close(m.predict(idx).cpu().numpy(), ref["p_bar"], t, "p_bar")
    loss, grad = m.loss_grad(idx)
    assert abs(loss.item() - ref["loss"]) <= t * ref["loss"]
    g = grad.cpu().numpy()
    pairs = list(zip(split_grad(g, net), split_grad(ref["grad"], net)))
    for L, ((gw, gb), (ow, ob)) in enumerate(pairs[:-1]):
        assert_close(gw, ow, t, f"dW layer {L}")
        assert_close(gb, ob, t, f"db layer {L}")
    (gw, gb), (ow, ob) = pairs[-1]
    assert_close(np.concatenate([gw, gb]), np.concatenate([ow, ob]), t, "output layer")
