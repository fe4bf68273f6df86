"""GPU parity of the plain FP32 path against the FP64 oracle, called through
the C ABI. Tolerance for the FP32 path: 1e-5, norm-wise relative per tensor
and element-wise relative to the tensor's largest magnitude; integer work
(indices, sampler) bit-exact."""
import math

import numpy as np
import pytest
import torch

from oracle import phantom as ophantom, sampler as osampler, step as ostep
from synthetic import workloads as wl

from gpu_util import assert_close, make_model, projections_for, rel_err, require_gpu, split_grad

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def _grad_check(g_gpu, g_or, net, tol):
    for L, ((gw, gb), (ow, ob)) in enumerate(zip(split_grad(g_gpu, net), split_grad(g_or, net))):
        assert_close(gw, ow, tol, f"dW layer {L}")
        assert_close(gb, ob, tol, f"db layer {L}")


# ------------------------------------------------------------ integer work

def test_sampler_bit_exact():
    for c, B, steps in ((1, 1024, (0, 1, 63, 64, 65, 200)), (3, 4096, (0, 7, 65535))):
        w = wl.workload(c)
        m, _, _ = make_model(w, "fp32", net=wl.Net(0, 1, 16), batch=B,
                             geom=w.geom if c == 1 else w.geom)
        for s in steps:
            got = m.sample_indices(s, B).cpu().numpy()
            want = osampler.minibatch(s, B, w.geom.n_proj, w.seeds["sampler"])
            assert np.array_equal(got, want), (c, s)
        m.close()


def test_phantom_projections_match_closed_form():
    from paper_2404_19075_b300 import phantom_project
    for c in (1, 2, 3):
        w = wl.workload(c)
        g = w.geom
        idx = np.arange(g.n_proj) if c == 1 else wl.ray_subset(g.n_proj, 20000, 77)
        got = phantom_project(g, wl.phantom(w), idx).cpu().numpy()
        want = ophantom.projections(wl.phantom(w), g, idx)
        assert_close(got, want, 1e-6, f"workload {c}")


# ------------------------------------------------------- workload 1, full size

@pytest.fixture(scope="module")
def c1():
    w = wl.workload(1)
    idx = wl.ray_subset(w.geom.n_proj, 1024, w.seeds["sampler"])
    m, theta, proj = make_model(w, "fp32", idx=idx)
    ref = ostep.loss_and_grad(theta, w.geom, w.net, idx, proj.astype(np.float64))
    yield w, m, theta, proj, idx, ref
    m.close()


def test_c1_forward_model(c1):
    w, m, theta, proj, idx, ref = c1
    assert_close(m.predict(idx).cpu().numpy(), ref["p_bar"], TOL, "p_bar")


def test_c1_loss_and_gradient(c1):
    w, m, theta, proj, idx, ref = c1
    loss, grad = m.loss_grad(idx)
    assert abs(loss.item() - ref["loss"]) <= TOL * ref["loss"]
    _grad_check(grad.cpu().numpy(), ref["grad"], w.net, TOL)


def test_c1_train_step_adam(c1):
    w, m, theta, proj, idx, ref = c1
    m.set_params(theta.astype(np.float32))
    st = m.get_state()
    loss = m.train_step(idx)
    out = ostep.train_step(theta, np.zeros_like(theta), np.zeros_like(theta), 1, w.geom, w.net,
                           w.train, idx, proj.astype(np.float64))
    assert abs(loss - out["loss"]) <= TOL * out["loss"]
    new = m.params().cpu().numpy()
    # the update itself (about lr per entry) to 1e-5 of its norm, except
    # entries whose gradient is below FP32 resolution of the largest one
    d_gpu, d_or = new - theta, out["theta"] - theta
    big = np.abs(out["grad"]) > 1e-4 * np.abs(out["grad"]).max()
    assert rel_err(d_gpu[big], d_or[big]) <= 1e-4
    m.set_state(st)


def test_c1_sampler_step_deterministic(c1):
    w, m, theta, proj, idx, ref = c1
    st = m.get_state()
    l1 = m.train_step(None, n=1024)
    p1 = m.params().cpu().numpy()
    m.set_state(st)
    l2 = m.train_step(None, n=1024)
    p2 = m.params().cpu().numpy()
    assert l1 == l2 and np.array_equal(p1, p2)
    m.set_state(st)


def test_c1_chunked_passes_match(c1):
    w, m, theta, proj, idx, ref = c1
    m2, _, _ = make_model(w, "fp32", proj=proj, chunk=100)
    loss, grad = m2.loss_grad(idx)
    assert_close(grad.cpu().numpy(), ref["grad"], TOL, "chunked gradient")
    m2.close()


def test_c1_ragged_and_single_ray_batches(c1):
    w, m, theta, proj, idx, ref = c1
    for n in (1, 7, 333):
        sub = idx[:n]
        r = ostep.loss_and_grad(theta, w.geom, w.net, sub, proj.astype(np.float64))
        loss, grad = m.loss_grad(sub)
        assert abs(loss.item() - r["loss"]) <= TOL * r["loss"] + 1e-12
        assert_close(grad.cpu().numpy(), r["grad"], TOL, f"n={n}")


def test_c1_autograd_function(c1):
    from paper_2404_19075_b300 import DinrStep
    w, m, theta, proj, idx, ref = c1
    p = torch.tensor(theta, dtype=torch.float32, device="cuda", requires_grad=True)
    loss = DinrStep.apply(p, m, torch.as_tensor(idx, device="cuda"))
    (3.0 * loss).backward()
    assert_close(p.grad.cpu().numpy(), 3.0 * ref["grad"], TOL, "autograd")


def test_bad_indices_are_rejected(c1):
    from paper_2404_19075_b300 import DinrError
    w, m, theta, proj, idx, ref = c1
    st = m.get_state()
    with pytest.raises(DinrError):
        m.train_step_host(np.array([0, w.geom.n_proj], np.int64))   # host: checked up front
    assert m.get_state() == st                                       # nothing ran
    bad = torch.tensor([1, -5, 3], dtype=torch.int64, device="cuda")
    with pytest.raises(DinrError):
        m.train_step(bad)                             # device: replaced by 0, then reported
    with pytest.raises(DinrError):
        m.train_step(None, n=0)
    with pytest.raises(DinrError):
        m.train_step(None, n=1025)                    # more than the batch the context holds
    m.set_state(st)


def test_host_and_device_indices_agree(c1):
    w, m, theta, proj, idx, ref = c1
    st = m.get_state()
    l_host = m.train_step_host(idx)
    p_host = m.params().cpu().numpy()
    m.set_state(st)
    l_dev = m.train_step(torch.as_tensor(idx, device="cuda"))
    assert l_host == l_dev and np.array_equal(p_host, m.params().cpu().numpy())
    m.set_state(st)


# ------------------------------------------------------- queries (Sec. V)

def test_c1_query_project_grid(c1):
    w, m, theta, proj, idx, ref = c1
    g, net = w.geom, w.net
    rng = np.random.default_rng(3)
    coords = np.stack([rng.uniform(0, 1, 500), rng.uniform(-1, 1, 500),
                       rng.uniform(-0.7, 0.7, 500), rng.uniform(-0.7, 0.7, 500)], 1)
    coords = coords.astype(np.float32).astype(np.float64)       # what the device sees
    assert_close(m.query(coords).cpu().numpy(), ostep.query(theta, g, net, coords), TOL, "query")
    img = m.project(0.3, 0.41, 17, 23, 19).cpu().numpy()
    want = ostep.project_view(theta, g, net, 0.3, 0.41, 17, 23, 19)
    assert_close(img, want, TOL, "project")
    lo, hi, dims = (-0.5, -0.4, 0.1), (0.5, 0.3, 0.2), (9, 7, 3)
    vol = m.query_grid(0.7, lo, hi, dims).cpu().numpy()
    ax = [lo[d] + (np.arange(dims[d]) + 0.5) * (hi[d] - lo[d]) / dims[d] for d in range(3)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    pts = np.stack([np.full(X.size, 0.7), Z.ravel(), Y.ravel(), X.ravel()], 1)
    assert_close(vol.ravel(), ostep.query(theta, g, net, pts), TOL, "grid")


# --------------------------------------- workloads 2 and 3 on ray subsets

@pytest.mark.parametrize("c,n", [(2, 128), (3, 64)])
def test_subset_parity_fp32(c, n):
    w = wl.workload(c)
    idx = wl.ray_subset(w.geom.n_proj, n, 99)
    m, theta, proj = make_model(w, "fp32", idx=idx, batch=n)
    ref = ostep.loss_and_grad(theta, w.geom, w.net, idx, proj.astype(np.float64))
    assert_close(m.predict(idx).cpu().numpy(), ref["p_bar"], TOL, "p_bar")
    loss, grad = m.loss_grad(idx)
    assert abs(loss.item() - ref["loss"]) <= TOL * ref["loss"]
    _grad_check(grad.cpu().numpy(), ref["grad"], w.net, TOL)
    m.close()


def test_state_roundtrip_bitwise():
    w = wl.workload(1)
    idx = wl.ray_subset(w.geom.n_proj, 256, 5)
    m, theta, proj = make_model(w, "fp32", idx=idx, batch=256)
    for _ in range(2):
        m.train_step(idx)
    blob = m.get_state()
    m.train_step(idx)
    a = m.params().cpu().numpy()
    m2, _, _ = make_model(w, "fp32", proj=proj, batch=256)
    m2.set_state(blob)
    m2.train_step(idx)
    assert np.array_equal(a, m2.params().cpu().numpy())
    m.close()
    m2.close()
