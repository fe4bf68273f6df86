"""GPU parity of the BF16 tensor-core path (tcgen05 GEMMs, FP32
accumulation) against the FP64 oracle through the C ABI. Tolerance for the
BF16 path: 2e-2, norm-wise relative per tensor and element-wise relative to
the tensor's largest magnitude. Every tensor is held to it against the plain
FP64 oracle (unless a test states a wider bound and why) and, as a
diagnostic, against the oracle with its ReLU decisions taken on a
BF16-rounded forward (a ReLU mask is an integer decided by floating point;
units whose pre-activation is within BF16 rounding of zero can flip)."""
import numpy as np
import pytest
import torch

from oracle import step as ostep
from synthetic import workloads as wl

from gpu_util import (assert_close, check_step, gate_tensors, make_model, oracle_refs, rel_err,
                      require_gpu, split_grad, step_tensors)

pytestmark = pytest.mark.gpu
TOL = 2e-2
# Bounds against the plain oracle where 2e-2 does not hold, by (workload,
# rays) and tensor: the first-layer weight gradient of the cone-beam network
# (measured 2.6 % and 2.7 % on a B300; 0.7 % and 0.8 % against the oracle
# with BF16-taken ReLU decisions): units whose pre-activation lies within
# BF16 rounding of zero flip between the two forwards, and each flip moves
# a whole delta entry of that unit into the gradient sum.
PLAIN_TOL = {(3, 64): {"dW layer 0": 4e-2}, (3, 160): {"dW layer 0": 4e-2}}


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def _grad_check(g_gpu, g_or, net, tol):
    for L, ((gw, gb), (ow, ob)) in enumerate(zip(split_grad(g_gpu, net), split_grad(g_or, net))):
        assert_close(gw, ow, tol, f"dW layer {L}")
        assert_close(gb, ob, tol, f"db layer {L}")


@pytest.fixture(scope="module")
def c1():
    w = wl.workload(1)
    idx = wl.ray_subset(w.geom.n_proj, 1024, w.seeds["sampler"])
    m, theta, proj = make_model(w, "bf16", idx=idx)
    plain, decided = oracle_refs(theta, w.geom, w.net, idx, proj, "bf16")
    yield w, m, theta, proj, idx, plain, decided
    m.close()


def _gate(label, w, p_bar, grad, plain, decided, tol=TOL, plain_tol=None):
    net = w.net
    gate_tensors(label, step_tensors(p_bar, grad, net),
                 step_tensors(plain["p_bar"], plain["grad"], net),
                 step_tensors(decided["p_bar"], decided["grad"], net), tol, plain_tol)


def test_c1_forward_model_bf16(c1):
    w, m, theta, proj, idx, plain, decided = c1
    p = m.predict(idx).cpu().numpy()
    assert_close(p, decided["p_bar"], TOL, "p_bar (BF16-decided oracle)")
    assert_close(p, plain["p_bar"], TOL, "p_bar (plain oracle)")


def test_c1_loss_and_gradient_bf16(c1):
    w, m, theta, proj, idx, plain, decided = c1
    p = m.predict(idx).cpu().numpy()
    loss, grad = m.loss_grad(idx)
    for ref in (plain, decided):
        assert abs(loss.item() - ref["loss"]) <= TOL * ref["loss"]
    _gate("workload 1, 1024 rays", w, p, grad.cpu().numpy(), plain, decided)


def test_c1_deterministic_bf16(c1):
    w, m, theta, proj, idx, plain, decided = c1
    l1, g1 = m.loss_grad(idx)
    l2, g2 = m.loss_grad(idx)
    assert l1.item() == l2.item() and torch.equal(g1, g2)


def test_c1_ragged_batches_bf16(c1):
    """Batches that leave the 128-row tiles ragged. A single ray sums only
    32 samples per gradient entry, and sign cancellation in so short a sum
    magnifies the BF16 rounding of the operands; its gradient is held to
    5e-2, every other quantity to the path's 2e-2. Against the plain
    oracle, the gradients of batches of at most five rays (160 samples) are
    held to 5e-2: in so short a sum one unit whose ReLU decision flips moves
    an entry by a whole delta (measured 3.2 % and 3.5 % norm-wise, 4.7 %
    element-wise for 1 and 5 rays; 0.3 % with BF16-taken decisions)."""
    w, m, theta, proj, idx, plain, decided = c1
    for n in (1, 5, 129):
        sub = idx[:n]
        pl, de = oracle_refs(theta, w.geom, w.net, sub, proj, "bf16")
        p = m.predict(sub).cpu().numpy()
        loss, grad = m.loss_grad(sub)
        for ref in (pl, de):
            assert abs(loss.item() - ref["loss"]) <= TOL * ref["loss"] + 1e-9
        t = TOL if n > 1 else 5e-2
        _gate(f"workload 1, {n} rays", w, p, grad.cpu().numpy(), pl, de, tol=t,
              plain_tol=5e-2 if n <= 5 else None)


def test_c1_train_step_bf16(c1):
    w, m, theta, proj, idx, plain, decided = c1
    st = m.get_state()
    loss = m.train_step(idx)
    assert abs(loss - plain["loss"]) <= TOL * plain["loss"]
    out = ostep.train_step(theta, np.zeros_like(theta), np.zeros_like(theta), 1, w.geom, w.net,
                           w.train, idx, proj.astype(np.float64))
    d_gpu = m.params().cpu().numpy() - theta
    d_or = out["theta"] - theta
    big = np.abs(out["grad"]) > 1e-2 * np.abs(out["grad"]).max()
    assert rel_err(d_gpu[big], d_or[big]) <= 5e-2
    m.set_state(st)


def test_c1_queries_bf16(c1):
    w, m, theta, proj, idx, plain, decided = c1
    g, net = w.geom, w.net
    rng = np.random.default_rng(3)
    coords = np.stack([rng.uniform(0, 1, 300), rng.uniform(-1, 1, 300),
                       rng.uniform(-0.7, 0.7, 300), rng.uniform(-0.7, 0.7, 300)], 1)
    coords = coords.astype(np.float32).astype(np.float64)
    assert_close(m.query(coords).cpu().numpy(), ostep.query(theta, g, net, coords), TOL, "query")
    img = m.project(1.1, 0.3, 20, 24, 40).cpu().numpy()
    assert_close(img, ostep.project_view(theta, g, net, 1.1, 0.3, 20, 24, 40), TOL, "project")


@pytest.mark.parametrize("c,n", [(2, 128), (3, 64), (2, 512), (3, 160)])
def test_subset_parity_bf16(c, n):
    """Subsets of the benchmark (parallel beam, 5x256) and cone-beam (6x256)
    workloads. 128 and 64 rays are 128 tiles, fewer than the chains' 148
    CTAs (one tile per CTA); 512 rays of 128 samples (512 tiles) and 160
    rays of 256 samples (320 tiles) give every CTA two or more tiles, so
    both slots of the chains' tile ping-pong and a second pair run, in the
    forward and in the backward chain."""
    w = wl.workload(c)
    idx = wl.ray_subset(w.geom.n_proj, n, 99)
    m, theta, proj = make_model(w, "bf16", idx=idx, batch=n)
    try:
        check_step(m, w, w.net, theta, idx, proj, "bf16", plain_tol=PLAIN_TOL.get((c, n)),
                   label=f"workload {c}, {n} rays")
    finally:
        m.close()


def test_bf16_matches_fp32_path_full_batch_c2():
    """At the full 65,536-ray batch of the parallel-beam workload the two
    library paths agree (the FP32 path is within 1e-5 of the oracle on
    subsets), checked on p_bar of the whole batch and on the gradient."""
    from paper_2404_19075_b300 import phantom_project
    w = wl.workload(2)
    proj = phantom_project(w.geom, wl.phantom(w))
    th = wl.he_init(w.net, w.seeds["weights"]).astype(np.float32)
    idx = torch.as_tensor(wl.ray_subset(w.geom.n_proj, 65536, 5), device="cuda")
    from paper_2404_19075_b300 import Dinr
    out = {}
    for prec in ("fp32", "bf16"):
        m = Dinr(w.geom, w.net, w.train, proj, prec=prec, init_params=th)
        p = m.predict(idx).cpu().numpy()
        loss, grad = m.loss_grad(idx)
        out[prec] = (p, loss.item(), grad.cpu().numpy())
        m.close()
    assert_close(out["bf16"][0], out["fp32"][0], TOL, "p_bar")
    assert abs(out["bf16"][1] - out["fp32"][1]) <= TOL * out["fp32"][1]
    _grad_check(out["bf16"][2], out["fp32"][2], w.net, TOL)
