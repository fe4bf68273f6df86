"""The autograd split of the training step through the C ABI: a forward
that runs the forward model and the loss only (no backward kernel
launches), and a backward that launches the adjoint kernels on the
activations the forward kept (one workspace pass) or recomputes them
(several passes). Both give bitwise the gradient of the combined
loss-and-gradient call; the upstream factor scales it; a backward with no
forward to differentiate is refused."""
import numpy as np
import pytest
import torch

from synthetic import workloads as wl

from gpu_util import make_model, require_gpu

pytestmark = pytest.mark.gpu


def _kernels(m):
    rep = m.profile_report()
    return {k for k, v in rep.items() if not k.startswith("total_") and v["launches"] > 0}


@pytest.mark.parametrize("prec,chunk", [("bf16", 0), ("bf16", 300), ("fp32", 0), ("fp32", 300)])
def test_forward_then_backward_equals_loss_grad(prec, chunk):
    require_gpu()
    w = wl.workload(1)
    idx = wl.ray_subset(w.geom.n_proj, 1024, 61)
    m, theta, proj = make_model(w, prec, idx=idx, batch=1024, chunk=chunk)
    try:
        loss_ref, grad_ref = m.loss_grad(idx)
        m.profile(True)
        loss = m.forward_loss(idx)
        m.profile(False)
        fwd = _kernels(m)
        assert torch.equal(loss, loss_ref)
        if prec == "bf16":
            assert "tc_fwd_chain" in fwd
            assert not fwd & {"tc_bwd_chain", "tc_dw", "dw_out"}, fwd
        else:
            assert not any(k.startswith("sgemm_d") or k.startswith("dw") for k in fwd), fwd
        m.profile(True)
        grad = m.backward_grad()
        m.profile(False)
        bwd = _kernels(m)
        assert torch.equal(grad, grad_ref)
        if prec == "bf16":
            assert {"tc_bwd_chain", "tc_dw"} <= bwd
            # one pass: the kept activations, no forward again; several: recomputed
            assert ("tc_fwd_chain" in bwd) == (chunk != 0), bwd
        # the upstream factor of an autograd backward
        g3 = m.backward_grad(torch.tensor([3.0], device="cuda"))
        assert torch.equal(g3, grad_ref * 3.0)
    finally:
        m.close()


@pytest.mark.parametrize("case", ["subpixel", "wide", "fp8"])
def test_split_on_other_paths(case):
    """The same split on the App. A forward model (sub-pixel rays through
    the fused chains, two passes), the wide unfused network (512-wide
    layers) and the FP8 forward variant: bitwise the combined call."""
    require_gpu()
    from dataclasses import replace
    if case == "subpixel":
        w = wl.workload(9)
        n, prec, chunk, net = 96, "bf16", 48, wl.workload(9).net
    elif case == "wide":
        w = wl.workload(1)
        net = replace(w.net, width=512, hidden_layers=2, out_act="identity")
        n, prec, chunk = 64, "bf16", 0
    else:
        w = wl.workload(3)
        n, prec, chunk, net = 64, "fp8", 0, wl.workload(3).net
    idx = wl.ray_subset(w.geom.n_proj, n, 64)
    params = wl.he_init(net, w.seeds["weights"])
    # two fresh contexts (the FP8 delayed scales move after every step)
    m1, _, proj = make_model(w, prec, idx=idx, net=net, batch=n, chunk=chunk, params=params)
    m2, _, _ = make_model(w, prec, proj=proj, net=net, batch=n, chunk=chunk, params=params)
    try:
        loss_ref, grad_ref = m1.loss_grad(idx)
        loss = m2.forward_loss(idx)
        grad = m2.backward_grad()
        assert torch.equal(loss, loss_ref)
        assert torch.equal(grad, grad_ref)
    finally:
        m1.close()
        m2.close()


def test_autograd_function_bf16():
    require_gpu()
    from paper_2404_19075_b300 import DinrStep
    w = wl.workload(1)
    idx = wl.ray_subset(w.geom.n_proj, 512, 62)
    m, theta, proj = make_model(w, "bf16", idx=idx, batch=512)
    try:
        _, grad_ref = m.loss_grad(idx)
        p = torch.tensor(theta, dtype=torch.float32, device="cuda", requires_grad=True)
        m.profile(True)
        loss = DinrStep.apply(p, m, torch.as_tensor(idx, device="cuda"))
        m.profile(False)
        assert not _kernels(m) & {"tc_bwd_chain", "tc_dw", "dw_out"}
        (2.0 * loss).backward()
        assert torch.equal(p.grad, 2.0 * grad_ref)
    finally:
        m.close()


def test_backward_without_a_forward_is_refused():
    require_gpu()
    from paper_2404_19075_b300 import DinrError
    w = wl.workload(1)
    idx = wl.ray_subset(w.geom.n_proj, 256, 63)
    m, theta, proj = make_model(w, "bf16", idx=idx, batch=256)
    try:
        with pytest.raises(DinrError, match="no dinr_forward"):
            m.backward_grad()
        m.forward_loss(idx)
        m.predict(idx[:10])                 # restages the indices
        with pytest.raises(DinrError, match="no dinr_forward"):
            m.backward_grad()
        m.forward_loss(idx)
        m.set_params(torch.tensor(theta, dtype=torch.float32, device="cuda"))
        with pytest.raises(DinrError, match="no dinr_forward"):
            m.backward_grad()
    finally:
        m.close()
