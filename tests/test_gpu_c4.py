"""GPU parity of the wide network (8 hidden layers of 512, 12 octaves) on the
cone-beam geometry: the N-tiled BF16 path against the FP64 oracle on a
64-ray subset (tolerance 2e-2, ReLU decisions taken in BF16 on both sides),
and activation recomputation on vs off (bitwise equal loss and gradient,
several passes per step)."""
import numpy as np
import pytest
import torch

from oracle import step as ostep
from synthetic import workloads as wl

from gpu_util import assert_close, make_model, projections_for, require_gpu, split_grad

pytestmark = pytest.mark.gpu
TOL = 2e-2


@pytest.fixture(scope="module")
def c4():
    require_gpu()
    w = wl.workload(4)
    idx = wl.ray_subset(w.geom.n_proj, 512, w.seeds["sampler"])
    proj = projections_for(w, idx)
    return w, idx, proj


def test_c4_gradient_bf16_vs_oracle(c4):
    w, idx, proj = c4
    sub = idx[:64]
    m, theta, _ = make_model(w, "bf16", proj=proj, batch=64)
    ref = ostep.loss_and_grad(theta, w.geom, w.net, sub, proj.astype(np.float64), decide="bf16")
    assert_close(m.predict(sub).cpu().numpy(), ref["p_bar"], TOL, "p_bar")
    loss, grad = m.loss_grad(sub)
    assert abs(loss.item() - ref["loss"]) <= TOL * ref["loss"]
    g = grad.cpu().numpy()
    for L, ((gw, gb), (ow, ob)) in enumerate(zip(split_grad(g, w.net), split_grad(ref["grad"], w.net))):
        assert_close(gw, ow, TOL, f"dW layer {L}")
        assert_close(gb, ob, TOL, f"db layer {L}")
    m.close()


def test_c4_recompute_bitwise_equal(c4):
    w, idx, proj = c4
    out = {}
    for rc in (0, 1):
        m, theta, _ = make_model(w, "bf16", proj=proj, batch=512, chunk=256, recompute=rc)
        m.profile(True)
        loss, grad = m.loss_grad(idx)
        m.profile(False)
        rep = m.profile_report()
        st0 = m.get_state()
        m.train_step(idx)
        out[rc] = (loss.clone(), grad.clone(), m.params().clone(), rep)
        m.close()
    assert torch.equal(out[0][0], out[1][0])
    assert torch.equal(out[0][1], out[1][1])
    assert torch.equal(out[0][2], out[1][2])
    assert "tc_fwd_recompute" not in out[0][3]
    assert out[1][3]["tc_fwd_recompute"]["launches"] > 0
