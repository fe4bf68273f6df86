"""GPU parity of the wide network (8 hidden layers of 512, 12 octaves) on the
cone-beam geometry: the N-tiled BF16 path against the FP64 oracle on a
64-ray subset (tolerance 2e-2 against the plain oracle unless stated, and
against the oracle with ReLU decisions taken in BF16),
and activation recomputation on vs off (bitwise equal loss and gradient,
several passes per step)."""
import numpy as np
import pytest
import torch

from synthetic import workloads as wl

from gpu_util import check_step, make_model, projections_for, require_gpu

pytestmark = pytest.mark.gpu
TOL = 2e-2
# Bound against the plain oracle where 2e-2 does not hold: the first-layer
# weight gradient (measured 2.6 % on a B300, 0.6 % with BF16-taken ReLU
# decisions; units within BF16 rounding of zero flip, each flip moving a
# whole delta entry into the gradient sum).
PLAIN_TOL = {"dW layer 0": 4e-2}


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
    try:
        check_step(m, w, w.net, theta, sub, proj, "bf16", plain_tol=PLAIN_TOL,
                   label="workload 4, 64 rays")
    finally:
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
