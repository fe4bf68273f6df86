"""Steps split into several passes (the workspace holds fewer rays than the
minibatch): the fused chains over four passes and the App. A forward model
with the unfused wide network and activation recomputation, against the
FP64 oracle (BF16 2e-2, against the plain oracle and the one with
BF16-taken ReLU decisions), and
recomputation on vs off bitwise equal on the App. A model."""
from dataclasses import replace

import pytest
import torch

from synthetic import workloads as wl

from gpu_util import check_step, make_model, require_gpu

pytestmark = pytest.mark.gpu


def test_chains_over_four_passes():
    require_gpu()
    w = wl.workload(1)
    idx = wl.ray_subset(w.geom.n_proj, 1024, 41)
    m, theta, proj = make_model(w, "bf16", idx=idx, batch=1024, chunk=300)
    try:
        m.profile(True)
        check_step(m, w, w.net, theta, idx, proj, "bf16", label="passes chains")
        m.profile(False)
        assert m.profile_report()["tc_fwd_chain"]["launches"] >= 4
    finally:
        m.close()


def test_subpixel_wide_network_recompute():
    require_gpu()
    w = wl.workload(9)
    net = replace(w.net, act="relu", out_act="softplus", encoding="octave", grff_c=0,
                  n_freq=6, width=512, hidden_layers=4)
    idx = wl.ray_subset(w.geom.n_proj, 96, 43)
    params = wl.he_init(net, w.seeds["weights"])
    out = {}
    for rc in (0, 1):
        m, theta, proj = make_model(w, "bf16", idx=idx, net=net, batch=96, chunk=40,
                                    params=params, recompute=rc)
        try:
            if rc == 1:
                m.profile(True)
                check_step(m, w, net, theta, idx, proj, "bf16", label="passes App. A wide")
                m.profile(False)
                assert m.profile_report()["tc_fwd_recompute"]["launches"] > 0
            loss, grad = m.loss_grad(idx)
            out[rc] = (loss.clone(), grad.clone())
        finally:
            m.close()
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
