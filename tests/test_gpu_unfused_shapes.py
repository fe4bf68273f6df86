"""The unfused tcgen05 GEMM path (one kernel per layer) at the shapes the
fused chains do not take: widths that are not whole 64-column chunks (96,
224) and wide layers split into three or four 256-column N tiles (768,
1024), with ReLU and Swish. BF16 p_bar, loss and every gradient against the
FP64 oracle (2e-2; with ReLU against the plain oracle and the one with
BF16-taken ReLU decisions) on a ragged batch
(8,000 samples), and the profile shows the per-layer GEMMs ran."""
from dataclasses import replace

import pytest

from synthetic import workloads as wl

from gpu_util import check_step, make_model, require_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("W,H,F,act,out_act", [
    (96, 2, 6, "relu", "softplus"),
    (224, 3, 10, "swish", "identity"),
    (768, 2, 6, "relu", "identity"),
    (1024, 2, 4, "relu", "softplus"),
])
def test_unfused_shapes(W, H, F, act, out_act):
    require_gpu()
    w = wl.workload(1)
    net = replace(w.net, width=W, hidden_layers=H, n_freq=F, act=act, out_act=out_act)
    idx = wl.ray_subset(w.geom.n_proj, 250, 37)
    m, theta, proj = make_model(w, "bf16", idx=idx, net=net, batch=250,
                                params=wl.he_init(net, w.seeds["weights"]))
    try:
        m.profile(True)
        check_step(m, w, net, theta, idx, proj, "bf16", label=f"unfused {H}x{W} F={F} {act}")
        m.profile(False)
        report = m.profile_report()
        assert "tc_fwd" in report and "tc_dw" in report and "tc_fwd_chain" not in report
    finally:
        m.close()
