"""The fused chains at the widths, depths and encodings the benchmark
workloads do not use: one, two or three 64-column chunks per layer (an odd
count splits unevenly between the two epilogue warps of a lane quadrant),
layer-0 inputs wider than the hidden layers, every octave count the chain
is built for, ReLU and Swish, softplus and identity outputs. BF16 p_bar,
loss and every gradient against the FP64 oracle (2e-2; with ReLU against
the plain oracle and the one with BF16-taken ReLU decisions), on a ragged batch (8,000 samples: 62.5 tiles), and
the profile shows that both chains ran."""
from dataclasses import replace

import pytest

from synthetic import workloads as wl

from gpu_util import check_step, make_model, require_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("W,H,F,act,out_act", [
    (128, 3, 8, "relu", "softplus"),
    (192, 2, 12, "relu", "identity"),
    (64, 4, 16, "relu", "identity"),
    (192, 3, 10, "swish", "identity"),
    (128, 2, 6, "swish", "softplus"),
])
def test_chain_shapes(W, H, F, act, out_act):
    require_gpu()
    w = wl.workload(1)
    net = replace(w.net, width=W, hidden_layers=H, n_freq=F, act=act, out_act=out_act)
    idx = wl.ray_subset(w.geom.n_proj, 250, 31)
    m, theta, proj = make_model(w, "bf16", idx=idx, net=net, batch=250,
                                params=wl.he_init(net, w.seeds["weights"]))
    try:
        m.profile(True)
        check_step(m, w, net, theta, idx, proj, "bf16", label=f"chain {H}x{W} F={F} {act}")
        m.profile(False)
        report = m.profile_report()
        assert "tc_fwd_chain" in report and "tc_bwd_chain" in report
    finally:
        m.close()
