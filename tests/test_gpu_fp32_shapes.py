"""The FP32 SIMT path at widths off every tile grid (1, 17, 100, 300),
depths 1 to 3, few or no octaves (d_in = 4 + 8F down to the raw
coordinates), ReLU and Swish, softplus and identity outputs: p_bar, loss and
every gradient against the FP64 oracle at the FP32 tolerance (1e-5), on a
ragged batch."""
from dataclasses import replace

import pytest

from synthetic import workloads as wl

from gpu_util import check_step, make_model, require_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("W,H,F,act,out_act", [
    (17, 1, 0, "swish", "identity"),
    (100, 3, 3, "swish", "softplus"),
    (300, 2, 5, "relu", "identity"),
    (1, 2, 1, "swish", "softplus"),
])
def test_fp32_shapes(W, H, F, act, out_act):
    require_gpu()
    w = wl.workload(1)
    net = replace(w.net, width=W, hidden_layers=H, n_freq=F, act=act, out_act=out_act)
    idx = wl.ray_subset(w.geom.n_proj, 173, 47)
    m, theta, proj = make_model(w, "fp32", idx=idx, net=net, batch=173,
                                params=wl.he_init(net, w.seeds["weights"]))
    try:
        check_step(m, w, net, theta, idx, proj, "fp32")
    finally:
        m.close()
