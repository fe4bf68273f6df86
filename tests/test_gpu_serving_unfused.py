"""The query server on networks the fused chain does not take: an FP32
context, a BF16 context of width 512 (two 256-column N tiles) and an FP8
context.
The same mixed requests as the fused-chain tests, in small batches so that
large requests span several pieces: every result bitwise equals the
single-query call of the same request."""
from dataclasses import replace

import numpy as np
import pytest

from synthetic import workloads as wl

from gpu_util import make_model, require_gpu
from test_gpu_serving import _requests, _serve

pytestmark = pytest.mark.gpu


def _single(m, kind, kw):
    if kind == "grid":
        return m.query_grid(kw["t"], kw["lo"], kw["hi"], kw["dims"]).cpu().numpy().ravel()
    if kind == "points":
        return m.query(kw["coords"]).cpu().numpy()
    return m.project(kw["theta"], kw["t"], kw["rows"], kw["cols"], kw["S"]).cpu().numpy().ravel()


@pytest.mark.parametrize("prec,W", [("fp32", 64), ("bf16", 512), ("fp8", 256)])
def test_served_equals_single_queries(prec, W):
    require_gpu()
    w = wl.workload(1)
    net = replace(w.net, width=W, hidden_layers=2)
    m, theta, _ = make_model(w, prec, net=net, batch=256,
                             params=wl.he_init(net, w.seeds["weights"]))
    try:
        reqs = _requests(5)
        m.serve_config(max_batch_samples=2048)
        m.profile(True)
        served = _serve(m, reqs)
        m.profile(False)
        assert "tc_serve_chain" not in m.profile_report()
        for (kind, kw), got in zip(reqs, served):
            assert np.isfinite(got).all()
            assert np.array_equal(got, _single(m, kind, kw)), kind
    finally:
        m.close()
