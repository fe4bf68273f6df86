"""Queries on a cone-beam geometry (source-to-object 4, source-to-detector
8): a re-projection at an angle and time between the views, on a detector
of another size covering the same area, against the FP64 oracle (FP32 1e-5,
BF16 2e-2), and the same re-projection served by the query server, bitwise
the single call."""
from dataclasses import replace

import numpy as np
import pytest
import torch

from oracle import step as ostep
from synthetic import workloads as wl

from gpu_util import TOL, assert_close, make_model, require_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_cone_reprojection(prec):
    require_gpu()
    k = np.arange(64.0)
    geom = wl.cone_geometry(64, 32, 32, 2 * np.pi * k / 64, k / 64, 32)
    w = replace(wl.workload(1), geom=geom)
    m, theta, _ = make_model(w, prec, batch=64)
    try:
        img = m.project(1.3, 0.45, 24, 20, 48).cpu().numpy()
        want = ostep.project_view(theta, geom, w.net, 1.3, 0.45, 24, 20, 48)
        assert np.isfinite(img).all()
        assert_close(img, want, TOL[prec], "cone re-projection")
        if prec == "bf16":
            out = torch.full((24 * 20,), float("nan"), device="cuda")
            m.serve_config(max_batch_samples=4096)   # the request spans several launches
            rid = m.serve_submit("project", out, t=0.45, theta=1.3, rows=24, cols=20, S=48)
            assert rid is not None
            for _ in range(100000):
                m.serve_step()
                if m.serve_poll(rid):
                    break
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy(), img.ravel())
    finally:
        m.close()
