"""Failure detection without a GPU fault: a kernel's bounded wait is made
to run out (a barrier nothing arrives on, limit 50 ms), the call reports
DINR_ERR_TIMEOUT like a real timeout, and the context stays usable: the
next step is bitwise the one of a fresh context."""
import time

import pytest

from paper_2404_19075_b300 import DinrError, _abi
from synthetic import workloads as wl

from gpu_util import make_model, require_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_bounded_wait_times_out_and_context_stays_usable(prec):
    require_gpu()
    w = wl.workload(1)
    idx = wl.ray_subset(w.geom.n_proj, 256, 17)
    m, theta, proj = make_model(w, prec, idx=idx, batch=256)
    t0 = time.perf_counter()
    with pytest.raises(DinrError) as ei:
        m.selftest_timeout(0.05)
    dt = time.perf_counter() - t0
    assert ei.value.status == _abi.ERR_TIMEOUT
    assert 0.05 <= dt < 2.0
    l1, g1 = m.loss_grad(idx)
    fresh, _, _ = make_model(w, prec, idx=idx, batch=256)
    l2, g2 = fresh.loss_grad(idx)
    assert l1.item() == l2.item()
    assert bool((g1 == g2).all())
    m.close()
    fresh.close()
