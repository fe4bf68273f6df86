"""Training steps replayed from a CUDA graph of one step (dinr_train_graph)
against the same number of ordinary steps, through the C ABI: the same
minibatches from the built-in sampler, the same App. C learning rates
across epoch boundaries and Adam bias corrections, so the parameters,
Adam moments and loss must be bitwise equal; a second call reuses the
graph, a new minibatch size captures a new one, and App. A steps (which
read sample counts back) run as ordinary steps."""
import numpy as np
import pytest
import torch

from oracle import phantom as ophantom
from synthetic import workloads as wl

from gpu_util import make_model, require_gpu

pytestmark = pytest.mark.gpu


def _pair(prec):
    from paper_2404_19075_b300 import Dinr
    w = wl.workload(1)
    k = np.arange(8.0)
    g = wl.parallel_geometry(8, 16, 16, np.pi * k / 8, k / 8, 32)   # 2,048 pixels
    proj = ophantom.projections(wl.phantom(w), g, np.arange(g.n_proj)).astype(np.float32)
    theta = wl.he_init(w.net, w.seeds["weights"]).astype(np.float32)
    tr = wl.Train(512, lr=1e-3, lr_decay_per_epoch=0.95)          # four steps per epoch
    return [Dinr(g, w.net, tr, proj, prec=prec, init_params=theta, sampler_seed=7)
            for _ in range(2)]


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_graph_steps_equal_ordinary_steps(prec):
    require_gpu()
    a, b = _pair(prec)
    try:
        for _ in range(7):
            la = a.train_step(None, n=512)
        b.train_graph(512, 3, sync=False)
        lb = b.train_graph(512, 4)            # the same graph, the next four steps
        assert la == lb
        assert torch.equal(a.params(), b.params())
        assert a.get_state() == b.get_state()   # parameters, moments, step counter
        # a different minibatch size captures a new graph
        for _ in range(2):
            la = a.train_step(None, n=256)
        lb = b.train_graph(256, 2)
        assert la == lb and a.get_state() == b.get_state()
        # ordinary steps continue from the graph's step counter
        assert a.train_step(None, n=512) == b.train_step(None, n=512)
        assert a.get_state() == b.get_state()
    finally:
        a.close()
        b.close()


def test_graph_call_runs_app_a_steps_as_ordinary_steps():
    require_gpu()
    w = wl.workload(9)
    idx = wl.ray_subset(w.geom.n_proj, 64, 5)
    out = []
    for graph in (False, True):
        m, theta, proj = make_model(w, "bf16", idx=idx, batch=64)
        try:
            if graph:
                loss = m.train_graph(64, 2)
            else:
                m.train_step(None, n=64)
                loss = m.train_step(None, n=64)
            out.append((loss, m.get_state()))
        finally:
            m.close()
    assert out[0] == out[1]


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_host_index_steps_replayed_equal_ordinary_steps(prec):
    """Host-index steps that read the loss back run as one graph launch each
    (captured once per minibatch size); without the loss read-back they run
    as ordinary launches. Both must give bitwise the same state, across an
    epoch boundary of the App. C decay and a change of minibatch size."""
    require_gpu()
    a, b = _pair(prec)
    rng = np.random.default_rng(11)
    try:
        for k in range(7):
            n = 512 if k < 5 else 384
            idx = torch.from_numpy(rng.integers(0, 2048, n)).pin_memory()
            la = a.train_step_host(idx, sync=True)        # graph replay
            b.train_step_host(idx, sync=False)             # ordinary launches
            assert la == b.loss()
        assert torch.equal(a.params(), b.params())
        assert a.get_state() == b.get_state()
    finally:
        a.close()
        b.close()
