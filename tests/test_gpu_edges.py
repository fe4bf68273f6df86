"""Degenerate and edge inputs on both GPU paths, through the C ABI: rays
whose chord misses the field of view (cone-beam detector corners, l = 0)
predict exactly 0 and contribute exactly zero gradient while still counting
in the 1/B of the loss; mixed batches of empty and full rays match the FP64
oracle; a minibatch of one ray and one empty ray works at every tile
boundary the chains have."""
import numpy as np
import pytest
import torch

from oracle import geometry
from synthetic import workloads as wl

from gpu_util import gate_tensors, make_model, oracle_refs, projections_for, require_gpu

pytestmark = pytest.mark.gpu
TOL = {"fp32": 1e-5, "bf16": 2e-2}


def _corner_rays(g):
    N = g.det_rows * g.det_cols
    idx = [m * N + r * g.det_cols + c for m in (0, 100, 511, 1023)
           for r in (0, 1, 2, g.det_rows - 1) for c in (0, 1, g.det_cols - 1)]
    idx = np.array(idx, np.int64)
    assert (geometry.rays(g, idx)[3] == 0).all()
    return idx


@pytest.fixture(scope="module")
def cone():
    require_gpu()
    w = wl.workload(3)
    empty = _corner_rays(w.geom)
    full = wl.ray_subset(w.geom.n_proj, 80, 99)
    full = full[geometry.rays(w.geom, full)[3] > 0][:64]
    proj = projections_for(w, np.concatenate([empty, full]))
    # measurements where the ray misses: nonzero on purpose, the residual
    # then enters the loss but no gradient flows through the empty ray
    proj[empty] = 0.25
    return w, empty, full, proj


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_empty_rays(cone, prec):
    w, empty, full, proj = cone
    m, theta, _ = make_model(w, prec, proj=proj, batch=256)
    assert torch.count_nonzero(m.predict(empty)) == 0
    loss, grad = m.loss_grad(empty)
    assert torch.count_nonzero(grad) == 0
    assert abs(loss.item() - 0.25 ** 2) <= 1e-7
    mix = np.concatenate([full[:32], empty, full[32:]])
    plain, decided = oracle_refs(theta, w.geom, w.net, mix, proj, prec)
    p = m.predict(mix).cpu().numpy()
    assert (p[32:32 + len(empty)] == 0).all()
    loss, grad = m.loss_grad(mix)
    assert abs(loss.item() - plain["loss"]) <= TOL[prec] * plain["loss"]
    got = {"p_bar": p, "grad": grad.cpu().numpy()}
    gate_tensors(f"empty and full rays {prec}", got, plain, decided, TOL[prec])
    m.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_single_full_and_single_empty_ray(cone, prec):
    w, empty, full, proj = cone
    m, theta, _ = make_model(w, prec, proj=proj, batch=256)
    for sub in (full[:1], empty[:1], np.array([full[0], empty[0]])):
        ref, decided = oracle_refs(theta, w.geom, w.net, sub, proj, prec)
        p = m.predict(sub).cpu().numpy().astype(np.float64)
        gate_tensors(f"single rays {prec}", {"p_bar": p}, ref, decided, TOL[prec])
        loss, grad = m.loss_grad(sub)
        # the loss of one or two rays is (p_bar - p)^2 with cancellation in
        # the difference, so the tolerance is held on p_bar above; the loss
        # must be the one of the path's own p_bar (and, in FP32, the oracle's)
        own = float(np.mean((p - proj[sub].astype(np.float64)) ** 2))
        assert abs(loss.item() - own) <= 1e-5 * own + 1e-9
        if prec == "fp32":
            assert abs(loss.item() - ref["loss"]) <= TOL[prec] * ref["loss"] + 1e-9
        if np.abs(ref["grad"]).max() == 0:
            assert torch.count_nonzero(grad) == 0
        else:
            # one ray of 256 samples: the per-ray tolerance of the BF16 path
            gate_tensors(f"single rays {prec} n={len(sub)}", {"grad": grad.cpu().numpy()}, ref,
                         decided, TOL[prec] if prec == "fp32" else 5e-2)
    m.close()
