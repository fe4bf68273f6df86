"""Full-size parity in the launch configuration the benchmark times: the
whole minibatch of a workload (65,536 rays at the workload's samples per
ray, through its network, in one call of the library) is predicted, and the
FP64 oracle recomputes the prediction of a seeded sample of those rays one
by one (with ReLU, against the plain oracle and against the oracle with its
ReLU decisions taken on the BF16-rounded forward, as the BF16 path takes
them). Workloads: the parallel-beam benchmark (2), the cone-beam
network (3), the paper's network (6) and the paper's network with its
sub-pixel forward model (8). BF16 tolerance 2e-2."""
import numpy as np
import pytest
import torch

from oracle import network as onet
from oracle import step as ostep
from synthetic import workloads as wl

from gpu_util import assert_close, make_model, plain_gate, require_gpu

pytestmark = pytest.mark.gpu
TOL = 2e-2


def oracle_p_bar(theta, geom, net, idx, decide_bf16):
    """p_bar of rays idx (Eq. 1-2; App. A for sub-pixel geometries), FP64."""
    if getattr(geom, "subpixels", 0) > 0:
        e, wgt, pix, n_pix = ostep.subpixel_model(geom, net, idx)
        masks = onet.relu_decisions_bf16(theta, net, e) if decide_bf16 else None
        M, _ = onet.forward(theta, net, e, masks)
        return ostep.forward_model_subpixel(M, wgt, pix, n_pix)
    S = geom.samples_per_ray
    e, l = ostep.encoded_samples(geom, net, idx)
    masks = onet.relu_decisions_bf16(theta, net, e) if decide_bf16 else None
    M, _ = onet.forward(theta, net, e, masks)
    return ostep.forward_model(M.reshape(len(idx), S), l, S, geom.mu0)


@pytest.mark.parametrize("c", [2, 3, 6, 8])
def test_full_batch_sampled_rays_match_oracle(c):
    require_gpu()
    w = wl.workload(c)
    B = w.train.batch_rays
    idx = wl.ray_subset(w.geom.n_proj, B, 21)
    m, theta, _ = make_model(w, "bf16", batch=B)
    try:
        p = m.predict(idx).cpu().numpy()
    finally:
        m.close()
    assert p.shape == (B,) and np.isfinite(p).all()
    pick = np.sort(np.random.default_rng(22).choice(B, 96, replace=False))
    plain = oracle_p_bar(theta, w.geom, w.net, idx[pick], False)
    if w.net.act == "relu":
        decided = oracle_p_bar(theta, w.geom, w.net, idx[pick], True)
        assert_close(p[pick], decided, TOL, f"p_bar of sampled rays, workload {c} (BF16-decided)")
        plain_gate(f"full batch, workload {c}", "p_bar of sampled rays", p[pick], plain, TOL,
                   decided)
    else:
        assert_close(p[pick], plain, TOL, f"p_bar of sampled rays, workload {c}")
