"""Twenty Adam steps of the parity workload (1,024 rays x 32 samples, 3x64,
exact phantom projections), the library and the FP64 oracle stepping side
by side on the same minibatches (the library's sampler draws them): the
loss of every step and the reconstruction mu0 * M on a 16^3 grid at
t = 0.5 after the last step, against the oracle's. Adam's normalisation
amplifies the rounding of near-zero gradient entries over a trajectory, so
the bounds are looser than a single step's: losses 1e-4 (FP32) and 3e-2
(BF16) relative, the volume 5e-5 (FP32) and 2e-2 (BF16) relative L2
(measured on a B300: 1.1e-5 and 4.5e-3)."""
import numpy as np
import pytest

from oracle import phantom as ophantom
from oracle import step as ostep
from synthetic import workloads as wl

from gpu_util import make_model, rel_err, require_gpu

pytestmark = pytest.mark.gpu
LOSS_TOL = {"fp32": 1e-4, "bf16": 3e-2}
VOL_TOL = {"fp32": 5e-5, "bf16": 2e-2}


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_twenty_steps_against_the_oracle(prec):
    require_gpu()
    w = wl.workload(1)
    g, net, train = w.geom, w.net, w.train
    proj = ophantom.projections(wl.phantom(w), g, np.arange(g.n_proj)).astype(np.float32)
    m, theta, _ = make_model(w, prec, proj=proj)
    th, mo, vo = theta.copy(), np.zeros_like(theta), np.zeros_like(theta)
    p64 = proj.astype(np.float64)
    try:
        for t in range(1, 21):
            idx = m.sample_indices(t - 1, train.batch_rays).cpu().numpy()
            loss = m.train_step(idx)
            out = ostep.train_step(th, mo, vo, t, g, net, train, idx, p64)
            th, mo, vo = out["theta"], out["m"], out["v"]
            assert abs(loss - out["loss"]) <= LOSS_TOL[prec] * out["loss"], (t, loss, out["loss"])
        n = 16
        ax = -1 + (np.arange(n) + 0.5) * 2 / n
        Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
        pts = np.stack([np.full(X.size, 0.5), Z.ravel(), Y.ravel(), X.ravel()], 1)
        want = ostep.query(th, g, net, pts)
        got = m.query_grid(0.5, (-1, -1, -1), (1, 1, 1), (n, n, n)).cpu().numpy().ravel()
        err = rel_err(got, want)
        print(f"{prec}: volume after 20 steps, relative L2 {err:.3e}")
        assert err <= VOL_TOL[prec]
    finally:
        m.close()
