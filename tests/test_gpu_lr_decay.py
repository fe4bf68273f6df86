"""The learning-rate decay of App. C (the rate is multiplied by a fixed
factor, 0.95 in the paper, after every epoch) through the C ABI, beside the
FP64 oracle. A small parallel-beam problem (8 views of 16 x 16 pixels, 512
rays per step: four steps per epoch) trains for twelve steps, three epochs,
on the library's own minibatches, and the oracle takes each step with the
rate of that step's epoch. The loss of every step (1e-4 relative) and the
reconstruction after the last one (5e-5 relative L2, the bounds of the
twenty-step trajectory test) must match; the same oracle run without the
decay must not, so the test sees the decay itself."""
import numpy as np
import pytest

from oracle import phantom as ophantom
from oracle import sampler, step as ostep
from synthetic import workloads as wl

from gpu_util import rel_err, require_gpu

pytestmark = pytest.mark.gpu


def test_lr_decay_over_three_epochs_fp32():
    require_gpu()
    from paper_2404_19075_b300 import Dinr
    w = wl.workload(1)
    k = np.arange(8.0)
    g = wl.parallel_geometry(8, 16, 16, np.pi * k / 8, k / 8, 32)
    net, B = w.net, 512
    ph = wl.phantom(w)
    proj = ophantom.projections(ph, g, np.arange(g.n_proj)).astype(np.float32)
    p64 = proj.astype(np.float64)
    theta = wl.he_init(net, w.seeds["weights"]).astype(np.float32).astype(np.float64)
    tr = wl.Train(B, lr=1e-3, lr_decay_per_epoch=0.95)
    flat = wl.Train(B, lr=1e-3)
    assert sampler.steps_per_epoch(B, g.n_proj) == 4
    m = Dinr(g, net, tr, proj, prec="fp32", init_params=theta.astype(np.float32),
             sampler_seed=w.seeds["sampler"])
    runs = {"decay": (theta.copy(), np.zeros_like(theta), np.zeros_like(theta)),
            "flat": (theta.copy(), np.zeros_like(theta), np.zeros_like(theta))}
    try:
        for t in range(1, 13):
            idx = m.sample_indices(t - 1, B).cpu().numpy()
            loss = m.train_step(idx)
            e = sampler.epoch_of(t - 1, B, g.n_proj)
            for name, trn in (("decay", tr), ("flat", flat)):
                th, mo, vo = runs[name]
                out = ostep.train_step(th, mo, vo, t, g, net, trn, idx, p64, epoch=e)
                runs[name] = (out["theta"], out["m"], out["v"])
                if name == "decay":
                    assert abs(loss - out["loss"]) <= 1e-4 * out["loss"], (t, loss, out["loss"])
        n = 16
        ax = -1 + (np.arange(n) + 0.5) * 2 / n
        Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
        pts = np.stack([np.full(X.size, 0.5), Z.ravel(), Y.ravel(), X.ravel()], 1)
        got = m.query_grid(0.5, (-1, -1, -1), (1, 1, 1), (n, n, n)).cpu().numpy().ravel()
        err = rel_err(got, ostep.query(runs["decay"][0], g, net, pts))
        err_flat = rel_err(got, ostep.query(runs["flat"][0], g, net, pts))
        print(f"volume after 3 epochs: {err:.3e} from the decayed oracle, "
              f"{err_flat:.3e} from the one without decay")
        assert err <= 5e-5
        assert err_flat > 10 * max(err, 5e-6)
    finally:
        m.close()
