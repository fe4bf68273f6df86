"""Pins of the oracle's epoch schedule and learning-rate decay (App. C: the
learning rate is multiplied by 0.95 after every epoch; Sec. III: an epoch
draws every pixel once), checked against facts fixed outside the two
functions: the decay's half-life, the sampler's own epoch coverage, and the
first Adam step, which is linear in the learning rate."""
import math

import numpy as np

from oracle import sampler, step
from synthetic import workloads as wl


def test_lr_at_epoch_zero_and_no_decay():
    tr = wl.Train(64, lr=1e-3)
    assert all(step.lr_at(tr, e) == 1e-3 for e in range(50))
    assert step.lr_at(wl.Train(64, lr=2e-3, lr_decay_per_epoch=0.95), 0) == 2e-3


def test_lr_at_ratio_and_half_life():
    """Each epoch multiplies the rate by the factor; at 0.95 per epoch it
    halves between epochs 13 and 14 (ln 2 / -ln 0.95 = 13.51)."""
    tr = wl.Train(64, lr=1e-3, lr_decay_per_epoch=0.95)
    for e in range(40):
        assert math.isclose(step.lr_at(tr, e + 1) / step.lr_at(tr, e), 0.95, rel_tol=1e-14)
    assert step.lr_at(tr, 13) > 0.5e-3 > step.lr_at(tr, 14)
    assert math.isclose(math.log(2) / -math.log(0.95), 13.513, abs_tol=1e-3)


def test_epoch_of_matches_the_sampler_coverage():
    """Steps the schedule counts as one epoch are exactly the steps whose
    minibatches together cover every pixel once (brute force, tiny n)."""
    for n, B in ((10, 4), (12, 4), (7, 7), (5, 8)):
        spe = sampler.steps_per_epoch(B, n)
        assert spe == math.ceil(n / B)
        for e in range(3):
            steps = [s for s in range(4 * spe) if sampler.epoch_of(s, B, n) == e]
            assert steps == list(range(e * spe, (e + 1) * spe))
            seen = np.concatenate([sampler.minibatch(s, B, n, 7) for s in steps])
            assert set(seen.tolist()) == set(range(n))


def test_first_adam_step_scales_with_the_epoch_rate():
    """Adam's first step is -lr g / (|g| + eps): train_step at epoch 2 must
    move every parameter by 0.95^2 times its move at epoch 0."""
    g = wl.parallel_geometry(4, 4, 4, np.arange(4) * 0.7, np.arange(4) / 4, 8)
    net = wl.Net(n_freq=1, hidden_layers=1, width=4, act="swish", out_act="identity")
    theta = wl.he_init(net, 3)
    idx = np.arange(16)
    proj = np.random.default_rng(2).uniform(0, 0.5, g.n_proj)
    tr = wl.Train(16, lr=1e-3, lr_decay_per_epoch=0.95)
    z = np.zeros_like(theta)
    d0 = step.train_step(theta, z, z, 1, g, net, tr, idx, proj, epoch=0)["theta"] - theta
    d2 = step.train_step(theta, z, z, 1, g, net, tr, idx, proj, epoch=2)["theta"] - theta
    big = np.abs(d0) > 1e-4
    assert big.sum() > theta.size // 2
    assert np.allclose(d2[big] / d0[big], 0.95 ** 2, rtol=1e-9)
