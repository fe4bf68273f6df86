"""Central finite differences of the oracle's gradient at the wide network's
shape (8 hidden layers of 512, 12 octaves, identity output) on the cone-beam
geometry: 32 seeded parameters, step h = 1e-3 in FP64.

With an identity output and fixed ReLU masks the loss is quadratic in any
one parameter, so the central difference is exact up to rounding. A step
that moves a pre-activation across zero changes a mask; the test detects
that (sign patterns of every hidden layer at theta +- h) and takes the
difference again at h = 1e-6, where no mask of this batch changes."""
from dataclasses import replace

import numpy as np

from oracle import network, step
from synthetic import workloads as wl


def _views_subset(g, every):
    return replace(g, n_views=g.n_views // every, view_angle=g.view_angle[::every],
                   view_time=g.view_time[::every])


def _signs(theta, g, net, idx):
    e, _ = step.encoded_samples(g, net, idx)
    _, cache = network.forward(theta, net, e)
    return [z > 0 for z in cache["zs"]]


def test_wide_network_gradient_central_differences():
    w = wl.workload(4)
    g = _views_subset(w.geom, 128)              # 8 views of the schedule, same cone geometry
    net = w.net
    assert (net.hidden_layers, net.width, net.n_freq, net.out_act) == (8, 512, 12, "identity")
    theta = wl.he_init(net, w.seeds["weights"])
    idx = wl.ray_subset(g.n_proj, 2, 4242)      # 2 rays x 256 samples
    proj = np.random.default_rng(5).uniform(0.0, 2.0, g.n_proj)
    out = step.loss_and_grad(theta, g, net, idx, proj)
    grad = out["grad"]
    assert np.abs(grad).max() > 0
    shapes = net.layer_shapes()
    starts = np.cumsum([0] + [o * i + o for o, i in shapes])
    rng = np.random.default_rng(11)
    ks = list(rng.choice(theta.size, 24, replace=False))
    ks += [0, int(starts[1]) - 1,                # first weight, last bias of layer 0
           int(starts[7]), int(starts[8]) - 1,   # first weight, last bias of layer 7
           int(starts[8]), int(starts[8]) + 511, # output weights
           theta.size - 1, int(starts[3]) + 5]   # output bias, a weight of layer 3
    scale = np.abs(grad).max()
    refine = 0
    for k in ks:
        h = 1e-3
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        if any((a != b).any() for a, b in zip(_signs(tp, g, net, idx), _signs(tm, g, net, idx))):
            h, refine = 1e-6, refine + 1
        fd = step.fd_grad(theta, g, net, idx, proj, k, h=h)
        assert abs(fd - grad[k]) <= 1e-6 * scale, (k, h, fd, grad[k])
    assert refine < len(ks)                     # most parameters pass at h = 1e-3
