"""CPU pins of the oracle's encoding, network, forward model, gradient and
Adam against special values, hand expansion, brute force, invariants and
finite differences."""
import math
import os
from types import SimpleNamespace

import numpy as np
import pytest

from oracle import network, step
from synthetic import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------- encoding

def test_encoding_special_values():
    F = 6
    e = network.encode(np.array([[0.0, 0.5, -0.5, 1.0]]), F)[0]
    assert e.shape == (4 + 8 * F,)
    assert np.array_equal(e[:4], [0.0, 0.5, -0.5, 1.0])
    sin = lambda c, l: e[4 + 2 * (c * F + l)]
    cos = lambda c, l: e[4 + 2 * (c * F + l) + 1]
    for l in range(F):
        assert sin(0, l) == 0.0 and cos(0, l) == 1.0            # c = 0
        assert abs(sin(3, l)) < 1e-12                            # c = 1: sin(2^l pi)
        assert abs(cos(3, l) - (-1.0 if l == 0 else 1.0)) < 1e-12
    # c = 1/2: sin(pi/2) = 1, cos(pi) = -1, cos(2^l pi/2) = 1 for l >= 2
    assert abs(sin(1, 0) - 1) < 1e-15 and abs(cos(1, 1) + 1) < 1e-15
    assert all(abs(cos(1, l) - 1) < 1e-12 for l in range(2, F))
    assert abs(sin(2, 0) + 1) < 1e-15                             # c = -1/2


def test_encoding_octave_doubling():
    r = np.random.default_rng(1).uniform(-1, 1, (100, 4))
    F = 10
    e = network.encode(r, F)
    s = e[:, 4:].reshape(100, 4, F, 2)
    assert np.allclose(s[..., 0] ** 2 + s[..., 1] ** 2, 1.0)
    # sin(2a) = 2 sin a cos a between consecutive octaves
    assert np.allclose(s[:, :, 1:, 0], 2 * s[:, :, :-1, 0] * s[:, :, :-1, 1], atol=1e-12)
    assert np.allclose(s[:, :, 0, 0], np.sin(math.pi * r))


# -------------------------------------------------------------- network

def test_mlp_hand_expanded_tiny():
    """H = 1, W = 2, F = 0 (4 inputs), softplus output, written out
    scalar by scalar."""
    net = SimpleNamespace(n_freq=0, d_in=4, hidden_layers=1, width=2, act="relu",
                          out_act="softplus")
    W = np.array([[0.5, -1.0, 0.25, 2.0], [-0.3, 0.7, 1.1, -0.4]])
    b = np.array([0.1, -0.2])
    wo, bo = np.array([1.5, -0.75]), 0.3
    theta = np.concatenate([W.ravel(), b, wo, [bo]])
    r = np.array([0.2, -0.4, 0.9, 0.1])
    h0 = max(0.0, 0.5 * 0.2 - 1.0 * -0.4 + 0.25 * 0.9 + 2.0 * 0.1 + 0.1)
    h1 = max(0.0, -0.3 * 0.2 + 0.7 * -0.4 + 1.1 * 0.9 - 0.4 * 0.1 - 0.2)
    z = 1.5 * h0 - 0.75 * h1 + 0.3
    want = math.log(1.0 + math.exp(z))
    M, _ = network.forward(theta, net, r[None, :])
    assert abs(M[0] - want) < 1e-15


def test_mlp_brute_force_loops():
    """H = 2, W = 3, F = 1: explicit loops over every product."""
    net = SimpleNamespace(n_freq=1, d_in=12, hidden_layers=2, width=3, act="relu",
                          out_act="identity")
    rng = np.random.default_rng(5)
    theta = rng.normal(size=sum(o * i + o for o, i in network.layer_shapes(net)))
    rbar = rng.uniform(-1, 1, (7, 4))
    e = network.encode(rbar, 1)
    layers = network.unpack(theta, net)
    for n in range(7):
        x = list(e[n])
        for W, bb in layers[:-1]:
            y = []
            for o in range(W.shape[0]):
                acc = bb[o]
                for i in range(W.shape[1]):
                    acc += W[o, i] * x[i]
                y.append(acc if acc > 0 else 0.0)
            x = y
        acc = layers[-1][1][0]
        for i in range(3):
            acc += layers[-1][0][0, i] * x[i]
        M, _ = network.forward(theta, net, e[n:n + 1])
        assert abs(M[0] - acc) < 1e-13


def test_param_count_paper():
    with open(os.path.join(GOLDEN, "param_count.txt")) as f:
        d_in, H, W, P = [int(x) for ln in f if ln.strip() and not ln.startswith("#")
                         for x in ln.split()]
    net = SimpleNamespace(d_in=d_in, hidden_layers=H, width=W)
    assert sum(o * i + o for o, i in network.layer_shapes(net)) == P
    assert wl.workload(1).net.n_params == 11777       # 64*52+64 + 2*(64*64+64) + 65


# ------------------------------------------- forward model and loss (Eq. 1-5)

def _small(act="relu", out_act="softplus", B=24, S=8):
    wk = wl.workload(1)
    g = wl.parallel_geometry(64, 32, 32, wk.geom.view_angle, wk.geom.view_time, S)
    net = wl.Net(2, 2, 8, act, out_act)
    theta = wl.he_init(net, 2001)
    idx = wl.ray_subset(g.n_proj, B, 3001)
    return g, net, theta, idx


def test_loss_zero_at_self_generated_data():
    g, net, theta, idx = _small()
    proj = np.zeros(g.n_proj)
    proj[idx] = step.loss_and_grad(theta, g, net, idx, proj)["p_bar"]
    out = step.loss_and_grad(theta, g, net, idx, proj)
    assert out["loss"] == 0.0
    assert np.abs(out["grad"]).max() == 0.0


def test_forward_model_is_linear_in_outputs():
    """dp_bar_i / dM_ij = mu0 * l_i / S (Eq. 1, 2), exactly."""
    M = np.random.default_rng(2).normal(size=(5, 16))
    l = np.array([0.5, 1.0, 1.5, 2.0, 0.0])
    base = step.forward_model(M, l, 16, 0.75)
    for i in range(5):
        for j in (0, 7, 15):
            M2 = M.copy()
            M2[i, j] += 1.0
            dp = step.forward_model(M2, l, 16, 0.75) - base
            assert abs(dp[i] - 0.75 * l[i] / 16) < 1e-14
            assert np.all(np.delete(dp, i) == 0)


def test_loss_is_mean_square():
    p_bar = np.array([1.0, 2.0, 3.0])
    p = np.array([1.5, 2.0, 1.0])
    assert step.loss(p_bar, p) == pytest.approx((0.25 + 0 + 4) / 3, abs=1e-15)


# --------------------------------------------------------- gradients (App. A)

@pytest.mark.parametrize("act,out_act", [("swish", "softplus"), ("swish", "identity")])
def test_gradient_central_differences_smooth(act, out_act):
    g, net, theta, idx = _small(act, out_act)
    proj = np.random.default_rng(3).uniform(0, 1, g.n_proj)
    out = step.loss_and_grad(theta, g, net, idx, proj)
    ks = np.random.default_rng(4).choice(theta.size, 32, replace=False)
    ks[:2] = [0, theta.size - 1]                  # first weight, output bias
    for k in ks:
        fd = step.fd_grad(theta, g, net, idx, proj, k, h=1e-5)
        assert abs(fd - out["grad"][k]) <= 1e-7 * max(1e-3, abs(out["grad"]).max()), k


def test_gradient_central_differences_relu():
    """ReLU has kinks; with h = 1e-7 no pre-activation of this batch changes
    sign, which the test checks before comparing."""
    g, net, theta, idx = _small("relu", "softplus")
    proj = np.random.default_rng(3).uniform(0, 1, g.n_proj)
    out = step.loss_and_grad(theta, g, net, idx, proj)
    ks = np.random.default_rng(6).choice(theta.size, 32, replace=False)
    for k in ks:
        fd = step.fd_grad(theta, g, net, idx, proj, k, h=1e-7)
        assert abs(fd - out["grad"][k]) <= 1e-6 * max(1e-3, abs(out["grad"]).max()), k


# ----------------------------------------------------------------- Adam

def test_adam_first_step_and_constant_gradient():
    """Bias correction makes m_hat = g and v_hat = g^2 whenever the gradient
    has been constant, so every step moves by -lr * g / (|g| + eps)."""
    g = np.array([3.0, -2e-3, 0.0, 1e-9])
    th, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    for t in range(1, 6):
        new, m, v = step.adam(th, m, v, g, t, 1e-3)
        assert np.allclose(new - th, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-18)
        th = new


def test_train_step_descends():
    g, net, theta, idx = _small(B=64)
    proj = np.random.default_rng(8).uniform(0, 0.5, g.n_proj)
    tr = wl.Train(64, lr=1e-3)
    m = v = np.zeros_like(theta)
    L0 = step.loss_and_grad(theta, g, net, idx, proj)["loss"]
    th = theta
    for t in range(1, 11):
        out = step.train_step(th, m, v, t, g, net, tr, idx, proj)
        th, m, v = out["theta"], out["m"], out["v"]
    assert step.loss_and_grad(th, g, net, idx, proj)["loss"] < L0


def test_query_matches_network_at_sample_points():
    """Voxel queries evaluate mu0 * M at given (t, z, y, x)."""
    g, net, theta, idx = _small()
    coords = np.array([[0.25, 0.1, -0.2, 0.3], [0.9, -0.9, 0.0, 0.0]])
    rbar = np.stack([2 * coords[:, 0] - 1, coords[:, 1], coords[:, 2], coords[:, 3]], 1)
    M, _ = network.forward(theta, net, network.encode(rbar, net.n_freq))
    assert np.allclose(step.query(theta, g, net, coords), g.mu0 * M)


# ------------------------------------------- BF16 decisions (comparison aid)

def test_round_bf16_definition():
    """Round to nearest with 8 significant bits, ties to even."""
    vals = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -9, -2.5,
                     1.0 + 2.0 ** -7 + 2.0 ** -8, 3.0e38])
    want = np.array([1.0, 1.0, 1.0 + 2.0 ** -6, 1.0, -2.5, 1.0 + 2.0 ** -6, 2.9980e38])
    got = network.round_bf16(vals)
    assert np.array_equal(got[:6], want[:6])
    assert abs(got[6] / 3.0e38 - 1) < 2 ** -8


def test_bf16_decisions_only_change_near_kinks():
    """Deciding ReLUs in BF16 changes the network only where a
    pre-activation is within BF16 rounding of zero; with all decisions equal
    to z > 0 the FP64 results are unchanged."""
    g, net, theta, idx = _small(B=48)
    e, l = step.encoded_samples(g, net, idx)
    masks = network.relu_decisions_bf16(theta, net, e)
    _, cache = network.forward(theta, net, e)
    for k, z in enumerate(cache["zs"]):
        differ = masks[k] != (z > 0)
        assert differ.mean() < 0.01
        assert np.all(np.abs(z[differ]) < 0.05 * np.abs(z).max())
    exact = [z > 0 for z in cache["zs"]]
    M1, _ = network.forward(theta, net, e, exact)
    M0, _ = network.forward(theta, net, e)
    assert np.array_equal(M1, M0)


# ---------------------------------------------------------- GRFF (App. B)

def test_grff_reproduces_octave_features():
    """cos/sin(2 pi b . r) with b = 2^(l-1) e_k is the octave feature
    sin/cos(2^l pi r_k): pins the 2 pi, B's orientation (row per frequency,
    column per coordinate t, z, y, x) and the cosines-first order."""
    F = 5
    rbar = np.random.default_rng(0).uniform(-1, 1, (50, 4))
    rows = [(k, l) for k in range(4) for l in range(F)]
    B = np.zeros((len(rows), 4))
    for i, (k, l) in enumerate(rows):
        B[i, k] = 2.0 ** (l - 1)
    g = network.encode_grff(rbar, B)
    o = network.encode(rbar, F)
    C = len(rows)
    for i, (k, l) in enumerate(rows):
        col = 4 + 2 * F * k + 2 * l          # octave layout: sin, cos
        assert np.allclose(g[:, C + i], o[:, col], atol=1e-12)
        assert np.allclose(g[:, i], o[:, col + 1], atol=1e-12)


def test_grff_zero_matrix_and_unit_pairs():
    rbar = np.random.default_rng(1).uniform(-1, 1, (20, 4))
    g0 = network.encode_grff(rbar, np.zeros((8, 4)))
    assert np.array_equal(g0[:, :8], np.ones((20, 8))) and np.array_equal(g0[:, 8:], np.zeros((20, 8)))
    B = wl.workload(6).net.grff_B
    g = network.encode_grff(rbar, B)
    C = B.shape[0]
    assert np.allclose(g[:, :C] ** 2 + g[:, C:] ** 2, 1.0, atol=1e-12)


def test_grff_matrix_columns():
    """Column 0 (time) has std sigma_t, columns 1-3 (z, y, x) sigma_s; values
    are FP32-representable so the GPU gets exactly the oracle's B."""
    from dataclasses import replace
    net = replace(wl.workload(6).net, grff_c=20000)
    B = net.grff_B
    sd = B.std(axis=0)
    assert abs(sd[0] / net.sigma_t - 1) < 0.03
    assert np.all(np.abs(sd[1:] / net.sigma_s - 1) < 0.03)
    assert np.array_equal(B, B.astype(np.float32).astype(np.float64))


def test_paper_network_parameter_count():
    """2C = 256 GRFF inputs, L = 5 Swish layers of 256, linear output: the
    parameter count the paper prints (329,217)."""
    net = wl.workload(6).net
    assert (net.d_in, net.hidden_layers, net.width, net.act) == (256, 5, 256, "swish")
    assert net.n_params == 329217
