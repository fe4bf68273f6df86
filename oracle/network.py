"""The coordinate network M(r; gamma) and its backward, in FP64.

Appendix B: normalised coordinates -> Fourier features -> hidden
fully-connected layers with an activation -> a final linear layer to one
scalar (no activation in the paper).

Readings of the workloads this library targets (where they differ from the
paper's defaults):
  * encoding: octave positional features instead of the paper's Gaussian
    random Fourier features: [t, z, y, x, then for each coordinate c in
    (t, z, y, x) and octave l = 0..F-1: sin(2^l pi c), cos(2^l pi c)], so the
    input width is 4 + 8F (52 for F = 6).
  * activation: ReLU with relu'(0) = 0 (the paper's Swish is an option).
  * output: identity as in the paper, or softplus log(1 + e^z).
  * parameter layout (flat): [W_1 (W x d_in, row-major), b_1, W_2, b_2, ...,
    W_H, b_H, w_out (W), b_out].

The backward is the chain rule written out by hand (the gradient equation
of Appendix A, label "partiald", states the gradient of the loss through the
forward model; the
network part is ordinary back-propagation). No automatic differentiation.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np


def encode(rbar, n_freq: int):
    """Octave Fourier features of normalised coordinates rbar [..., 4]
    ordered (t, z, y, x). Returns [..., 4 + 8F]."""
    rbar = np.asarray(rbar, np.float64)
    feats = [rbar]
    for c in range(4):
        for l in range(n_freq):
            ang = (2.0 ** l) * np.pi * rbar[..., c]
            feats.append(np.sin(ang)[..., None])
            feats.append(np.cos(ang)[..., None])
    return np.concatenate(feats, axis=-1)


def encode_grff(rbar, B):
    """Gaussian random Fourier features (App. B item 2) of normalised
    coordinates rbar [..., 4] with the frozen matrix B [C][4]:
    [cos(2 pi B rbar), sin(2 pi B rbar)], the C cosines first. Returns
    [..., 2C]."""
    u = np.asarray(rbar, np.float64) @ np.asarray(B, np.float64).T
    return np.concatenate([np.cos(2.0 * np.pi * u), np.sin(2.0 * np.pi * u)], axis=-1)


def encode_net(rbar, net):
    """The encoding the network uses (octave features or GRFF)."""
    if getattr(net, "encoding", "octave") == "grff":
        return encode_grff(rbar, net.grff_B)
    return encode(rbar, net.n_freq)


def layer_shapes(net):
    shapes = [(net.width, net.d_in)]
    shapes += [(net.width, net.width)] * (net.hidden_layers - 1)
    shapes.append((1, net.width))
    return shapes


def unpack(theta, net):
    """Views (W_k, b_k) into the flat parameter vector, output layer last."""
    out, p = [], 0
    for o, i in layer_shapes(net):
        W = theta[p:p + o * i].reshape(o, i)
        p += o * i
        b = theta[p:p + o]
        p += o
        out.append((W, b))
    if p != theta.size:
        raise ValueError("parameter vector does not match the network shape")
    return out


def act(z, kind):
    if kind == "relu":
        return np.maximum(z, 0.0)
    if kind == "swish":
        return z / (1.0 + np.exp(-z))
    raise ValueError(kind)


def act_grad(z, kind):
    if kind == "relu":
        return (z > 0.0).astype(np.float64)
    if kind == "swish":
        s = 1.0 / (1.0 + np.exp(-z))
        return s * (1.0 + z * (1.0 - s))
    raise ValueError(kind)


def out_act(z, kind):
    if kind == "identity":
        return z
    if kind == "softplus":
        return np.logaddexp(0.0, z)
    raise ValueError(kind)


def out_act_grad(z, kind):
    if kind == "identity":
        return np.ones_like(z)
    if kind == "softplus":
        return 1.0 / (1.0 + np.exp(-z))
    raise ValueError(kind)


def round_bf16(x):
    """Round to the nearest BF16 value (8 significant bits, ties to even),
    returned as float64. Used only to take ReLU decisions in BF16."""
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def relu_decisions_bf16(theta, net, e):
    """Which hidden units are active, decided the way a BF16 tensor-core
    forward decides them: operands (features, weights, activations) rounded
    to BF16, products summed in FP32, bias added in FP32. Returns one
    boolean mask per hidden layer. (A ReLU mask is an integer decided by
    floating point; to compare a BF16 path with this oracle both take that
    decision in BF16, while every value stays FP64.)"""
    layers = unpack(theta, net)
    h = round_bf16(e).astype(np.float32)
    masks = []
    for W, b in layers[:-1]:
        z = h @ round_bf16(W).astype(np.float32).T + np.asarray(b, np.float32)
        masks.append(z > 0)
        h = round_bf16(np.maximum(z, 0)).astype(np.float32)
    return masks


def forward(theta, net, e, masks=None):
    """M(r; gamma) for encoded inputs e [n, d_in]. Returns (M [n], cache).
    masks: optional ReLU decisions per hidden layer (default: z > 0)."""
    layers = unpack(theta, net)
    h = np.asarray(e, np.float64)
    hs, zs = [h], []
    for k, (W, b) in enumerate(layers[:-1]):
        z = h @ W.T + b
        if masks is not None:
            h = np.where(masks[k], z, 0.0)
        else:
            h = act(z, net.act)
        zs.append(z)
        hs.append(h)
    w_out, b_out = layers[-1]
    z_out = h @ w_out[0] + b_out[0]
    return out_act(z_out, net.out_act), dict(hs=hs, zs=zs, z_out=z_out, masks=masks)


def backward(theta, net, cache, dM):
    """Gradient of sum_n dM[n] * M_n with respect to the flat parameters.

    dz_out = dM * out'(z_out); grad w_out = h_H^T dz_out; then for each
    hidden layer from the last: delta_k = (upstream) * act'(z_k),
    grad W_k = delta_k^T h_{k-1}, grad b_k = sum delta_k, and the upstream
    of the layer below is delta_k W_k."""
    layers = unpack(theta, net)
    grads = [None] * len(layers)
    hs, zs = cache["hs"], cache["zs"]
    dz = dM * out_act_grad(cache["z_out"], net.out_act)
    w_out = layers[-1][0]
    grads[-1] = (np.outer(np.ones(1), dz @ hs[-1]), np.array([dz.sum()]))
    up = np.outer(dz, w_out[0])
    for k in range(len(layers) - 2, -1, -1):
        if cache.get("masks") is not None:
            delta = up * cache["masks"][k]
        else:
            delta = up * act_grad(zs[k], net.act)
        grads[k] = (delta.T @ hs[k], delta.sum(axis=0))
        if k > 0:
            up = delta @ layers[k][0]
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return flat
