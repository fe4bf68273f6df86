"""Forward model, loss, gradient, Adam and the whole training step in FP64.

Sec. III, Eq. 1 and Eq. 2: p_bar_i = (1/|Phi_i|) sum_j w(r_ij) M(r_ij; gamma)
with w = mu0 * l, where l is the length of the ray inside the cylindrical
FOV. With one ray of S samples per pixel |Phi_i| = S, so
p_bar_i = mu0 * (l_i / S) * sum_j M_ij.
Eq. 3 and Eq. 5: d_i = (p_i - p_bar_i)^2 and L = (1/|Omega|) sum d_i over the
minibatch Omega.
Appendix A (gradient equation "partiald"):
dL/dgamma = (1/|Omega|) sum_i 2 (p_bar_i - p_i) (1/S) sum_j mu0 l_i dM_ij/dgamma.
Sec. III and Appendix C: Adam (Kingma & Ba 2015, bias-corrected, defaults
beta = (0.9, 0.999), eps = 1e-8) with learning rate 1e-3.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from . import geometry, network


def encoded_samples(geom, net, idx):
    """Rays of the minibatch, their samples and Fourier features.
    Returns (e [n*S, d_in], l [n])."""
    o, d, s0, l, t = geometry.rays(geom, idx)
    P = geometry.sample_points(o, d, s0, l, geom.samples_per_ray)
    rbar = geometry.normalize(geom, P, t[:, None])
    e = network.encode_net(rbar, net)
    return e.reshape(-1, net.d_in), l


def subpixel_model(geom, net, idx):
    """App. A forward model of the minibatch: D x D rays per pixel, samples
    about Delta/D apart inside the FOV. Returns the features of all samples
    (ray by ray, pixel by pixel), each sample's weight factor mu0 * l of
    its ray (Eq. 2), each sample's pixel and |Phi_i| of each pixel."""
    D2 = geom.subpixels ** 2
    o, d, s0, l, t = geometry.subpixel_rays(geom, idx)
    n = geometry.subpixel_counts(geom, l)
    P, ray = geometry.subpixel_samples(o, d, s0, l, n)
    rbar = geometry.normalize(geom, P, t[ray])
    e = network.encode_net(rbar, net).reshape(-1, net.d_in)
    return e, geom.mu0 * l[ray], ray // D2, n.reshape(-1, D2).sum(axis=1)


def forward_model_subpixel(M, w, pix, n_pix):
    """Eq. 1 over the pixel's samples Phi_i: p_bar_i = (1/|Phi_i|) sum_j
    w(r_ij) M(r_ij), 0 for a pixel none of whose rays meets the FOV."""
    tot = np.bincount(pix, weights=w * M, minlength=len(n_pix))
    return np.where(n_pix > 0, tot / np.maximum(n_pix, 1), 0.0)


def forward_model(M, l, S: int, mu0: float):
    """Eq. 1 with w = mu0*l (Eq. 2) and |Phi| = S. M: [n, S]."""
    return mu0 * (l / S) * M.sum(axis=1)


def loss(p_bar, p):
    """Eq. 3 summed as in Eq. 5 (mean over the minibatch)."""
    r = p_bar - p
    return float(np.mean(r * r))


def loss_and_grad(theta, geom, net, idx, proj, decide=None):
    """Loss of Eq. 5 and its gradient (Appendix A, "partiald") for the
    minibatch idx against the projection stack proj (flat, length MN).
    decide="bf16" takes the ReLU decisions in BF16 (see
    network.relu_decisions_bf16); all values are FP64 either way."""
    S, B = geom.samples_per_ray, len(idx)
    p = np.asarray(proj, np.float64)[np.asarray(idx)]
    if getattr(geom, "subpixels", 0) > 0:
        e, w, pix, n_pix = subpixel_model(geom, net, idx)
        masks = network.relu_decisions_bf16(theta, net, e) if decide == "bf16" else None
        M, cache = network.forward(theta, net, e, masks)
        p_bar = forward_model_subpixel(M, w, pix, n_pix)
        L = loss(p_bar, p)
        # dL/dM_ij = (2/B) (p_bar_i - p_i) * w(r_ij) / |Phi_i|
        dM = (2.0 / B) * (p_bar - p)[pix] * w / np.maximum(n_pix, 1)[pix]
        g = network.backward(theta, net, cache, dM)
        return dict(loss=L, p_bar=p_bar, grad=g, M=M, dM=dM, n_pix=n_pix)
    e, l = encoded_samples(geom, net, idx)
    masks = network.relu_decisions_bf16(theta, net, e) if decide == "bf16" else None
    M, cache = network.forward(theta, net, e, masks)
    M = M.reshape(B, S)
    p_bar = forward_model(M, l, S, geom.mu0)
    L = loss(p_bar, p)
    # dL/dM_ij = (2/B) (p_bar_i - p_i) * mu0 * l_i / S
    dM = (2.0 / B) * (p_bar - p)[:, None] * (geom.mu0 * l / S)[:, None] * np.ones((1, S))
    g = network.backward(theta, net, cache, dM.reshape(-1))
    return dict(loss=L, p_bar=p_bar, grad=g, l=l, M=M, dM=dM)


def adam(theta, m, v, g, t: int, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One bias-corrected Adam update at step t >= 1. Returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return theta - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def lr_at(train, epoch: int) -> float:
    """Appendix C: the learning rate is multiplied by a fixed factor after
    every epoch (0.95 in the paper; 1.0 disables the decay)."""
    return train.lr * (train.lr_decay_per_epoch ** epoch)


def train_step(theta, m, v, t: int, geom, net, train, idx, proj, epoch=0):
    """One stochastic training step (Sec. III, Fig. 1(d) on one process):
    forward model, loss, gradient, Adam. t is the 1-based Adam step."""
    out = loss_and_grad(theta, geom, net, idx, proj)
    th, m2, v2 = adam(theta, m, v, out["grad"], t, lr_at(train, epoch),
                      train.beta1, train.beta2, train.eps)
    out.update(theta=th, m=m2, v=v2)
    return out


def project_view(theta, geom, net, view_theta, view_t, rows, cols, S):
    """Re-projection of the network at angle view_theta and time view_t on a
    rows x cols detector covering the same physical area as the
    acquisition detector. Returns [rows, cols]."""
    pu = geom.det_pitch_u * geom.det_cols / cols
    pv = geom.det_pitch_v * geom.det_rows / rows
    col, row = np.meshgrid(np.arange(cols), np.arange(rows))
    u = geom.det_off_u + (col.ravel() + 0.5) * pu
    v = geom.det_off_v + (row.ravel() + 0.5) * pv
    o, d = geometry.rays_at(geom, view_theta, u, v)
    s0, l = geometry.fov_chord(geom, o, d)
    P = geometry.sample_points(o, d, s0, l, S)
    rbar = geometry.normalize(geom, P, view_t)
    M, _ = network.forward(theta, net, network.encode_net(rbar, net).reshape(-1, net.d_in))
    return forward_model(M.reshape(-1, S), l, S, geom.mu0).reshape(rows, cols)


def query(theta, geom, net, coords):
    """Reconstructed attenuation mu0 * M at object coordinates
    coords [n, 4] ordered (t, z, y, x) (Sec. V: inference on a 4D grid)."""
    coords = np.asarray(coords, np.float64)
    P = coords[:, [3, 2, 1]]
    rbar = geometry.normalize(geom, P, coords[:, 0])
    M, _ = network.forward(theta, net, network.encode_net(rbar, net))
    return geom.mu0 * M


def fd_grad(theta, geom, net, idx, proj, k, h=1e-3):
    """Central finite difference of the loss in parameter k."""
    tp = theta.copy()
    tp[k] += h
    tm = theta.copy()
    tm[k] -= h
    return (loss_and_grad(tp, geom, net, idx, proj)["loss"]
            - loss_and_grad(tm, geom, net, idx, proj)["loss"]) / (2.0 * h)
