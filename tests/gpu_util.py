"""Helpers shared by the GPU parity tests: build a library context for a
workload with the oracle's inputs, and the comparison measures."""
import numpy as np
import pytest
import torch

from oracle import phantom as ophantom
from oracle import step as ostep
from synthetic import workloads as wl


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def rel_err(got, want):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    return float(np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-300))


def assert_close(got, want, tol, what=""):
    """Norm-wise relative error <= tol and every element within
    tol * max|want| (the measure the tolerances are stated in)."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    assert got.shape == want.shape, (what, got.shape, want.shape)
    r = rel_err(got, want)
    m = float(np.abs(got - want).max()) / max(float(np.abs(want).max()), 1e-300)
    assert r <= tol and m <= tol, f"{what}: norm-wise {r:.3e}, element-wise {m:.3e} > {tol}"


def split_grad(g, net):
    """Per-layer (W, b) views of a flat gradient, output layer last."""
    out, p = [], 0
    for o, i in net.layer_shapes():
        out.append((g[p:p + o * i], g[p + o * i:p + o * i + o]))
        p += o * i + o
    return out


def projections_for(w, idx):
    """A full projection stack with the oracle's exact phantom projections
    at the indices used (zeros elsewhere)."""
    g = w.geom
    p = np.zeros(g.n_proj, np.float32)
    p[idx] = ophantom.projections(wl.phantom(w), g, idx)
    return p


def make_model(w, prec, idx=None, proj=None, net=None, geom=None, batch=None, chunk=0,
               params=None, recompute=0):
    from paper_2404_19075_b300 import Dinr
    net = net or w.net
    geom = geom or w.geom
    if params is None:
        params = wl.he_init(net, w.seeds["weights"])
    if proj is None:
        proj = projections_for(w, idx) if idx is not None else np.zeros(geom.n_proj, np.float32)
    train = wl.Train(batch or w.train.batch_rays)
    m = Dinr(geom, net, train, proj, prec=prec, init_params=params.astype(np.float32),
             sampler_seed=w.seeds["sampler"], chunk_rays=chunk, recompute=recompute)
    return m, params.astype(np.float32).astype(np.float64), proj


TOL = {"fp32": 1e-5, "bf16": 2e-2}


def errors(got, want):
    """(norm-wise relative, element-wise relative to max|want|) errors."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    m = float(np.abs(got - want).max()) / max(float(np.abs(want).max()), 1e-300)
    return rel_err(got, want), m


def plain_gate(label, name, got, want, bound, decided=None):
    """The BF16 path against the unmodified FP64 oracle (ReLU decided on
    the FP64 pre-activations): both error measures within `bound`. Prints
    both errors, and those against the oracle with BF16-taken ReLU decisions
    when given (the diagnostic that separates mask flips from rounding)."""
    r, m = errors(got, want)
    line = f"PARITY {label} {name}: plain oracle {r:.3e} / {m:.3e}"
    if decided is not None:
        rd, md = errors(got, decided)
        line += f"; BF16-decided {rd:.3e} / {md:.3e}"
    print(line)
    assert r <= bound and m <= bound, f"{label} {name}: plain oracle {r:.3e} / {m:.3e} > {bound}"


def oracle_refs(theta, geom, net, idx, proj, prec):
    """The FP64 oracle's loss, p_bar and gradient for the minibatch, and for
    the BF16 path with ReLU also the same with the ReLU decisions taken on
    a BF16-rounded forward (None otherwise)."""
    proj = np.asarray(proj, np.float64)
    plain = ostep.loss_and_grad(theta, geom, net, idx, proj)
    decided = None
    if prec == "bf16" and net.act == "relu":
        decided = ostep.loss_and_grad(theta, geom, net, idx, proj, decide="bf16")
    return plain, decided


def step_tensors(p_bar, grad, net):
    """p_bar, then every layer's weight and bias gradients, then the output
    layer's weights and bias as one tensor (its bias gradient is one number,
    a sum of signed residuals in which cancellation magnifies rounding)."""
    out = {"p_bar": np.asarray(p_bar, np.float64)}
    parts = split_grad(np.asarray(grad, np.float64), net)
    for L, (gw, gb) in enumerate(parts[:-1]):
        out[f"dW layer {L}"] = gw
        out[f"db layer {L}"] = gb
    gw, gb = parts[-1]
    out["output layer"] = np.concatenate([gw, gb])
    return out


def gate_tensors(label, got, plain, decided, tol, plain_tol=None):
    """Every tensor of `got` (dicts as step_tensors makes them) within tol of
    the oracle. Without `decided` (FP32 path, Swish) that is the plain
    oracle. With it (BF16 path with ReLU), each tensor is held to tol
    against the oracle that takes the ReLU decisions in BF16, and to
    plain_tol (a number, or a dict by tensor name; default tol) against the
    plain oracle."""
    for name, g in got.items():
        if decided is None:
            assert_close(g, plain[name], tol, f"{label} {name}")
            continue
        assert_close(g, decided[name], tol, f"{label} {name} (BF16-decided oracle)")
        b = plain_tol.get(name, tol) if isinstance(plain_tol, dict) else (
            tol if plain_tol is None else plain_tol)
        plain_gate(label, name, g, plain[name], b, decided[name])


def check_step(m, w, net, theta, idx, proj, prec, tol=None, plain_tol=None, label=""):
    """p_bar, loss and every layer's weight and bias gradients within the
    path's tolerance (or `tol`) of the FP64 oracle; for the BF16 path with
    ReLU against both the plain oracle (bound plain_tol, default the same)
    and the oracle with BF16-taken ReLU decisions (see gate_tensors)."""
    t = TOL[prec] if tol is None else tol
    plain, decided = oracle_refs(theta, w.geom, net, idx, proj, prec)
    p_bar = m.predict(idx).cpu().numpy()
    loss, grad = m.loss_grad(idx)
    assert abs(loss.item() - plain["loss"]) <= t * plain["loss"] + 1e-12
    if decided is not None:
        assert abs(loss.item() - decided["loss"]) <= t * decided["loss"] + 1e-12
    got = step_tensors(p_bar, grad.cpu().numpy(), net)
    gate_tensors(label or f"{net.hidden_layers}x{net.width} {net.act}", got,
                 step_tensors(plain["p_bar"], plain["grad"], net),
                 None if decided is None else step_tensors(decided["p_bar"], decided["grad"], net),
                 t, plain_tol)
