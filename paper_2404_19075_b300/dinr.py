"""Python binding of libdinr: the calls of the C ABI, with torch CUDA
tensors as device memory and the current torch stream as the context stream.

    model = Dinr(geometry, net, train, proj, prec="bf16")
    loss = model.train_step()                 # one stochastic DINR step
    img = model.project(theta, t, 256, 256, 256)
    vol = model.query_grid(t, lo, hi, (64, 64, 64))

`geometry`, `net` and `train` are any objects with the attribute names of
the C structs (the seeded workloads of this repository provide them).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _abi


class DinrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_abi.STATUS_NAMES[status]}: {msg}")
        self.status = status


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _cuda_f32(x):
    if isinstance(x, torch.Tensor):
        return x.to(device="cuda", dtype=torch.float32).contiguous()
    return torch.as_tensor(np.ascontiguousarray(x, np.float32), device="cuda")


def _cuda_i64(x):
    if isinstance(x, torch.Tensor):
        return x.to(device="cuda", dtype=torch.int64).contiguous()
    return torch.as_tensor(np.ascontiguousarray(x, np.int64), device="cuda")


def param_count(n_freq, hidden_layers, width) -> int:
    """Parameters of an octave-encoded network."""
    return int(_abi.lib().dinr_param_count(n_freq, hidden_layers, width))


def param_count_net(net) -> int:
    """Parameters of a network description (any encoding)."""
    return int(_abi.lib().dinr_param_count_din(net.d_in, net.hidden_layers, net.width))


def geometry_struct(g):
    angle = np.ascontiguousarray(g.view_angle, np.float64)
    time = np.ascontiguousarray(g.view_time, np.float64)
    s = _abi.Geometry(
        _abi.BEAM[g.beam] if isinstance(g.beam, str) else int(g.beam), g.n_views, g.det_rows,
        g.det_cols, angle.ctypes.data_as(C.POINTER(C.c_double)),
        time.ctypes.data_as(C.POINTER(C.c_double)), g.det_pitch_u, g.det_pitch_v,
        g.det_off_u, g.det_off_v, g.sod, g.sdd, g.fov_r, g.fov_z0, g.fov_z1, g.t0, g.t1,
        g.samples_per_ray, g.mu0, getattr(g, "subpixels", 0))
    return s, (angle, time)


def _check(status, ctx=None):
    if status != _abi.OK:
        msg = _abi.lib().dinr_last_error(ctx).decode()
        raise DinrError(status, msg)


class Dinr:
    """One DINR reconstruction on the current CUDA device."""

    def __init__(self, geometry, net, train, proj, prec="bf16", init_params=None,
                 seed=0, sampler_seed=0, chunk_rays=0, recompute=0):
        L = _abi.lib()
        self.geometry, self.net = geometry, net
        gs, self._keep = geometry_struct(geometry)
        self.n_params = param_count_net(net)
        init = None
        if init_params is not None:
            init = np.ascontiguousarray(init_params, np.float32)
            if init.size != self.n_params:
                raise ValueError("init_params has the wrong length")
        enc = getattr(net, "encoding", "octave")
        B = None
        if enc == "grff":
            B = np.ascontiguousarray(net.grff_B, np.float32)
            self._keep = self._keep + (B,)
        ns = _abi.Net(net.n_freq, net.hidden_layers, net.width,
                      _abi.ACT[net.act], _abi.OUT_ACT[net.out_act], _abi.PREC[prec],
                      init.ctypes.data_as(C.POINTER(C.c_float)) if init is not None else None,
                      seed, _abi.ENCODING[enc], net.grff_c if B is not None else 0,
                      B.ctypes.data_as(C.POINTER(C.c_float)) if B is not None else None)
        ts = _abi.Train(train.lr, train.beta1, train.beta2, train.eps,
                        getattr(train, "lr_decay_per_epoch", 1.0), train.batch_rays,
                        chunk_rays, sampler_seed, recompute)
        self.stream = torch.cuda.current_stream()
        proj_t = _cuda_f32(proj)
        self.n_proj = geometry.n_views * geometry.det_rows * geometry.det_cols
        if proj_t.numel() != self.n_proj:
            raise ValueError("projection stack has the wrong size")
        h = C.c_void_p()
        st = L.dinr_create(C.byref(gs), C.byref(ns), C.byref(ts), _ptr(proj_t), 1,
                           C.c_void_p(self.stream.cuda_stream), C.byref(h))
        _check(st, None)
        self._h = h
        self.prec = prec

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            _abi.lib().dinr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _c(self, status):
        _check(status, self._h)

    # -- training
    def _idx(self, idx):
        if idx is None:
            return None, 0, 0
        t = _cuda_i64(idx)
        return t, t.numel(), 1

    def train_step(self, idx=None, n=None, sync=True):
        """One step; returns the loss (float) when sync, else None.
        idx: None (built-in sampler, n rays), a CUDA tensor or an array
        (moved to the device first)."""
        t, m, on_dev = self._idx(idx)
        n = m if t is not None else (n or 0)
        out = C.c_float()
        self._c(_abi.lib().dinr_train_step(self._h, _ptr(t), n, on_dev,
                                           C.byref(out) if sync else None))
        return out.value if sync else None

    def train_graph(self, n, steps, sync=True):
        """`steps` steps of n sampled rays replayed from a CUDA graph of one
        step (bitwise the same as that many train_step(None, n) calls);
        returns the last step's loss when sync, else None."""
        out = C.c_float()
        self._c(_abi.lib().dinr_train_graph(self._h, n, steps, C.byref(out) if sync else None))
        return out.value if sync else None

    def train_step_host(self, idx_host, sync=True):
        """One step with indices in host memory (an int64 numpy array or a
        CPU tensor, ideally pinned); the library copies them itself."""
        if isinstance(idx_host, torch.Tensor):
            assert idx_host.device.type == "cpu" and idx_host.dtype == torch.int64
            ptr, n = C.c_void_p(idx_host.data_ptr()), idx_host.numel()
        else:
            a = np.ascontiguousarray(idx_host, np.int64)
            ptr, n = C.c_void_p(a.ctypes.data), a.size
        out = C.c_float()
        self._c(_abi.lib().dinr_train_step(self._h, ptr, n, 0, C.byref(out) if sync else None))
        return out.value if sync else None

    def loss_grad(self, idx=None, n=None):
        """(loss, grad) as CUDA tensors, no parameter update."""
        t, m, on_dev = self._idx(idx)
        n = m if t is not None else (n or 0)
        loss = torch.empty(1, device="cuda")
        grad = torch.empty(self.n_params, device="cuda")
        self._c(_abi.lib().dinr_loss_grad(self._h, _ptr(t), n, on_dev, _ptr(loss), _ptr(grad)))
        return loss, grad

    def forward_loss(self, idx=None, n=None):
        """The loss of a minibatch (CUDA tensor [1]) from the forward model
        alone; the backward is left for backward_grad."""
        t, m, on_dev = self._idx(idx)
        n = m if t is not None else (n or 0)
        loss = torch.empty(1, device="cuda")
        self._c(_abi.lib().dinr_forward(self._h, _ptr(t), n, on_dev, _ptr(loss)))
        return loss

    def backward_grad(self, dloss=None):
        """Gradient of dloss * L for the minibatch of the last forward_loss
        (dloss: a one-element CUDA float32 tensor, or None for 1)."""
        grad = torch.empty(self.n_params, device="cuda")
        d = None
        if dloss is not None:
            d = dloss.detach().reshape(1).to(device="cuda", dtype=torch.float32).contiguous()
        self._c(_abi.lib().dinr_backward(self._h, _ptr(d), _ptr(grad)))
        return grad

    def predict(self, idx):
        t, n, _ = self._idx(idx)
        out = torch.empty(n, device="cuda")
        self._c(_abi.lib().dinr_predict(self._h, _ptr(t), n, 1, _ptr(out)))
        return out

    def sample_indices(self, step, n):
        out = torch.empty(n, dtype=torch.int64, device="cuda")
        self._c(_abi.lib().dinr_sample_indices(self._h, step, n, _ptr(out)))
        return out

    # -- serving
    def project(self, theta, t, rows, cols, S):
        out = torch.empty(rows * cols, device="cuda")
        self._c(_abi.lib().dinr_project(self._h, float(theta), float(t), rows, cols, S, _ptr(out)))
        return out.view(rows, cols)

    def query(self, coords):
        c = _cuda_f32(coords).view(-1, 4)
        out = torch.empty(c.shape[0], device="cuda")
        self._c(_abi.lib().dinr_query(self._h, _ptr(c), c.shape[0], _ptr(out)))
        return out

    def query_grid(self, t, lo, hi, dims):
        lo_a = (C.c_double * 3)(*lo)
        hi_a = (C.c_double * 3)(*hi)
        d_a = (C.c_int * 3)(*dims)
        out = torch.empty(int(np.prod(dims)), device="cuda")
        self._c(_abi.lib().dinr_query_grid(self._h, float(t), lo_a, hi_a, d_a, _ptr(out)))
        return out.view(dims[2], dims[1], dims[0])

    def selftest_timeout(self, limit_s=0.05):
        """Make a kernel's bounded wait run out (see dinr_selftest_timeout);
        raises DinrError with status TIMEOUT."""
        self._c(_abi.lib().dinr_selftest_timeout(self._h, int(limit_s * 1e9)))

    def export(self, times, lo, hi, dims, sink):
        """4D export: sink(k, t, volume) for each time in order, volume a
        host float32 array [nz, ny, nx] valid during the call (copy it to
        keep it); a sink returning True stops the export (DinrError)."""
        t = np.ascontiguousarray(times, np.float64)
        lo_a, hi_a = (C.c_double * 3)(*lo), (C.c_double * 3)(*hi)
        d_a = (C.c_int * 3)(*dims)
        shape = (dims[2], dims[1], dims[0])

        def _cb(user, k, tk, ptr, n):
            vol = np.ctypeslib.as_array(ptr, shape=(n,)).reshape(shape)
            return 1 if sink(k, tk, vol) else 0

        cb = _abi.VOLUME_SINK(_cb)
        self._c(_abi.lib().dinr_export(self._h, t.ctypes.data_as(C.POINTER(C.c_double)), t.size,
                                       lo_a, hi_a, d_a, cb, None))

    # -- query server (continuous batching)
    def serve_config(self, max_batch_samples=0, max_inflight_bytes=0):
        self._c(_abi.lib().dinr_serve_config(self._h, int(max_batch_samples),
                                             int(max_inflight_bytes)))

    def serve_policy(self, policy="arrival"):
        """Batch scheduling of the query server: "arrival" (default) or
        "least_work" (requests with the least work left first)."""
        self._c(_abi.lib().dinr_serve_policy(self._h, _abi.SERVE_POLICY[policy]))

    def serve_submit(self, kind, out, coords=None, t=0.0, lo=(0, 0, 0), hi=(0, 0, 0),
                     dims=(1, 1, 1), theta=0.0, rows=0, cols=0, S=0):
        """Admit a query writing into the CUDA tensor `out`; returns its id,
        or None when the in-flight budget is full (retry later)."""
        r = _abi.Request()
        r.kind = _abi.QUERY[kind]
        keep = [out]
        if kind == "points":
            ct = _cuda_f32(coords).view(-1, 4)
            keep.append(ct)
            r.coords_dev, r.n = ct.data_ptr(), ct.shape[0]
        r.t = float(t)
        r.lo = (C.c_double * 3)(*lo)
        r.hi = (C.c_double * 3)(*hi)
        r.dims = (C.c_int * 3)(*dims)
        r.theta, r.rows, r.cols, r.S = float(theta), rows, cols, S
        r.out_dev = out.data_ptr()
        rid = C.c_int64()
        st = _abi.lib().dinr_serve_submit(self._h, C.byref(r), C.byref(rid))
        if st == _abi.ERR_BUSY:
            return None
        self._c(st)
        self._serving = getattr(self, "_serving", {})
        self._serving[rid.value] = keep
        return rid.value

    def serve_step(self) -> int:
        n = C.c_int()
        self._c(_abi.lib().dinr_serve_step(self._h, C.byref(n)))
        return n.value

    def serve_poll(self, rid) -> bool:
        d = C.c_int()
        self._c(_abi.lib().dinr_serve_poll(self._h, int(rid), C.byref(d)))
        if d.value:
            self._serving.pop(rid, None)
        return bool(d.value)

    # -- state
    def params(self):
        out = torch.empty(self.n_params, device="cuda")
        self._c(_abi.lib().dinr_get_params(self._h, _ptr(out), 1))
        return out

    def set_params(self, p):
        t = _cuda_f32(p)
        self._c(_abi.lib().dinr_set_params(self._h, _ptr(t), 1))

    def grads(self):
        out = np.empty(self.n_params, np.float32)
        self._c(_abi.lib().dinr_get_grads(self._h, out.ctypes.data_as(C.c_void_p)))
        return out

    def loss(self):
        out = C.c_float()
        self._c(_abi.lib().dinr_get_loss(self._h, C.byref(out)))
        return out.value

    def get_state(self) -> bytes:
        n = C.c_size_t()
        self._c(_abi.lib().dinr_get_state(self._h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._c(_abi.lib().dinr_get_state(self._h, buf, C.byref(n)))
        return buf.raw

    def set_state(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        self._c(_abi.lib().dinr_set_state(self._h, buf, len(blob)))

    def profile(self, enable: bool):
        self._c(_abi.lib().dinr_profile(self._h, 1 if enable else 0))

    def profile_report(self) -> dict:
        """{kernel: dict(launches, ms, flops, bytes)} of the recorded launches."""
        buf = C.create_string_buffer(1 << 16)
        self._c(_abi.lib().dinr_profile_report(self._h, buf, len(buf)))
        out = {}
        for line in buf.value.decode().splitlines():
            name, n, ms, fl, by = line.split()
            out[name] = dict(launches=int(n), ms=float(ms), flops=float(fl), bytes=float(by))
        return out

    def synchronize(self):
        self._c(_abi.lib().dinr_synchronize(self._h))


def phantom_project(geometry, phantom, idx=None):
    """Exact FOV-clipped line integrals of an ellipsoid phantom (CUDA)."""
    gs, keep = geometry_struct(geometry)
    n_ell = len(phantom.rho)
    cen = np.ascontiguousarray(phantom.centre, np.float64)
    axe = np.ascontiguousarray(phantom.axes, np.float64)
    rho = np.ascontiguousarray(phantom.rho, np.float64)
    vel = np.ascontiguousarray(phantom.vel, np.float64)
    if idx is None:
        n = geometry.n_views * geometry.det_rows * geometry.det_cols
        it = None
    else:
        it = _cuda_i64(idx)
        n = it.numel()
    out = torch.empty(n, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    s = _abi.lib().dinr_phantom_project(
        C.byref(gs), n_ell, cen.ctypes.data_as(C.c_void_p), axe.ctypes.data_as(C.c_void_p),
        rho.ctypes.data_as(C.c_void_p), vel.ctypes.data_as(C.c_void_p), float(phantom.growth),
        _ptr(it), n, _ptr(out), C.c_void_p(st))
    _check(s, None)
    return out


class DinrStep(torch.autograd.Function):
    """Loss of a DINR minibatch as an autograd function of a parameter
    tensor: forward runs the library's forward model and loss only;
    backward launches its hand-written adjoint kernels for that minibatch
    (on the activations the forward kept, or recomputing them when the
    minibatch spans several workspace passes)."""

    @staticmethod
    def forward(ctx, params, model, idx):
        model.set_params(params.detach())
        ctx.model = model
        return model.forward_loss(idx)[0]

    @staticmethod
    def backward(ctx, g):
        return ctx.model.backward_grad(g), None, None
