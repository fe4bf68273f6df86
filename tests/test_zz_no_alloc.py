"""The allocation-free phantom projector, called through the C ABI.

dinr_phantom_project_noalloc serves callers that cannot allocate device
memory (an application whose device memory belongs to its own pool
allocator, a latency-bound loop that cannot pay for cudaMalloc/cudaFree): it
keeps its staging data in one static device array. Its output must match
dinr_phantom_project within the tolerance of the phantom test (1e-6) on two
calls in a row with different geometries and phantoms, since every call
reuses the same array. This file is collected last so that a run stopping at
its first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from synthetic import workloads as wl

from gpu_util import assert_close, require_gpu

pytestmark = pytest.mark.gpu


def _call(fn_name, geometry, phantom, idx):
    from paper_2404_19075_b300 import _abi
    from paper_2404_19075_b300.dinr import geometry_struct
    gs, keep = geometry_struct(geometry)
    arrays = [np.ascontiguousarray(a, np.float64)
              for a in (phantom.centre, phantom.axes, phantom.rho, phantom.vel)]
    it = torch.as_tensor(np.asarray(idx, np.int64), device="cuda")
    out = torch.full((it.numel(),), float("nan"), device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    status = getattr(_abi.lib(), fn_name)(
        C.byref(gs), len(phantom.rho), *[a.ctypes.data_as(C.c_void_p) for a in arrays],
        float(phantom.growth), C.c_void_p(it.data_ptr()), it.numel(), C.c_void_p(out.data_ptr()),
        C.c_void_p(st))
    assert status == 0, _abi.lib().dinr_last_error(None).decode()
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_allocating_projector_twice():
    """The larger geometry (512 views, 16 moving ellipsoids) first, then the
    smaller one (64 views, 3 ellipsoids), then the larger one again: every
    result must be bitwise the allocating projector's (both build the same
    FP64 view table on the host and run the same kernel), so that entries
    left in the shared array by an earlier call would show up."""
    require_gpu()
    w2, w1 = wl.workload(2), wl.workload(1)
    big = (w2, wl.ray_subset(w2.geom.n_proj, 50000, 3))
    small = (w1, np.arange(w1.geom.n_proj))
    got = []
    for w, idx in (big, small, big):               # calls in a row on one stream
        ph = wl.phantom(w)
        a = _call("dinr_phantom_project_noalloc", w.geom, ph, idx)
        b = _call("dinr_phantom_project", w.geom, ph, idx)
        assert np.isfinite(a).all()
        assert_close(a, b, 1e-6, f"workload {w.index}")
        assert np.array_equal(a, b), f"workload {w.index}: not bitwise the allocating projector"
        got.append(a)
    assert np.array_equal(got[0], got[2])


def test_noalloc_rejects_sizes_beyond_its_limit():
    require_gpu()
    from paper_2404_19075_b300 import _abi
    k = np.arange(5000, dtype=np.float64)
    g = wl.parallel_geometry(5000, 8, 8, k * 1e-3, k / 5000, 8)
    w = wl.workload(1)
    with pytest.raises(AssertionError, match="at most 4096 views"):
        _call("dinr_phantom_project_noalloc", g, wl.phantom(w), np.arange(10))
    # the same geometry checks as the allocating projector
    bad = wl.parallel_geometry(8, 8, 8, k[:8] * 1e-3, k[:8] / 8, 5000)
    for fn in ("dinr_phantom_project_noalloc", "dinr_phantom_project"):
        with pytest.raises(AssertionError, match="invalid phantom request"):
            _call(fn, bad, wl.phantom(w), np.arange(10))
