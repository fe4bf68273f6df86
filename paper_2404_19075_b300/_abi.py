"""ctypes declarations of the libdinr C ABI (include/dinr.h).

Argument marshalling only: every step of the method runs in the CUDA
library. Loading fails loudly when the in-tree libdinr.so is missing; there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdinr.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "dinr.h")

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_NONFINITE, ERR_UNSUPPORTED, ERR_BUSY, \
    ERR_STATE = range(9)
STATUS_NAMES = ["OK", "ERR_ARG", "ERR_OOM", "ERR_CUDA", "ERR_TIMEOUT", "ERR_NONFINITE",
                "ERR_UNSUPPORTED", "ERR_BUSY", "ERR_STATE"]
BEAM = {"parallel": 0, "cone": 1}
ACT = {"relu": 0, "swish": 1}
OUT_ACT = {"identity": 0, "softplus": 1}
PREC = {"fp32": 0, "bf16": 1, "fp8": 2}
ENCODING = {"octave": 0, "grff": 1}


class Geometry(C.Structure):
    _fields_ = [("beam", C.c_int), ("n_views", C.c_int), ("det_rows", C.c_int),
                ("det_cols", C.c_int), ("view_angle", C.POINTER(C.c_double)),
                ("view_time", C.POINTER(C.c_double)), ("det_pitch_u", C.c_double),
                ("det_pitch_v", C.c_double), ("det_off_u", C.c_double),
                ("det_off_v", C.c_double), ("sod", C.c_double), ("sdd", C.c_double),
                ("fov_r", C.c_double), ("fov_z0", C.c_double), ("fov_z1", C.c_double),
                ("t0", C.c_double), ("t1", C.c_double), ("samples_per_ray", C.c_int),
                ("mu0", C.c_double), ("subpixels", C.c_int)]


class Net(C.Structure):
    _fields_ = [("n_freq", C.c_int), ("hidden_layers", C.c_int), ("width", C.c_int),
                ("act", C.c_int), ("out_act", C.c_int), ("prec", C.c_int),
                ("init_params", C.POINTER(C.c_float)), ("seed", C.c_uint64),
                ("encoding", C.c_int), ("grff_c", C.c_int), ("grff_B", C.POINTER(C.c_float))]


class Train(C.Structure):
    _fields_ = [("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double),
                ("eps", C.c_double), ("lr_decay_per_epoch", C.c_double),
                ("batch_rays", C.c_int), ("chunk_rays", C.c_int),
                ("sampler_seed", C.c_uint64), ("recompute", C.c_int)]


class Request(C.Structure):
    _fields_ = [("kind", C.c_int), ("coords_dev", C.c_void_p), ("n", C.c_int64),
                ("t", C.c_double), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("dims", C.c_int * 3), ("theta", C.c_double), ("rows", C.c_int),
                ("cols", C.c_int), ("S", C.c_int), ("out_dev", C.c_void_p)]


QUERY = {"points": 0, "grid": 1, "project": 2}
SERVE_POLICY = {"arrival": 0, "least_work": 1}

# dinr_volume_sink(user, k, t, volume, n) -> int
VOLUME_SINK = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_float),
                          C.c_int64)

vp, i64 = C.c_void_p, C.c_int64
PROTOTYPES = {
    "dinr_param_count": (C.c_int64, [C.c_int, C.c_int, C.c_int]),
    "dinr_param_count_din": (C.c_int64, [C.c_int, C.c_int, C.c_int]),
    "dinr_create": (C.c_int, [C.POINTER(Geometry), C.POINTER(Net), C.POINTER(Train), vp,
                              C.c_int, vp, C.POINTER(vp)]),
    "dinr_set_projections": (C.c_int, [vp, vp, C.c_int]),
    "dinr_train_step": (C.c_int, [vp, vp, C.c_int, C.c_int, C.POINTER(C.c_float)]),
    "dinr_loss_grad": (C.c_int, [vp, vp, C.c_int, C.c_int, vp, vp]),
    "dinr_forward": (C.c_int, [vp, vp, C.c_int, C.c_int, vp]),
    "dinr_train_graph": (C.c_int, [vp, C.c_int, C.c_int, vp]),
    "dinr_backward": (C.c_int, [vp, vp, vp]),
    "dinr_predict": (C.c_int, [vp, vp, C.c_int, C.c_int, vp]),
    "dinr_project": (C.c_int, [vp, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int, vp]),
    "dinr_query": (C.c_int, [vp, vp, i64, vp]),
    "dinr_query_grid": (C.c_int, [vp, C.c_double, C.POINTER(C.c_double),
                                  C.POINTER(C.c_double), C.POINTER(C.c_int), vp]),
    "dinr_selftest_timeout": (C.c_int, [vp, i64]),
    "dinr_export": (C.c_int, [vp, C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_double),
                              C.POINTER(C.c_double), C.POINTER(C.c_int), VOLUME_SINK, vp]),
    "dinr_set_params": (C.c_int, [vp, vp, C.c_int]),
    "dinr_get_params": (C.c_int, [vp, vp, C.c_int]),
    "dinr_get_grads": (C.c_int, [vp, vp]),
    "dinr_get_loss": (C.c_int, [vp, C.POINTER(C.c_float)]),
    "dinr_get_state": (C.c_int, [vp, vp, C.POINTER(C.c_size_t)]),
    "dinr_set_state": (C.c_int, [vp, vp, C.c_size_t]),
    "dinr_sample_indices": (C.c_int, [vp, i64, C.c_int, vp]),
    "dinr_phantom_project": (C.c_int, [C.POINTER(Geometry), C.c_int, vp, vp, vp, vp,
                                       C.c_double, vp, i64, vp, vp]),
    "dinr_phantom_project_noalloc": (C.c_int, [C.POINTER(Geometry), C.c_int, vp, vp, vp, vp,
                                               C.c_double, vp, i64, vp, vp]),
    "dinr_serve_config": (C.c_int, [vp, i64, i64]),
    "dinr_serve_policy": (C.c_int, [vp, C.c_int]),
    "dinr_serve_submit": (C.c_int, [vp, C.POINTER(Request), C.POINTER(C.c_int64)]),
    "dinr_serve_step": (C.c_int, [vp, C.POINTER(C.c_int)]),
    "dinr_serve_poll": (C.c_int, [vp, i64, C.POINTER(C.c_int)]),
    "dinr_profile": (C.c_int, [vp, C.c_int]),
    "dinr_profile_report": (C.c_int, [vp, C.c_char_p, C.c_size_t]),
    "dinr_synchronize": (C.c_int, [vp]),
    "dinr_last_error": (C.c_char_p, [vp]),
    "dinr_destroy": (None, [vp]),
}

_lib = None


def lib():
    """The loaded libdinr.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2404_19075_b300.build` (nvcc, sm_103a)")
    L = C.CDLL(LIB_PATH)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def declared_symbols(header: str = HEADER) -> list:
    """Entry points declared in include/dinr.h."""
    with open(header) as f:
        text = f.read()
    return sorted(set(re.findall(r"^DINR_API\s+[\w\s\*]*?\b(dinr_[a-z_0-9]+)\s*\(", text, re.M)))
