"""ctypes binding of libhjg.so (the C ABI in include/hjg.h): structures, status codes and
symbol signatures.  Argument marshalling only; every step of the sweep runs in the CUDA
library.  Loading fails loudly when the library has not been built."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhjg.so")

HJG_OK, HJG_EINVAL, HJG_ENOMEM, HJG_ECUDA, HJG_ENONFINITE, HJG_ETIMEOUT, \
    HJG_ENOTCONVERGED, HJG_EUNSUPPORTED = range(8)

GAMES = {"dubins3": 1, "rockets6": 2, "rockets45": 3, "flock4": 4, "rockets_rel3": 5,
         "double_int2": 6, "quadratic": 100, "zero_h": 101}
GAME_DIMS = {"dubins3": 3, "rockets6": 6, "rockets45": 45, "flock4": 4, "rockets_rel3": 3,
             "double_int2": 2}


class Dynamics(C.Structure):
    _fields_ = [("game", C.c_int32), ("n", C.c_int32), ("speed", C.c_double * 16),
                ("h_sign", C.c_double)]


class Target(C.Structure):
    _fields_ = [("radius", C.c_double), ("A", C.c_double * 64), ("x0", C.c_double * 8),
                ("d", C.c_double), ("obstacle_radius", C.c_double), ("obstacle_center", C.c_double * 2)]


class Options(C.Structure):
    _fields_ = [("N", C.c_int64), ("K", C.c_int32), ("tilt", C.c_int32), ("eps", C.c_double),
                ("eta", C.c_double), ("c_min", C.c_double), ("c_max", C.c_double),
                ("seed", C.c_uint64), ("instance", C.c_uint32), ("block_threads", C.c_int32),
                ("grid_blocks", C.c_int32), ("variant", C.c_int32), ("point_offset", C.c_uint32),
                ("tube", C.c_int32), ("cv", C.c_int32), ("precision", C.c_int32),
                ("reserved", C.c_int32 * 2)]


class Diag(C.Structure):
    _fields_ = [("M", C.c_int64), ("next_sweep", C.c_uint32), ("nonfinite", C.c_int64),
                ("clipped", C.c_int64), ("ess_min", C.c_double), ("ess_median", C.c_double),
                ("last_ms", C.c_double), ("block_threads", C.c_int32), ("grid_blocks", C.c_int32),
                ("variant", C.c_int32)]


# name -> (restype, argtypes)
_vp = C.c_void_p
_SIGS = {
    "hjg_create": (C.c_int, [C.POINTER(Dynamics), C.POINTER(Target), C.c_double, C.c_double,
                             C.POINTER(Options), C.POINTER(_vp)]),
    "hjg_set_points": (C.c_int, [_vp, _vp, C.c_int64, C.c_int64, C.c_int, _vp]),
    "hjg_picard_sweep": (C.c_int, [_vp, C.c_int, _vp, _vp]),
    "hjg_get_state": (C.c_int, [_vp, _vp, _vp, C.c_int64, _vp, _vp, C.c_int]),
    "hjg_set_state": (C.c_int, [_vp, _vp, _vp, C.c_int64, _vp, C.c_uint32, C.c_int]),
    "hjg_get_history": (C.c_int, [_vp, _vp, C.c_int]),
    "hjg_value_grad": (C.c_int, [_vp, _vp, C.c_int64, C.c_int64, C.c_int, _vp, _vp, C.c_int64,
                                 _vp, _vp]),
    "hjg_get_diagnostics": (C.c_int, [_vp, C.POINTER(Diag)]),
    "hjg_autotune": (C.c_int, [_vp, C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                               C.POINTER(C.c_double)]),
    "hjg_set_stream": (C.c_int, [_vp, _vp]),
    "hjg_destroy": (None, [_vp]),
    "hjg_last_error": (C.c_char_p, [_vp]),
    "hjg_status_string": (C.c_char_p, [C.c_int]),
    "hjg_value_grad_noalloc": (C.c_int, [C.POINTER(Dynamics), C.POINTER(Target), C.c_double,
                                         C.c_double, C.POINTER(Options), _vp, C.c_int64,
                                         C.c_int64, _vp, _vp, C.c_int64, _vp, _vp]),
    "hjg_flock_neighbours": (C.c_int, [_vp, C.c_int64, C.c_int64, C.c_int, _vp, _vp, _vp]),
    "hjg_warm_start": (C.c_int, [_vp, _vp, _vp, C.c_int64, C.c_int]),
    "hjg_warm_start_delta": (C.c_int, [_vp, _vp, C.c_int64]),
    "hjg_get_state_delta": (C.c_int, [_vp, _vp, C.c_int64]),
    "hjg_frame_features": (C.c_int, [_vp, _vp, C.c_int64]),
    "hjg_frame_targets": (C.c_int, [_vp, _vp, C.c_int64]),
    "hjg_warm_start_frame": (C.c_int, [_vp, _vp, C.c_int64, C.c_int]),
    "hjg_get_residual_parts": (C.c_int, [_vp, _vp]),
    "hjg_set_horizons": (C.c_int, [_vp, _vp, C.c_int]),
    "hjg_selftest_bounded_wait": (C.c_int, [C.c_int, C.c_int64, _vp]),
    "hjg_topology": (C.c_int, [_vp, C.c_int, C.c_int, C.c_double, _vp, _vp, _vp, _vp, _vp]),
    "hjg_certify": (C.c_int, [_vp, C.c_double, C.c_double, C.c_double, C.c_double, _vp, _vp, _vp, _vp,
                              C.c_int]),
    "hjg_mlp_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_uint64, C.POINTER(_vp)]),
    "hjg_mlp_destroy": (None, [_vp]),
    "hjg_mlp_set_stream": (C.c_int, [_vp, _vp]),
    "hjg_mlp_num_params": (C.c_int64, [_vp]),
    "hjg_mlp_get_params": (C.c_int, [_vp, _vp, C.c_int]),
    "hjg_mlp_set_params": (C.c_int, [_vp, _vp, C.c_int]),
    "hjg_mlp_forward": (C.c_int, [_vp, _vp, C.c_int64, C.c_int64, _vp, C.c_int64]),
    "hjg_mlp_gradients": (C.c_int, [_vp, _vp, C.c_int64, _vp, C.c_int64, C.c_int64,
                                    C.POINTER(C.c_double), _vp]),
    "hjg_gemm_bf16": (C.c_int, [_vp, C.c_int64, C.c_int64, _vp, C.c_int64, C.c_int64, C.c_int,
                                C.c_int, C.c_int, _vp, C.c_int64, C.POINTER(C.c_int), _vp]),
    "hjg_mlp_input_grad": (C.c_int, [_vp, _vp, C.c_int64, C.c_int64, C.c_int, _vp, C.c_int64]),
    "hjg_mlp_fit_scaling": (C.c_int, [_vp, _vp, C.c_int64, _vp, C.c_int64, C.c_int64]),
    "hjg_mlp_get_scaling": (C.c_int, [_vp, _vp]),
    "hjg_mlp_set_scaling": (C.c_int, [_vp, _vp]),
    "hjg_mlp_fit": (C.c_int, [_vp, _vp, C.c_int64, _vp, C.c_int64, C.c_int64, C.c_int, C.c_int64,
                              C.c_float, C.c_float, C.c_int, _vp]),
    "hjg_mlp_train_step": (C.c_int, [_vp, _vp, C.c_int64, _vp, C.c_int64, C.c_int64, C.c_float,
                                     C.POINTER(C.c_double)]),
    "hjg_batch_create": (C.c_int, [C.POINTER(_vp)]),
    "hjg_batch_add": (C.c_int, [_vp, _vp]),
    "hjg_batch_run": (C.c_int, [_vp, C.c_int, _vp, _vp, C.POINTER(C.c_double)]),
    "hjg_batch_destroy": (None, [_vp]),
    "hjg_batch_last_error": (C.c_char_p, [_vp]),
    "hjg_philox_blocks": (C.c_int, [_vp, _vp, _vp, C.c_int64, _vp]),
    "hjg_sample_normals": (C.c_int, [C.c_int, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                     C.c_int64, _vp, _vp]),
    "hjg_microbench": (C.c_int, [C.c_int, C.c_int64, C.POINTER(C.c_double),
                                 C.POINTER(C.c_double)]),
}

MICROBENCH = {"ffma": 1, "ex2": 2, "lg2": 3, "sin": 4, "cos": 5, "sqrt": 6, "philox": 7,
              "normals": 8, "imad_wide": 9, "imul_lo": 10, "imul_hi": 11, "philox_split": 12,
              "philox_mixed": 13}

_lib = None


def load(path: str = LIB_PATH):
    """Load libhjg.so and bind every exported symbol; raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libhjg.so not found at %s: build it first "
                           "(python -c 'import __graft_entry__ as g; g.build()')" % path)
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def symbols():
    return list(_SIGS)


class HJGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s (status %d): %s" % (status_string(status), status, msg))
        self.status = status


def status_string(st: int) -> str:
    return load().hjg_status_string(st).decode()
