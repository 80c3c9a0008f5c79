"""ctypes binding of include/octaoctree.h (argument marshalling only).

Loads the in-tree shared library built by paper_2606_08469_gb300.build and
declares every exported entry point with the header's names and signatures.
There is no fallback: a missing library raises immediately.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

OCTA_OK = 0
OCTA_EINVAL = -1
OCTA_ERANGE = -2
OCTA_ECUDA = -3
OCTA_ETIMEOUT = -4
OCTA_EUNSUPPORTED = -6

OCTA_STATUS_BAD_CHILD = 1
OCTA_STATUS_BAD_MAP = 2
OCTA_STATUS_TIMEOUT = 4

OCTA_MAX_LEVELS = 16
OCTA_MAX_LAYERS = 6
OCTA_MAX_SCENES = 16
OCTA_MAX_GROUPS = 16

OCTA_F32 = 0
OCTA_F16 = 1
OCTA_BF16 = 2
OCTA_FORM_CELL_BILINEAR = 0
OCTA_FORM_TRILINEAR_VERTEX = 1
OCTA_FORM_SHIFTED = 2

OCTA_OP_LOSS = 1
OCTA_OP_ADAM = 2
OCTA_OP_STEP = 3


class octa_tree_desc(C.Structure):
    _fields_ = [
        ("num_levels", C.c_int32),
        ("num_nodes", C.c_int32),
        ("num_texels", C.c_int64),
        ("R", C.c_int32 * OCTA_MAX_LEVELS),
        ("level_node_start", C.c_int32 * (OCTA_MAX_LEVELS + 1)),
        ("level_texel_base", C.c_int64 * (OCTA_MAX_LEVELS + 1)),
    ]


class octa_scene(C.Structure):
    _fields_ = [
        ("first_child", C.c_void_p),
        ("map_offset", C.c_void_p),
        ("tables", C.c_void_p),
        ("weights", C.c_void_p),
        ("num_levels", C.c_int32),
        ("num_nodes", C.c_int32),
        ("num_texels", C.c_int64),
        ("R", C.c_int32 * OCTA_MAX_LEVELS),
        ("F", C.c_int32),
        ("table_dtype", C.c_int32),
        ("weight_dtype", C.c_int32),
        ("n_layers", C.c_int32),
        ("widths", C.c_int32 * (OCTA_MAX_LAYERS + 1)),
        ("query_form", C.c_int32),
    ]


class octa_queries(C.Structure):
    _fields_ = [
        ("x", C.c_void_p),
        ("omega", C.c_void_p),
        ("n", C.c_int64),
        ("scene_start", C.c_int64 * (OCTA_MAX_SCENES + 1)),
        ("normal", C.c_void_p),
        ("disparity", C.c_void_p),
        ("attrs", C.c_void_p),
        ("n_attrs", C.c_int32),
        ("reserved_q", C.c_int32),
        ("d_disparity", C.c_void_p),
    ]


class octa_scene_grads(C.Structure):
    _fields_ = [("d_tables", C.c_void_p), ("d_weights", C.c_void_p)]


class octa_pairs(C.Structure):
    _fields_ = [
        ("x", C.c_void_p),
        ("omega", C.c_void_p),
        ("x2", C.c_void_p),
        ("omega2", C.c_void_p),
        ("E", C.c_void_p),
        ("w", C.c_void_p),
        ("n", C.c_int64),
        ("scene_start", C.c_int64 * (OCTA_MAX_SCENES + 1)),
        ("norm_pairs", C.c_int64 * OCTA_MAX_SCENES),
        ("normal", C.c_void_p),
        ("normal2", C.c_void_p),
        ("disparity", C.c_void_p),
        ("disparity2", C.c_void_p),
        ("d_disparity", C.c_void_p),
        ("d_disparity2", C.c_void_p),
    ]


class octa_scaler(C.Structure):
    _fields_ = [
        ("scale", C.c_float),
        ("inv_scale_used", C.c_float),
        ("good_steps", C.c_int32),
        ("growth_interval", C.c_int32),
        ("step", C.c_int32),
        ("skipped", C.c_int32),
        ("n_skipped", C.c_int32),
        ("reserved", C.c_int32),
        ("grad_norm", C.c_double),
        ("loss", C.c_double),
    ]


class octa_param_group(C.Structure):
    _fields_ = [
        ("param", C.c_void_p),
        ("grad", C.c_void_p),
        ("m", C.c_void_p),
        ("v", C.c_void_p),
        ("work", C.c_void_p),
        ("work_dtype", C.c_int32),
        ("lr", C.c_float),
        ("n", C.c_int64),
    ]


class octa_adam_cfg(C.Structure):
    _fields_ = [("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float)]


class octa_tuning(C.Structure):
    _fields_ = [("fwd_ctas_per_sm", C.c_int32), ("encode_ctas_per_sm", C.c_int32),
                ("engine_ctas_per_sm", C.c_int32), ("fwd_order", C.c_int32),
                ("train_order", C.c_int32), ("fwd_threads_per_query", C.c_int32),
                ("encode_threads_per_query", C.c_int32), ("train_threads_per_row", C.c_int32),
                ("fwd_run", C.c_int32), ("train_run", C.c_int32), ("gather_stages", C.c_int32),
                ("l1_carveout", C.c_int32)]


class octa_step_options(C.Structure):
    _fields_ = [("barrier_timeout_ns", C.c_uint64), ("extra_barrier_arrivals", C.c_int32),
                ("skip_first_mma", C.c_int32)]


OCTA_MAX_PRIMS = 64
OCTA_MAX_ATTRS = 16
OCTA_PRED_HIDDEN = 64
OCTA_PRED_MAX_LEVELS = 16


class octa_predictor(C.Structure):
    _fields_ = [("table", C.c_void_p), ("weights", C.c_void_p), ("weights_bf16", C.c_void_p),
                ("levels", C.c_int32), ("log2_T", C.c_int32),
                ("res", C.c_int32 * OCTA_PRED_MAX_LEVELS)]


class octa_prims(C.Structure):
    _fields_ = [("planes", C.c_void_p), ("spheres", C.c_void_p), ("n_planes", C.c_int32),
                ("n_spheres", C.c_int32)]


# Every symbol the header declares, with its ctypes signature.
_P = C.c_void_p
_SIGNATURES = {
    "octree_build": (C.c_int, [C.c_uint64, C.c_int32, C.c_double, _P, C.POINTER(octa_tree_desc),
                               _P, _P, _P]),
    "octree_from_flags": (C.c_int, [_P, C.c_int64, C.c_int32, _P, C.POINTER(octa_tree_desc),
                                    _P, _P, _P]),
    "octa_encode": (C.c_int, [C.POINTER(octa_scene), C.c_int32, C.POINTER(octa_queries), _P,
                              C.c_int32, C.c_int64, _P, _P, _P, _P]),
    "octa_query_fwd": (C.c_int, [C.POINTER(octa_scene), C.c_int32, C.POINTER(octa_queries), _P,
                                 _P, _P, _P, _P]),
    "octa_query_bwd": (C.c_int, [C.POINTER(octa_scene), C.c_int32, C.POINTER(octa_queries), _P,
                                 C.POINTER(octa_scene_grads), _P, _P]),
    "octa_train_fused": (C.c_int, [C.POINTER(octa_scene), C.c_int32, C.POINTER(octa_pairs), C.c_float,
                                   C.c_int32, _P, _P, C.POINTER(octa_scene_grads), _P, _P]),
    "octa_train_step_batched": (C.c_int, [C.POINTER(octa_scene), C.c_int32, C.POINTER(octa_pairs),
                                          C.POINTER(octa_scene_grads), C.POINTER(octa_param_group),
                                          C.c_int32, C.c_float, C.c_int32, C.POINTER(octa_adam_cfg),
                                          _P, _P, C.POINTER(octa_step_options), _P, C.c_size_t, _P,
                                          _P]),
    "residual_loss": (C.c_int, [_P, _P, _P, _P, C.c_int64, C.c_float, C.c_int32, _P, _P, _P, _P,
                                _P, C.c_size_t, _P]),
    "residual_loss_static": (C.c_int, [_P, _P, _P, _P, C.c_int64, C.c_float, C.c_int32, _P, _P,
                                       _P, _P, _P]),
    "residual_loss_multi": (C.c_int, [_P, _P, _P, _P, C.c_int64, C.c_int32, C.c_float, C.c_int32,
                                      _P, _P, _P, _P, _P, C.c_size_t, _P]),
    "octa_trace_rays": (C.c_int, [C.POINTER(octa_prims), _P, C.c_int32, _P, C.c_int64, C.c_float,
                                  _P, _P, _P, _P, _P]),
    "octa_disparity": (C.c_int, [C.POINTER(octa_predictor), C.POINTER(octa_queries), _P, _P]),
    "octa_disparity_bwd": (C.c_int, [C.POINTER(octa_predictor), C.POINTER(octa_queries), _P, _P,
                                     _P, _P]),
    "adam_step": (C.c_int, [C.POINTER(octa_param_group), C.c_int32, C.POINTER(octa_adam_cfg), _P,
                            _P, C.c_size_t, _P]),
    "octa_workspace_bytes": (C.c_size_t, [C.c_int32, C.c_int64]),
    "octa_set_tuning": (C.c_int, [C.POINTER(octa_tuning)]),
    "octa_get_tuning": (C.c_int, [C.POINTER(octa_tuning)]),
    "octa_last_error": (C.c_char_p, []),
    "octa_abi_version": (C.c_int32, []),
    "octa_measure_ffma": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _P]),
    "octa_measure_mma": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _P]),
}

_lib = None


def library_path():
    return _build.LIB


def load(path=None):
    """Load (once) and return the ctypes handle of the CUDA library."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise ImportError(
            f"OctaOctree CUDA library not built ({path}); run paper_2606_08469_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class OctaError(RuntimeError):
    def __init__(self, code, where):
        msg = load().octa_last_error().decode(errors="replace")
        super().__init__(f"{where} failed with status {code}: {msg}")
        self.code = code


def check(code, where):
    if code != OCTA_OK:
        raise OctaError(code, where)
    return code
