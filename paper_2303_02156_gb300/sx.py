"""ctypes binding of libsx (include/sx.h).

Argument marshalling only: every function below forwards to the C entry
point of the same name, and every step of the numerical path runs in the
library's CUDA kernels. Device memory comes from torch tensors
(``tensor.data_ptr()``). Importing works without a GPU; any call that
needs the library raises ``RuntimeError`` when ``libsx.so`` is missing,
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsx.so")

SX_OK, SX_EINVAL, SX_ENOMEM, SX_ECUDA, SX_ENAN = 0, -1, -2, -3, -4
SX_ENOTCONV, SX_ESTATE, SX_EDEGENERATE, SX_EBUDGET, SX_ELINESEARCH, SX_EORDER = (
    -5, -6, -7, -8, -9, -10)
SX_E, SX_EG, SX_EGH = 0, 1, 2
SX_FP64, SX_FP32 = 0, 1
SX_KIND_SNH_TET4, SX_KIND_HINGE4, SX_KIND_PT_BARRIER = 0, 1, 2
SX_SERVER_MAX_LANES = 8
SX_PROJECT_NONE, SX_PROJECT_ELEMENT, SX_PROJECT_MATERIAL = 0, 1, 2
SX_KIND_TET4 = SX_KIND_SNH_TET4
SX_KIND_PT_FRICTION = 3
SX_KIND_TET_HO = 4
SX_HO_MAX_QP = 64
SX_MODEL_SNH, SX_MODEL_NH, SX_MODEL_STVK, SX_MODEL_COROT, SX_MODEL_ARAP = 0, 1, 2, 3, 4

STATUS_NAMES = {0: "SX_OK", -1: "SX_EINVAL", -2: "SX_ENOMEM", -3: "SX_ECUDA", -4: "SX_ENAN",
                -5: "SX_ENOTCONV", -6: "SX_ESTATE", -7: "SX_EDEGENERATE", -8: "SX_EBUDGET",
                -9: "SX_ELINESEARCH", -10: "SX_EORDER"}

# every symbol include/sx.h declares
EXPORTS = [
    "sx_create", "sx_destroy", "sx_last_error", "sx_inject_alloc_failure", "sx_version",
    "sx_scene_create",
    "sx_scene_destroy", "sx_add_snh_tet4", "sx_add_hinge4", "sx_add_pt_barrier",
    "sx_add_node_mass", "sx_set_pinned", "sx_set_gravity", "sx_finalize", "sx_set_state",
    "sx_get_state", "sx_set_inertia", "sx_eval", "sx_eval_batch", "sx_get_bsr",
    "sx_get_grad", "sx_get_diag_slots", "sx_eval_elements", "sx_newton_opts_default",
    "sx_newton_step", "sx_newton_step_batch", "sx_scene_footprint", "sx_scene_bytes",
    "sx_copy_bsr", "sx_copy_grad", "sx_scene_info", "sx_block_info", "sx_eval_stats",
    "sx_profile", "sx_profile_read", "sx_projection_bins", "sx_eval_elements_noalloc",
    "sx_autotune", "sx_set_launch_shape", "sx_get_launch_shape", "sx_set_pairs",
    "sx_compact_pairs", "sx_add_tet4", "sx_update_rotations", "sx_get_rotations",
    "sx_set_rotations", "sx_add_pt_friction", "sx_update_friction", "sx_get_friction_lag",
    "sx_add_tet_ho", "sx_advance",
    "sx_server_create", "sx_server_set_lanes", "sx_server_set_lane_cap", "sx_server_submit",
    "sx_server_poll", "sx_server_result",
    "sx_server_drain", "sx_server_stats", "sx_server_destroy",
]
SX_NOALLOC_MAX_ELEMENTS = 65536
PHASES = ["elements", "clamp", "assemble", "grad", "reduce", "spmv", "pcg", "newton", "other"]


class sx_options(C.Structure):
    _fields_ = [("device", C.c_int), ("share_sms", C.c_int), ("reserved", C.c_int * 6)]


class sx_newton_opts(C.Structure):
    _fields_ = [("newton_tol", C.c_double), ("pcg_tol", C.c_double),
                ("max_newton", C.c_int), ("max_pcg", C.c_int), ("max_halvings", C.c_int),
                ("project", C.c_int), ("precision", C.c_int), ("armijo_c", C.c_double),
                ("forcing", C.c_int), ("graphs", C.c_int)]


class sx_step_report(C.Structure):
    _fields_ = [("status", C.c_int), ("newton_iters", C.c_int), ("pcg_iters", C.c_int),
                ("ls_halvings", C.c_int), ("g0_norm", C.c_double), ("g_norm", C.c_double),
                ("energy", C.c_double), ("ms", C.c_double)]


class sx_scene_desc(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_tets", C.c_int64), ("n_hinges", C.c_int64),
                ("n_pairs", C.c_int64), ("nnzb_hint", C.c_int64)]


class sx_snh_scene_spec(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("X", C.c_void_p), ("n_tets", C.c_int64),
                ("tets", C.c_void_p), ("young", C.c_void_p), ("poisson", C.c_void_p),
                ("density", C.c_double), ("n_pinned", C.c_int64), ("pinned", C.c_void_p),
                ("gravity", C.c_double * 3)]


class sx_completion(C.Structure):
    _fields_ = [("req_id", C.c_int64), ("status", C.c_int), ("steps", C.c_int),
                ("n_tets", C.c_int64), ("submit_ms", C.c_double), ("admit_ms", C.c_double),
                ("done_ms", C.c_double), ("mean_step_ms", C.c_double),
                ("error", C.c_char * 120)]


class sx_tune_report(C.Structure):
    _fields_ = [("clamp_threads", C.c_int), ("elem_blocks_per_sm", C.c_int),
                ("default_ms", C.c_double), ("tuned_ms", C.c_double), ("candidates", C.c_int)]


class sx_serve_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
                ("rejected", C.c_int64), ("element_steps", C.c_int64), ("wall_ms", C.c_double),
                ("busy_ms", C.c_double), ("step_p50_ms", C.c_double), ("step_p99_ms", C.c_double),
                ("request_p50_ms", C.c_double), ("request_p99_ms", C.c_double),
                ("bytes_in_use", C.c_int64), ("peak_bytes", C.c_int64), ("active", C.c_int),
                ("pending", C.c_int), ("ticks", C.c_int)]


_P = C.c_void_p
_I64 = C.c_int64
_D = C.c_double
_I = C.c_int
_PP = C.POINTER(C.c_void_p)

_SIGS = {
    "sx_create": (_I, [_PP, _P]),
    "sx_destroy": (_I, [_P]),
    "sx_last_error": (C.c_char_p, [_P]),
    "sx_inject_alloc_failure": (C.c_int, [_P, C.c_int]),
    "sx_version": (C.c_char_p, []),
    "sx_scene_create": (_I, [_P, _I64, _P, _I64, _P, _PP]),
    "sx_scene_destroy": (_I, [_P]),
    "sx_add_snh_tet4": (_I, [_P, _P, _I64, _P, _P, _D, _I, _P, C.POINTER(_I)]),
    "sx_add_hinge4": (_I, [_P, _P, _I64, _P, _P, _D, _P, C.POINTER(_I)]),
    "sx_add_pt_barrier": (_I, [_P, _P, _I64, _D, _D, _P, C.POINTER(_I)]),
    "sx_add_node_mass": (_I, [_P, _P, _P]),
    "sx_set_pinned": (_I, [_P, _P, _I64, _P]),
    "sx_set_gravity": (_I, [_P, C.POINTER(_D)]),
    "sx_finalize": (_I, [_P, _P]),
    "sx_set_state": (_I, [_P, _P, _P, _P]),
    "sx_get_state": (_I, [_P, _P, _P, _P]),
    "sx_set_inertia": (_I, [_P, _D, _P, _P]),
    "sx_eval": (_I, [_P, _I, _I, _I, C.POINTER(_D), _P]),
    "sx_eval_batch": (_I, [_P, C.POINTER(_P), _I, _I, _I, _I, C.POINTER(_D), _P]),
    "sx_get_bsr": (_I, [_P, _PP, _PP, _PP, C.POINTER(_I64), C.POINTER(_I)]),
    "sx_get_grad": (_I, [_P, _PP]),
    "sx_get_diag_slots": (_I, [_P, _PP]),
    "sx_eval_elements": (_I, [_P, _I, _I, _I, _P, _P, _P, _P, _P]),
    "sx_newton_opts_default": (None, [C.POINTER(sx_newton_opts)]),
    "sx_newton_step": (_I, [_P, _D, C.POINTER(sx_newton_opts), C.POINTER(sx_step_report), _P]),
    "sx_newton_step_batch": (_I, [_P, C.POINTER(_P), _I, _D, C.POINTER(sx_newton_opts),
                                  C.POINTER(sx_step_report), _P]),
    "sx_scene_footprint": (_I, [C.POINTER(sx_scene_desc), C.POINTER(_I64)]),
    "sx_scene_bytes": (_I, [_P, C.POINTER(_I64)]),
    "sx_copy_bsr": (_I, [_P, _P, _P, _P, C.POINTER(_I), _P]),
    "sx_copy_grad": (_I, [_P, _P, _P]),
    "sx_scene_info": (_I, [_P, C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_I)]),
    "sx_block_info": (_I, [_P, _I, C.POINTER(_I), C.POINTER(_I64)]),
    "sx_eval_stats": (_I, [_P, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I), _P]),
    "sx_profile": (_I, [_P, _I]),
    "sx_profile_read": (_I, [_P, C.POINTER(_D), C.POINTER(_I64), _I]),
    "sx_projection_bins": (_I, [_P, C.POINTER(_I), _P]),
    "sx_eval_elements_noalloc": (_I, [_P, _I, _I, _I, _P, _P, _P, _P]),
    "sx_server_create": (_I, [_P, _I64, C.POINTER(sx_newton_opts), _PP]),
    "sx_autotune": (_I, [_P, C.POINTER(_P), _I, _I, C.POINTER(sx_tune_report), _P]),
    "sx_set_pairs": (_I, [_P, _I, _P, _I64, _P]),
    "sx_add_tet4": (_I, [_P, _I, _P, _I64, _P, _P, _D, _P, C.POINTER(_I)]),
    "sx_update_rotations": (_I, [_P, _P]),
    "sx_get_rotations": (_I, [_P, _I, _P, _P]),
    "sx_set_rotations": (_I, [_P, _I, _P, _P]),
    "sx_add_pt_friction": (_I, [_P, _P, _I64, _D, _D, _D, _D, _P, C.POINTER(_I)]),
    "sx_add_tet_ho": (_I, [_P, _I, _P, _I64, _P, _P, _D, _P, _I, _P, C.POINTER(_I)]),
    "sx_advance": (_I, [_P, _D, _P, _I, _P, C.POINTER(_I), _P]),
    "sx_update_friction": (_I, [_P, _D, _P]),
    "sx_get_friction_lag": (_I, [_P, _I, _P, _P, _P, _P, _P]),
    "sx_compact_pairs": (_I, [_P, _I, C.POINTER(_I64), _P]),
    "sx_set_launch_shape": (_I, [_P, _I, _I, _I]),
    "sx_get_launch_shape": (_I, [_P, _I, C.POINTER(_I), C.POINTER(_I)]),
    "sx_server_set_lanes": (_I, [_P, _I, C.POINTER(_I64)]),
    "sx_server_set_lane_cap": (C.c_int, [_P, C.c_int]),
    "sx_server_submit": (_I, [_P, C.POINTER(sx_snh_scene_spec), _I, _D, C.POINTER(_I64)]),
    "sx_server_poll": (_I, [_P, C.POINTER(sx_completion), _I, C.POINTER(_I)]),
    "sx_server_result": (_I, [_P, _I64, _P, _P]),
    "sx_server_drain": (_I, [_P, _D]),
    "sx_server_stats": (_I, [_P, C.POINTER(sx_serve_stats)]),
    "sx_server_destroy": (_I, [_P]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libsx.so and declare every signature. Raises RuntimeError if
    the library was not built (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            "libsx.so not found at %s: build it with __graft_entry__.build() "
            "(or python -m paper_2303_02156_gb300.build); there is no CPU fallback" % path)
    L = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


class SxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(code, code), msg))
        self.code = code


def check(ctx, rc):
    if rc != SX_OK:
        msg = load().sx_last_error(ctx).decode() if ctx else ""
        raise SxError(rc, msg)
    return rc


def _def(name):
    def f(*args):
        return getattr(load(), name)(*args)
    f.__name__ = name
    f.__doc__ = "Forwards to the C entry point %s (include/sx.h)." % name
    return f


for _n in _SIGS:
    globals()[_n] = _def(_n)


# ---------------------------------------------------------------- helpers
def ptr(t):
    """Device (or host) address of a torch tensor / numpy array, or None."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data


def newton_opts(**kw):
    o = sx_newton_opts()
    load().sx_newton_opts_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o
