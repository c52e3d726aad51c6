"""ctypes declarations of the C ABI in include/dg_atmo.h (argument marshalling only).

The shared library is built in-tree (``build.py``); importing this module on
a machine without it raises, so no caller can silently fall back to another
implementation.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libdgatmo.so")

DG_OK = 0
DG_STATUS = {
    0: "DG_OK", -1: "DG_EINVAL", -2: "DG_ENOMEM", -3: "DG_ECUDA", -4: "DG_ENOTCONV",
    -5: "DG_ENONFINITE", -6: "DG_EUNBALANCED", -7: "DG_EBUDGET", -8: "DG_ETIMEOUT",
}
DG_FP64, DG_FP32 = 0, 1
DG_KRYLOV_AUTO, DG_KRYLOV_GMRES, DG_KRYLOV_CG, DG_KRYLOV_GMRES_CGS2, DG_KRYLOV_CHEBYSHEV = -1, 0, 1, 2, 3
DG_TERMS_FULL, DG_TERMS_IMEX_EXPLICIT = 0, 1
DG_HILL = {"none": 0, "gauss": 1, "bell": 2, "parabola": 3}
DG_ATM = {"none": 0, "isothermal": 1, "stratified": 2}
DG_INIT = {"rest": 0, "bubble": 1, "inflow": 2}

c_int, c_int64, c_double, c_void_p = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p


class MeshDesc(ctypes.Structure):
    _fields_ = [
        ("dim", c_int), ("degree", c_int), ("n_cells", c_int64),
        ("level", ctypes.POINTER(ctypes.c_uint8)), ("ijk", ctypes.POINTER(ctypes.c_int32)),
        ("base", c_int * 3), ("extent", c_double * 3), ("periodic", c_int * 3),
        ("hill_kind", c_int), ("hill_hc", c_double), ("hill_half_width", c_double),
        ("hill_xc", c_double), ("hill_yc", c_double),
        ("atm_kind", c_int), ("atm_T", c_double), ("atm_N", c_double), ("atm_p_ref", c_double),
        ("gravity", c_double),
        ("sponge_depth", c_double), ("sponge_rate", c_double), ("sponge_u0", c_double),
        ("sponge_lateral_width", c_double), ("sponge_lateral_rate", c_double),
        ("node_xyz", ctypes.POINTER(c_double)),
        ("n_conforming", c_int64), ("conforming", ctypes.POINTER(ctypes.c_int32)),
        ("n_subfaces", c_int64), ("subfaces", ctypes.POINTER(ctypes.c_int32)),
        ("n_walls", c_int64), ("walls", ctypes.POINTER(ctypes.c_int32)),
    ]


class MeshInfo(ctypes.Structure):
    _fields_ = [
        ("dim", c_int), ("degree", c_int), ("n_vars", c_int), ("nodes_per_cell", c_int),
        ("n_cells", c_int64), ("n_nodes", c_int64), ("n_dof", c_int64),
        ("n_conforming", c_int64), ("n_subfaces", c_int64), ("n_walls", c_int64),
        ("max_level", c_int), ("min_edge", c_double), ("device_bytes", ctypes.c_size_t),
        ("solver_form", c_int * 2), ("solver_ms", (ctypes.c_float * 3) * 2),
        ("n_batches", c_int * 2), ("solver_partition", c_int * 2), ("solver_ms_balanced", (ctypes.c_float * 3) * 2),
    ]


class SolverOpts(ctypes.Structure):
    _fields_ = [
        ("picard", c_int), ("restart", c_int), ("max_iters", c_int), ("tol", c_double),
        ("precision", c_int), ("inner_tol", c_double), ("max_refine", c_int), ("fused", c_int),
        ("krylov", c_int),
    ]


class StepStats(ctypes.Structure):
    _fields_ = [("gmres_iters", c_int), ("solves", c_int), ("refine_steps", c_int), ("max_rel_residual", c_double)]


class ServeOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_members", c_int)]


class Request(ctypes.Structure):
    _fields_ = [
        ("mesh", MeshDesc), ("init_kind", c_int), ("init_params", c_double * 8), ("n_init_params", c_int),
        ("dt", c_double), ("steps", c_int), ("solver", SolverOpts),
    ]


class RequestInfo(ctypes.Structure):
    _fields_ = [
        ("state", c_int), ("status", c_int), ("steps_done", c_int), ("gmres_iters", ctypes.c_longlong),
        ("t_submit", c_double), ("t_admit", c_double), ("t_finish", c_double),
        ("footprint_bytes", ctypes.c_size_t), ("n_dof", c_int64),
    ]


class ServeInfo(ctypes.Structure):
    _fields_ = [("queued", c_int), ("running", c_int), ("used_bytes", ctypes.c_size_t),
                ("ticks", ctypes.c_longlong), ("elapsed_s", c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            "libdgatmo.so is not built (%s); run __graft_entry__.build() or python -m "
            "paper_2408_08129_gb300.build" % LIB_PATH
        )
    lib = ctypes.CDLL(LIB_PATH)
    P = c_void_p
    sig = {
        "dg_ctx_create": (c_int, [c_int, ctypes.POINTER(P)]),
        "dg_ctx_destroy": (c_int, [P]),
        "dg_last_error": (ctypes.c_char_p, []),
        "dg_version": (ctypes.c_char_p, []),
        "dg_profile_enable": (c_int, [P, c_int]),
        "dg_profile_read": (c_int, [P, P, P]),
        "dg_profile_reset": (c_int, [P]),
        "dg_launch_count": (c_int, [P, P]),
        "dg_profile_read_gmres_phases": (c_int, [P, P]),
        "dg_profile_read_cta_passes": (c_int, [P, P, P, P, c_int]),
        "dg_mesh_create": (c_int, [P, ctypes.POINTER(MeshDesc), ctypes.POINTER(P)]),
        "dg_mesh_destroy": (c_int, [P]),
        "dg_mesh_get_info": (c_int, [P, ctypes.POINTER(MeshInfo)]),
        "dg_mesh_set_partition": (c_int, [P, c_int]),
        "dg_mesh_get_faces": (c_int, [P, P, P, P]),
        "dg_mesh_get_coords": (c_int, [P, P]),
        "dg_background": (c_int, [P, P, P, P]),
        "dg_init_state": (c_int, [P, P, c_int, P, c_int, P, P]),
        "dg_apply_explicit": (c_int, [P, P, P, P, c_int, c_int, P]),
        "dg_apply_grad": (c_int, [P, P, P, P, P, c_int, P]),
        "dg_apply_div": (c_int, [P, P, P, P, c_int, P]),
        "dg_apply_implicit": (c_int, [P, P, P, P, P, c_double, c_int, P]),
        "dg_apply_implicit_noalloc": (c_int, [P, P, P, P, P, c_double, c_int, P]),
        "dg_conservation": (c_int, [P, P, P, P, P]),
        "dg_solver_opts_default": (None, [ctypes.POINTER(SolverOpts)]),
        "dg_state_create": (c_int, [P, P, ctypes.POINTER(SolverOpts), ctypes.POINTER(P)]),
        "dg_state_destroy": (c_int, [P]),
        "dg_state_data": (P, [P]),
        "dg_state_upload": (c_int, [P, P]),
        "dg_state_download": (c_int, [P, P]),
        "dg_math_selftest": (c_int, [c_int, P, P, ctypes.c_int64, P]),
        "dg_batch_barrier_test": (c_int, [P, c_double, c_int]),
        "dg_peak_fma": (c_int, [c_int, ctypes.c_int64, c_int, P, P, P]),
        "dg_state_chebyshev_bound": (c_int, [P, P, P]),
        "imex_rk2_step": (c_int, [P, P, P, c_double, ctypes.POINTER(SolverOpts), ctypes.POINTER(StepStats), P]),
        "dg_batch_step": (c_int, [P, c_int, P, P, P, ctypes.POINTER(SolverOpts), P, P, P]),
        "dg_batch_plan_create": (c_int, [P, c_int, P, P, P, ctypes.POINTER(SolverOpts), ctypes.POINTER(P)]),
        "dg_batch_plan_step": (c_int, [P, P, P, P]),
        "dg_batch_plan_destroy": (c_int, [P]),
        "dg_serve_create": (c_int, [P, ctypes.POINTER(ServeOpts), ctypes.POINTER(P)]),
        "dg_serve_submit": (c_int, [P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
        "dg_serve_poll": (c_int, [P, ctypes.c_uint64, ctypes.POINTER(RequestInfo), P]),
        "dg_serve_wait": (c_int, [P, ctypes.c_uint64, c_double]),
        "dg_serve_release": (c_int, [P, ctypes.c_uint64]),
        "dg_serve_stats": (c_int, [P, ctypes.POINTER(ServeInfo)]),
        "dg_serve_destroy": (c_int, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


class DGError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = lib.dg_last_error().decode(errors="replace")
        super().__init__("%s failed: %s (%s)" % (where, DG_STATUS.get(status, status), msg))


def check(status, where):
    if status != DG_OK:
        raise DGError(status, where)
    return status
