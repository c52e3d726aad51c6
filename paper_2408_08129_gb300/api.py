"""Thin Python binding over the C ABI, with the same names (argument marshalling only).

Device arrays are torch CUDA tensors (contiguous, float64 or float32); their
``data_ptr()`` and the current torch stream are handed to the library.  Every
step of the computation runs in the library's CUDA kernels.
"""

import ctypes
from ctypes import c_double

import numpy as np
import torch

from . import _binding as B
from ._binding import (  # noqa: F401
    DG_ATM, DG_FP32, DG_FP64, DG_HILL, DG_INIT, DG_KRYLOV_AUTO, DG_KRYLOV_CG, DG_KRYLOV_CHEBYSHEV, DG_KRYLOV_GMRES, DG_KRYLOV_GMRES_CGS2,
    DG_TERMS_FULL,
    DG_TERMS_IMEX_EXPLICIT, DGError, check, lib,
)


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t, dtype=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError("expected dtype %s, got %s" % (dtype, t.dtype))
    return ctypes.c_void_p(t.data_ptr())


def _fdtype(precision):
    return torch.float64 if precision == DG_FP64 else torch.float32


class Context:
    """dg_ctx on one CUDA device."""

    def __init__(self, device=0):
        h = ctypes.c_void_p()
        check(lib.dg_ctx_create(int(device), ctypes.byref(h)), "dg_ctx_create")
        self.handle = h
        self.device = int(device)

    def close(self):
        if self.handle:
            lib.dg_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mesh_desc(case, gravity=None, node_xyz=None, faces=None):
    """dg_mesh_desc of a workload description; returns (desc, arrays to keep alive).

    node_xyz (dim x cells x nodes, float64) and faces ((conforming, subfaces, walls) int32 tables in
    the layout Mesh.faces() returns) optionally replace the geometry and connectivity the library
    would build from the tree and the terrain map."""
    d = B.MeshDesc()
    d.dim = case.dim
    d.degree = case.degree
    d.n_cells = case.n_cells
    level = np.ascontiguousarray(case.levels, dtype=np.uint8)
    ijk = np.ascontiguousarray(case.ijk, dtype=np.int32)
    d.level = level.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    d.ijk = ijk.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    for a in range(case.dim):
        d.base[a] = case.base[a]
        d.extent[a] = case.extent[a]
        d.periodic[a] = 1 if case.periodic[a] else 0
    hill = case.hill
    d.hill_kind = DG_HILL[hill["kind"]]
    d.hill_hc = hill.get("hc", 0.0)
    d.hill_half_width = hill.get("half_width", 1.0)
    d.hill_xc = hill.get("xc", 0.0)
    d.hill_yc = hill.get("yc", 0.0)
    atm = case.atmosphere
    d.atm_kind = DG_ATM[atm["kind"]]
    d.atm_T = atm.get("T0", atm.get("T_ref", 0.0))
    d.atm_N = atm.get("N", 0.0)
    d.atm_p_ref = atm.get("p_ref", 0.0)
    d.gravity = case.gravity if gravity is None else gravity
    sp = getattr(case, "sponge", None) or {}
    d.sponge_depth = sp.get("depth", 0.0)
    d.sponge_rate = sp.get("rate", 0.0)
    d.sponge_u0 = sp.get("u0", 0.0)
    d.sponge_lateral_width = sp.get("lateral_width", 0.0)
    d.sponge_lateral_rate = sp.get("lateral_rate", 0.0)
    keep = [level, ijk]
    if node_xyz is not None:
        X = np.ascontiguousarray(node_xyz, dtype=np.float64)
        if X.shape != (case.dim, case.n_cells, case.nodes_per_cell):
            raise ValueError("node_xyz must have shape (dim, cells, nodes per cell)")
        d.node_xyz = X.ctypes.data_as(ctypes.POINTER(c_double))
        keep.append(X)
    if faces is not None:
        conf, subs, walls = (np.ascontiguousarray(t, dtype=np.int32) for t in faces)
        for name, t, w in (("conforming", conf, 4), ("subfaces", subs, 4), ("walls", walls, 2)):
            if t.ndim != 2 or t.shape[1] != w:
                raise ValueError("%s table must have shape (n, %d)" % (name, w))
            setattr(d, "n_" + name, t.shape[0])
            setattr(d, name, t.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
            keep.append(t)
    return d, tuple(keep)


def init_params(case):
    """(dg_init_kind, parameter list) of a workload's initial state."""
    init = case.init
    if init["kind"] == "bubble":
        p = [init["amp"], init["radius"], init["xc"], init["zc"]]
        if case.dim == 3:
            p.append(init.get("yc", 0.5 * case.extent[1]))
        return DG_INIT["bubble"], p
    if init["kind"] == "inflow":
        return DG_INIT["inflow"], [init.get("u0", 10.0)]
    return DG_INIT["rest"], []


class Mesh:
    """dg_mesh built from a workload description (see workloads.Case)."""

    def __init__(self, ctx, case, gravity=None, node_xyz=None, faces=None):
        d, self._keep = mesh_desc(case, gravity, node_xyz, faces)
        h = ctypes.c_void_p()
        check(lib.dg_mesh_create(ctx.handle, ctypes.byref(d), ctypes.byref(h)), "dg_mesh_create")
        self.handle = h
        self.ctx = ctx
        self.case = case
        info = B.MeshInfo()
        check(lib.dg_mesh_get_info(h, ctypes.byref(info)), "dg_mesh_get_info")
        self.info = {k: getattr(info, k) for k, _ in B.MeshInfo._fields_
                     if k not in ("solver_form", "solver_ms", "n_batches", "solver_partition", "solver_ms_balanced")}
        self.n_batches = tuple(info.n_batches)
        self.dim = case.dim
        self.n_vars = info.n_vars
        self.n_cells = info.n_cells
        self.nodes_per_cell = info.nodes_per_cell
        self.n_nodes = info.n_nodes
        self.n_dof = info.n_dof

    def autotuned(self):
        """Autotuner outcome: per precision, the chosen Helmholtz solver form and cell partition
        ("uniform": CPB consecutive cells per batch; "balanced": cost-balanced batches, one per CTA of
        a persistent solve) and the timed solves (ms) on each partition."""
        info = B.MeshInfo()
        check(lib.dg_mesh_get_info(self.handle, ctypes.byref(info)), "dg_mesh_get_info")
        forms = {0: "gmres_multi_kernel", 1: "gmres_persistent", 2: "chebyshev", -1: None}
        parts = ("uniform", "balanced")
        return {p: {"form": forms[info.solver_form[i]],
                    "partition": parts[info.solver_partition[i]],
                    "batches": {parts[k]: info.n_batches[k] for k in range(2) if info.n_batches[k] > 0},
                    "ms": {forms[f]: info.solver_ms[i][f] for f in range(3) if info.solver_ms[i][f] > 0},
                    "ms_balanced": {forms[f]: info.solver_ms_balanced[i][f] for f in range(3)
                                    if info.solver_ms_balanced[i][f] > 0}}
                for i, p in enumerate(("fp64", "fp32"))}

    def set_partition(self, k):
        """Cell partition of the implicit passes: 0 uniform batches, 1 cost-balanced (where built)."""
        check(lib.dg_mesh_set_partition(self.handle, int(k)), "dg_mesh_set_partition")

    def faces(self):
        i = self.info
        conf = np.zeros((i["n_conforming"], 4), np.int32)
        subs = np.zeros((i["n_subfaces"], 4), np.int32)
        walls = np.zeros((i["n_walls"], 2), np.int32)
        check(lib.dg_mesh_get_faces(self.handle, conf.ctypes.data, subs.ctypes.data, walls.ctypes.data),
              "dg_mesh_get_faces")
        return conf, subs, walls

    def coords(self):
        X = np.zeros((self.dim, self.n_cells, self.nodes_per_cell))
        check(lib.dg_mesh_get_coords(self.handle, X.ctypes.data), "dg_mesh_get_coords")
        return X

    def shape(self, nv=None):
        return (self.n_vars if nv is None else nv, self.n_cells, self.nodes_per_cell)

    def close(self):
        if self.handle:
            lib.dg_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


PROF_CATEGORIES = {0: "explicit", 1: "helmholtz", 2: "grad", 3: "div", 4: "krylov", 5: "gmres", 6: "step"}


def dg_profile_enable(ctx, on=True):
    check(lib.dg_profile_enable(ctx.handle, int(on)), "dg_profile_enable")


def dg_profile_reset(ctx):
    check(lib.dg_profile_reset(ctx.handle), "dg_profile_reset")


def dg_profile_read(ctx):
    ms = np.zeros(8)
    n = np.zeros(8, dtype=np.int64)
    check(lib.dg_profile_read(ctx.handle, ms.ctypes.data, n.ctypes.data), "dg_profile_read")
    return {name: {"ms": float(ms[i]), "count": int(n[i])} for i, name in PROF_CATEGORIES.items()}


GMRES_PHASES = {1: "gradient", 3: "divergence", 4: "gs_dots_barrier", 5: "basis_update_barrier",
                6: "gs_second_pass", 7: "fp64_residual", 8: "solution_update", 9: "gs_dots_work",
                10: "partial_sums", 11: "givens", 12: "coefficients", 13: "basis_update_work"}


def dg_profile_read_gmres_phases(ctx):
    ns = np.zeros(16)
    check(lib.dg_profile_read_gmres_phases(ctx.handle, ns.ctypes.data), "dg_profile_read_gmres_phases")
    out = {name: ns[i] / 1e6 for i, name in GMRES_PHASES.items()}  # ms
    out["iterations"] = int(ns[15])
    out["second_passes"] = int(ns[14])
    return out


def dg_profile_read_cta_passes(ctx, max_ctas=512):
    """Per-CTA pass clocks of the persistent Chebyshev solves: (grad_ns, div_ns, coarse) arrays."""
    g = np.zeros(max_ctas)
    d = np.zeros(max_ctas)
    c = np.zeros(max_ctas, dtype=np.int32)
    check(lib.dg_profile_read_cta_passes(ctx.handle, g.ctypes.data, d.ctypes.data, c.ctypes.data, int(max_ctas)),
          "dg_profile_read_cta_passes")
    return g, d, c


def dg_math_selftest(op, x, y, stream=None):
    """Device self-test of the library's FP64 math (op 0: the Newton 1/sqrt); x, y: CUDA float64 tensors."""
    check(lib.dg_math_selftest(int(op), _ptr(x), _ptr(y), x.numel(), _stream(stream)), "dg_math_selftest")
    return y


def dg_batch_barrier_test(ctx, barrier_limit_s=2.0, missing_cta_member=-1):
    """Bounded-barrier test hook of batched launches (see include/dg_atmo.h)."""
    check(lib.dg_batch_barrier_test(ctx.handle, float(barrier_limit_s), int(missing_cta_member)),
          "dg_batch_barrier_test")


def dg_peak_fma(precision, iters, blocks, out, stream=None):
    """Enqueue the FMA-throughput probe; returns the floating-point operations it performs."""
    fl = ctypes.c_double(0.0)
    check(lib.dg_peak_fma(int(precision), int(iters), int(blocks), _ptr(out), _stream(stream), ctypes.byref(fl)),
          "dg_peak_fma")
    return float(fl.value)


def dg_launch_count(ctx):
    n = ctypes.c_longlong(0)
    check(lib.dg_launch_count(ctx.handle, ctypes.byref(n)), "dg_launch_count")
    return int(n.value)


def dg_background(ctx, mesh, Ubg, stream=None):
    check(lib.dg_background(ctx.handle, mesh.handle, _ptr(Ubg, torch.float64), _stream(stream)), "dg_background")


def dg_init_state(ctx, mesh, kind, params, U, stream=None):
    arr = (ctypes.c_double * max(1, len(params)))(*params)
    check(lib.dg_init_state(ctx.handle, mesh.handle, DG_INIT[kind] if isinstance(kind, str) else kind, arr,
                            len(params), _ptr(U, torch.float64), _stream(stream)), "dg_init_state")


def dg_apply_explicit(ctx, mesh, U, R, precision=DG_FP64, terms=DG_TERMS_FULL, stream=None):
    dt = _fdtype(precision)
    check(lib.dg_apply_explicit(ctx.handle, mesh.handle, _ptr(U, dt), _ptr(R, dt), precision, terms,
                                _stream(stream)), "dg_apply_explicit")


def dg_apply_grad(ctx, mesh, p, g, h=None, precision=DG_FP64, stream=None):
    dt = _fdtype(precision)
    check(lib.dg_apply_grad(ctx.handle, mesh.handle, _ptr(p, dt), _ptr(h, dt), _ptr(g, dt), precision,
                            _stream(stream)), "dg_apply_grad")


def dg_apply_div(ctx, mesh, f, out, precision=DG_FP64, stream=None):
    dt = _fdtype(precision)
    check(lib.dg_apply_div(ctx.handle, mesh.handle, _ptr(f, dt), _ptr(out, dt), precision, _stream(stream)),
          "dg_apply_div")


def dg_apply_implicit(ctx, mesh, h, p, Ap, alpha, precision=DG_FP64, stream=None):
    dt = _fdtype(precision)
    check(lib.dg_apply_implicit(ctx.handle, mesh.handle, _ptr(h, dt), _ptr(p, dt), _ptr(Ap, dt), float(alpha),
                                precision, _stream(stream)), "dg_apply_implicit")


def dg_apply_implicit_noalloc(ctx, mesh, h, p, Ap, alpha, precision=DG_FP64, stream=None):
    """dg_apply_implicit without any device allocation (scratch in a fixed 4 MiB library array)."""
    dt = _fdtype(precision)
    check(lib.dg_apply_implicit_noalloc(ctx.handle, mesh.handle, _ptr(h, dt), _ptr(p, dt), _ptr(Ap, dt),
                                        float(alpha), precision, _stream(stream)), "dg_apply_implicit_noalloc")


def dg_conservation(ctx, mesh, U, out, stream=None):
    check(lib.dg_conservation(ctx.handle, mesh.handle, _ptr(U, torch.float64), _ptr(out, torch.float64),
                              _stream(stream)), "dg_conservation")


def solver_opts(**kw):
    o = B.SolverOpts()
    lib.dg_solver_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class _DeviceArray:
    """Exposes a library-owned device buffer to torch through __cuda_array_interface__."""

    def __init__(self, ptr, shape, owner):
        self._owner = owner
        self.__cuda_array_interface__ = {
            "shape": tuple(shape), "typestr": "<f8", "data": (int(ptr), False), "version": 3, "strides": None,
        }


class State:
    """dg_state: the device-resident FP64 solution and the step workspaces."""

    def __init__(self, ctx, mesh, opts=None):
        h = ctypes.c_void_p()
        o = opts if opts is not None else solver_opts()
        check(lib.dg_state_create(ctx.handle, mesh.handle, ctypes.byref(o), ctypes.byref(h)), "dg_state_create")
        self.handle = h
        self.ctx = ctx
        self.mesh = mesh
        ptr = lib.dg_state_data(h)
        self.U = torch.as_tensor(_DeviceArray(ptr, mesh.shape(), self), device="cuda:%d" % ctx.device)

    def upload(self, host_U):
        a = np.ascontiguousarray(host_U, dtype=np.float64)
        check(lib.dg_state_upload(self.handle, a.ctypes.data), "dg_state_upload")

    def download(self):
        a = np.zeros(self.mesh.shape())
        check(lib.dg_state_download(self.handle, a.ctypes.data), "dg_state_download")
        return a

    def chebyshev_bound(self, set_to=None):
        """(lmax, alpha) the state's Chebyshev solves use; set_to=(lmax, alpha) replaces it first."""
        get = np.zeros(2)
        st = None if set_to is None else np.asarray(set_to, dtype=np.float64)
        check(lib.dg_state_chebyshev_bound(self.handle, get.ctypes.data,
                                           None if st is None else st.ctypes.data), "dg_state_chebyshev_bound")
        return (float(get[0]), float(get[1])) if set_to is None else self.chebyshev_bound()

    def close(self):
        if self.handle:
            lib.dg_state_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def imex_rk2_step(ctx, mesh, state, dt, opts=None, stream=None, raise_on_error=True):
    o = opts if opts is not None else solver_opts()
    st = B.StepStats()
    rc = lib.imex_rk2_step(ctx.handle, mesh.handle, state.handle, float(dt), ctypes.byref(o), ctypes.byref(st),
                           _stream(stream))
    if raise_on_error:
        check(rc, "imex_rk2_step")
    return {k: getattr(st, k) for k, _ in B.StepStats._fields_} | {"status": rc}


def dg_batch_step(ctx, meshes, states, dts, opts=None, stream=None, raise_on_error=True):
    """One IMEX-RK2 step of every member (mesh, state, dt); solves batched per (dim, degree, precision)."""
    n = len(states)
    if not (len(meshes) == n == len(dts)):
        raise ValueError("meshes, states and dts must have the same length")
    o = opts if opts is not None else solver_opts()
    mh = (ctypes.c_void_p * n)(*[m.handle.value for m in meshes])
    sh = (ctypes.c_void_p * n)(*[st.handle.value for st in states])
    dt = (ctypes.c_double * n)(*[float(x) for x in dts])
    stats = (B.StepStats * n)()
    statuses = (ctypes.c_int * n)()
    rc = lib.dg_batch_step(ctx.handle, n, mh, sh, dt, ctypes.byref(o), stats, statuses, _stream(stream))
    if raise_on_error:
        check(rc, "dg_batch_step")
    out = []
    for i in range(n):
        d = {k: getattr(stats[i], k) for k, _ in B.StepStats._fields_}
        d["status"] = statuses[i]
        out.append(d)
    return out


class BatchPlan:
    """dg_batch_plan: the ensemble step of dg_batch_step captured once as a CUDA graph, then replayed.

    Keeps references to the meshes and states, which the plan uses on every step.
    """

    def __init__(self, ctx, meshes, states, dts, opts=None):
        n = len(states)
        if not (len(meshes) == n == len(dts)):
            raise ValueError("meshes, states and dts must have the same length")
        self.ctx, self.meshes, self.states, self.n = ctx, list(meshes), list(states), n
        o = opts if opts is not None else solver_opts()
        mh = (ctypes.c_void_p * n)(*[m.handle.value for m in meshes])
        sh = (ctypes.c_void_p * n)(*[st.handle.value for st in states])
        dt = (ctypes.c_double * n)(*[float(x) for x in dts])
        h = ctypes.c_void_p()
        check(lib.dg_batch_plan_create(ctx.handle, n, mh, sh, dt, ctypes.byref(o), ctypes.byref(h)),
              "dg_batch_plan_create")
        self.handle = h

    def step(self, stream=None, raise_on_error=True):
        stats = (B.StepStats * self.n)()
        statuses = (ctypes.c_int * self.n)()
        rc = lib.dg_batch_plan_step(self.handle, stats, statuses, _stream(stream))
        if raise_on_error:
            check(rc, "dg_batch_plan_step")
        out = []
        for i in range(self.n):
            d = {k: getattr(stats[i], k) for k, _ in B.StepStats._fields_}
            d["status"] = statuses[i]
            out.append(d)
        return out

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib.dg_batch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


REQ_STATES = {0: "queued", 1: "running", 2: "done", 3: "failed"}


class Server:
    """dg_server: request loop with memory-budget admission and continuous batching."""

    def __init__(self, ctx, hbm_budget_bytes, max_members=0):
        o = B.ServeOpts(hbm_budget_bytes=int(hbm_budget_bytes), max_members=int(max_members))
        h = ctypes.c_void_p()
        check(lib.dg_serve_create(ctx.handle, ctypes.byref(o), ctypes.byref(h)), "dg_serve_create")
        self.handle = h
        self._shapes = {}

    def submit(self, case, steps, dt=None, opts=None):
        r = B.Request()
        desc, keep = mesh_desc(case)
        r.mesh = desc
        kind, params = init_params(case)
        r.init_kind = kind
        for i, v in enumerate(params):
            r.init_params[i] = v
        r.n_init_params = len(params)
        r.dt = case.dt if dt is None else dt
        r.steps = int(steps)
        r.solver = opts if opts is not None else solver_opts()
        rid = ctypes.c_uint64()
        check(lib.dg_serve_submit(self.handle, ctypes.byref(r), ctypes.byref(rid)), "dg_serve_submit")
        self._shapes[rid.value] = (case.dim + 2, case.n_cells, (case.degree + 1) ** case.dim)
        return rid.value

    def poll(self, rid, with_result=False):
        info = B.RequestInfo()
        U = np.zeros(self._shapes[rid]) if with_result else None
        check(lib.dg_serve_poll(self.handle, rid, ctypes.byref(info), U.ctypes.data if U is not None else None),
              "dg_serve_poll")
        d = {k: getattr(info, k) for k, _ in B.RequestInfo._fields_}
        d["state"] = REQ_STATES[d["state"]]
        if with_result:
            d["U"] = U
        return d

    def wait(self, rid, timeout_s=600.0):
        check(lib.dg_serve_wait(self.handle, rid, float(timeout_s)), "dg_serve_wait")

    def release(self, rid):
        check(lib.dg_serve_release(self.handle, rid), "dg_serve_release")
        self._shapes.pop(rid, None)

    def stats(self):
        i = B.ServeInfo()
        check(lib.dg_serve_stats(self.handle, ctypes.byref(i)), "dg_serve_stats")
        return {k: getattr(i, k) for k, _ in B.ServeInfo._fields_}

    def close(self):
        if self.handle:
            lib.dg_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def last_error():
    """Message of the last non-OK status returned by the library on this thread."""
    return lib.dg_last_error().decode(errors="replace")
