#!/usr/bin/env python
"""Benchmark of the GB300 DG solver on the 2D flow-over-orography workload.

Workload (one "step" = one IMEX-RK2 time step, i.e. one pass of the whole hot
path: explicit DG applies, the pressure Picard loop with GMRES on the
Helmholtz operator, gradients/divergences, the stage updates):
  hill2d -- 64x32 base quads over 40 km x 20 km, Gaussian hill (seeded), two
  2:1 refinement levels near the ground (2912 cells), degree 4, FP64,
  constant-N atmosphere with a 10 m/s inflow, 291,200 DoF.

Metric: DoF-steps per second (DoF x steps / s), whole job over all ranks.
Under torchrun each rank runs an independent replica (the workload is a
single mesh that this build does not partition), so scaling is weak.

``--impl reference`` times the CPU oracle (the plain FP64 restatement of the
method) on the same workload, on the host cores.
"""

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# per-node algorithmic counts (collocated GLL, sum factorised; see the design notes)
#   explicit apply: bytes/DoF = s (2 + 1/V); flops/node = 2Vdn + 2Vd^2 + P_vol + (d/n) P_face + V
#   Helmholtz apply: bytes/node = 3 s;       flops/node = 2 (2dn + 2d^2) + 10
P_VOL = {2: 25, 3: 45}
P_FACE = {2: 70, 3: 90}
# ALU peaks: measured at start-up by the library's FMA-throughput probe (measure_alu_peaks); these
# nominal figures (SM count x FMA lanes x 2 x maximum clock) stand in only if the probe fails
ALU_PEAK_TFLOPS = {"fp64": 152 * 4 * 2.07e9 / 1e12, "fp32": 152 * 256 * 2.07e9 / 1e12}
ALU_PEAK_SOURCE = "nominal"
L2_FLUSH_BYTES = 256 << 20
# dram__bytes_read.sum + dram__bytes_write.sum per launch from one ncu capture of the kernel as it
# stands (the persistent solve with the autotuned Chebyshev body, FP64, on hill2d); set to None
# whenever that kernel changes
NCU_TRAFFIC_BYTES = {("hill2d", "chebyshev", "fp64"): 5.022e6 + 0.298e6}


def algorithmic(dim, degree, n_nodes, kind, s=8):
    n = degree + 1
    V = dim + 2
    if kind == "explicit":
        flops = 2 * V * dim * n + 2 * V * dim * dim + P_VOL[dim] + (dim / n) * P_FACE[dim] + V
        byts = s * (2 * V + 1)
    else:
        flops = 2 * (2 * dim * n + 2 * dim * dim) + 10
        byts = 3 * s
    return flops * n_nodes, byts * n_nodes


def max_over_ranks(x, dist, device):
    """The largest of the ranks' x (the job's time is that of its slowest replica)."""
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, dof, steps, total_ms):
    """DoF-steps per second of the whole job: every rank advances its own replica of `dof` DoF."""
    return world * dof * steps / (total_ms / 1e3)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def measure_alu_peaks(dg, torch, reps=5):
    """FP64 and FP32 FMA throughput of the whole GPU: the library's probe (16 independent FMA chains
    per thread, 8 CTAs of 256 threads per SM), best of `reps` launches timed with CUDA events, with
    the SM clock sampled meanwhile.  Sets ALU_PEAK_TFLOPS to the measured values."""
    global ALU_PEAK_SOURCE
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks = 8 * sms
    stream = torch.cuda.current_stream()
    out = {}
    clk = Clocks(os.path.join(tempfile.gettempdir(), "dg_bench_peak_clocks.csv"))
    with clk:
        for name, prec, dtype, iters in (("fp64", dg.DG_FP64, torch.float64, 4096),
                                         ("fp32", dg.DG_FP32, torch.float32, 262144)):
            buf = torch.empty(blocks * 256, dtype=dtype, device="cuda")
            dg.dg_peak_fma(prec, 64, blocks, buf)
            torch.cuda.synchronize()
            best = None
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fl = dg.dg_peak_fma(prec, iters, blocks, buf)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
            out[name] = fl / (best / 1e3) / 1e12
            if not math.isfinite(float(buf.sum())):
                raise RuntimeError("FMA probe produced non-finite values")
    c = clk.summary(torch.cuda.current_device())
    for k in ("fp64", "fp32"):
        ALU_PEAK_TFLOPS[k] = out[k]
    ALU_PEAK_SOURCE = "measured"
    return {"fp64_tflops": out["fp64"], "fp32_tflops": out["fp32"], "sm_mhz": c.get("sm_mhz"),
            "sm_max_mhz": c.get("sm_max_mhz"), "reasons": c.get("reasons"),
            "how": "dg_peak_fma: 16 independent FMA chains per thread, %d CTAs x 256 threads, best of %d "
                   "launches timed with CUDA events" % (blocks, reps)}


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self, device):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines()]
        except Exception:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = [[c.strip() for c in r] for r in rows if len(r) >= 9 and r[0].strip() == str(device)]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


_ORACLE_STEPS = r"""
import json, os, sys, time
sys.path.insert(0, %r)
from workloads import make_case
from oracle.dg import DG
from oracle.imex import Stepper
case = make_case(%r, 0)
dg = DG(case)
st = Stepper(dg, tol=1e-12)
U = dg.state()
n = 0
t0 = time.perf_counter()
while True:
    U = st.step(U, case.dt)
    n += 1
    if time.perf_counter() - t0 > %f:
        break
el = time.perf_counter() - t0
print(json.dumps({"steps": n, "seconds": el, "dof": case.n_dof}))
"""


def _one_thread_env():
    return dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")


def cpu_baseline_sample(case_name, seconds, replicas=None):
    """Time the CPU oracle (as it stands) on whole IMEX-RK2 steps of the workload, on the host cores:
    `replicas` independent single-threaded oracle processes (default: one per host core) stepping
    the same case for about `seconds` each, and one of them alone.  Returns the all-cores figure
    with the one-thread figure beside it."""
    ncores = os.cpu_count() or 1
    replicas = replicas or ncores
    code = _ORACLE_STEPS % (ROOT, case_name, seconds)

    def run(n):
        procs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                  text=True, env=_one_thread_env()) for _ in range(n)]
        outs = []
        for p in procs:
            o, e = p.communicate(timeout=900)
            if p.returncode != 0:
                raise RuntimeError(e[-2000:])
            outs.append(json.loads(o.strip().splitlines()[-1]))
        return outs

    one = run(1)[0]
    many = run(replicas)
    v1 = one["dof"] * one["steps"] / one["seconds"]
    vall = sum(d["dof"] * d["steps"] / d["seconds"] for d in many)
    return {"value": vall, "unit": "DoF/s", "cores": replicas, "kind": "oracle",
            "sample": "%d independent single-threaded oracle processes on %d host cores, each %d-%d IMEX-RK2 "
                      "steps of %s (about %.0f s each); whole-job DoF-steps/s" % (
                          replicas, ncores, min(d["steps"] for d in many), max(d["steps"] for d in many),
                          case_name, seconds),
            "one_thread": {"value": v1, "unit": "DoF/s", "cores": 1,
                           "sample": "%d step(s) of %s on 1 host thread (%.1f s)" % (one["steps"], case_name,
                                                                                   one["seconds"])}}


def start_oracle_step(case_name, path, threads):
    """One oracle IMEX-RK2 step of a workload from its initial state, in a background process that
    writes the result to `path` (.npy); returns the process."""
    code = r"""
import sys
import numpy as np
sys.path.insert(0, %r)
from workloads import make_case
from oracle.dg import DG
from oracle.imex import Stepper
case = make_case(%r, 0)
dg = DG(case)
U1 = Stepper(dg, tol=1e-12).step(dg.state(), case.dt)
np.save(%r, U1)
np.save(%r, dg.Ubg)
""" % (ROOT, case_name, path, path + ".bg.npy")
    env = dict(os.environ, OMP_NUM_THREADS=str(threads), OPENBLAS_NUM_THREADS=str(threads),
               MKL_NUM_THREADS=str(threads))
    return subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.DEVNULL, stderr=subprocess.PIPE,
                            text=True, env=env)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per_step = max(3.0, 60.0 / max(1, args.steps + args.warmup))
    cb = cpu_baseline_sample(args.workload, min(20.0, per_step * max(1, args.steps)))
    line = {
        "impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "DoF/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": CONFIG[args.workload],
        "cpu_baseline": cb,
        "e2e": {"value": cb["value"], "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def precision_forms_3d(dg, torch, case_name="hill3d", steps=2, inner_tol=1e-6):
    """The 3D workload stepped in FP64 and in the FP32-refined form from the same start (autotuned
    solver each): time per step, the FP32 form's deviation from the FP64 result, and each form's
    state after one step (returned under "_one_step" for the comparison with the oracle)."""
    import numpy as np
    from workloads import make_case

    case = make_case(case_name, 0)
    ctx = dg.Context(torch.cuda.current_device())
    mesh = dg.Mesh(ctx, case)
    st = dg.State(ctx, mesh)
    kind, params = dg.api.init_params(case)
    dg.dg_init_state(ctx, mesh, kind, params, st.U)
    U0 = st.download()
    bg = torch.empty(mesh.shape(), dtype=torch.float64, device="cuda")
    dg.dg_background(ctx, mesh, bg)
    bg = bg.cpu().numpy()
    stream = torch.cuda.current_stream()
    out, res, one_step = {}, {}, {}
    for name, prec in (("fp64", dg.DG_FP64), ("fp32_refined", dg.DG_FP32)):
        o = dg.solver_opts(tol=1e-12, precision=prec, inner_tol=inner_tol)
        st.upload(U0)
        dg.imex_rk2_step(ctx, mesh, st, case.dt, o)  # warm-up (and the autotuner's first solve)
        st.upload(U0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            dg.imex_rk2_step(ctx, mesh, st, case.dt, o)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        res[name] = st.download()
        st.upload(U0)
        dg.imex_rk2_step(ctx, mesh, st, case.dt, o)
        one_step[name] = st.download()
        out[name] = {"ms_per_step": ms, "dof_steps_per_s": mesh.n_dof / (ms / 1e3),
                     "solver": mesh.autotuned()[name[:4]]["form"], "helmholtz_kappa": spectrum_of(st)}
    dev = max(np.linalg.norm(res["fp32_refined"][v] - res["fp64"][v])
              / max(np.linalg.norm(res["fp64"][v] - bg[v]), 1e-300) for v in range(mesh.n_vars))
    out["fp32_refined"]["speedup_vs_fp64"] = out["fp64"]["ms_per_step"] / out["fp32_refined"]["ms_per_step"]
    out["fp32_refined"]["rel_err_vs_fp64_deviation"] = dev
    out["workload"] = "%s: %d cells, degree %d, %d DoF, %d IMEX-RK2 steps per form" % (
        case_name, mesh.n_cells, case.degree, mesh.n_dof, steps)
    st.close()
    mesh.close()
    ctx.close()
    out["_one_step"] = one_step
    return out


def cta_pass_summary(grad_ns, div_ns, coarse, steps):
    """Per-CTA pass clocks of the persistent Chebyshev solve, per step: the slowest CTA against the
    mean one, split by whether the CTA's cell batch holds a coarse side (the 2:1 face work)."""
    used = (grad_ns + div_ns) > 0
    if not used.any():
        return None
    g, d, c = grad_ns[used] / 1e3 / steps, div_ns[used] / 1e3 / steps, coarse[used] > 0
    out = {"ctas": int(used.sum()), "coarse_ctas": int(c.sum())}
    for name, sel in (("coarse", c), ("plain", ~c)):
        if sel.any():
            out["grad_mean_" + name] = float(g[sel].mean())
            out["grad_max_" + name] = float(g[sel].max())
            out["div_mean_" + name] = float(d[sel].mean())
            out["div_max_" + name] = float(d[sel].max())
    return out


def spectrum_of(state):
    """Condition number of the state's last Helmholtz operator: the power-iteration upper bound the
    Chebyshev solves keep (less its 5% margin) over the lower bound 1/(gamma-1) = 2.5 (0 if the
    state has not run a Chebyshev solve)."""
    lmax, _ = state.chebyshev_bound()
    return lmax / 1.05 / 2.5 if lmax > 0 else 0.0


def paper_pair(dg, torch, steps=3):
    """Sec. 3.1/3.2's comparison: the bell-shaped hill on the uniform 60x40x16 mesh and on the
    non-conforming mesh of the same finest resolution, FP64 IMEX-RK2 steps of dt = 2 s (autotuned
    Helmholtz solver), timed with CUDA events after one warm-up step; the wall clock of T_f = 1 h
    (1800 steps) extrapolated from the step time, beside the paper's figures (context only)."""
    from workloads import make_case

    out = {}
    stream = torch.cuda.current_stream()
    for name in ("bell3d_nc", "bell3d_uniform"):
        case = make_case(name, 0)
        ctx = dg.Context(torch.cuda.current_device())
        mesh = dg.Mesh(ctx, case)
        o = dg.solver_opts(tol=1e-12)
        st = dg.State(ctx, mesh, o)
        kind, params = dg.api.init_params(case)
        dg.dg_init_state(ctx, mesh, kind, params, st.U)
        dg.imex_rk2_step(ctx, mesh, st, case.dt, o)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        its = 0
        for _ in range(steps):
            its += dg.imex_rk2_step(ctx, mesh, st, case.dt, o)["gmres_iters"]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"cells": mesh.n_cells, "dof": mesh.n_dof, "ms_per_step": ms,
                     "dof_steps_per_s": mesh.n_dof / (ms / 1e3), "iters_per_step": its / steps,
                     "wall_clock_1h_s": 1800 * ms / 1e3, "solver": mesh.autotuned()["fp64"]["form"],
                     "helmholtz_kappa": spectrum_of(st)}
        st.close()
        mesh.close()
        ctx.close()
    nc, un = out["bell3d_nc"], out["bell3d_uniform"]
    out["saving_vs_uniform"] = 1.0 - nc["ms_per_step"] / un["ms_per_step"]
    out["paper"] = ("Sec. 3.2, context only: 2560 s (1958-cell non-conforming mesh) vs 36500 s (uniform "
                    "60x40x16) wall clock, a ~93% saving, on MeluXina CPU nodes (core count not stated)")
    return out


def oracle_errors(forms, proc, path):
    """Relative L2 error (largest over the variables, of the deviation from the background) of each
    form's one-step state against the oracle's step, once the background oracle process is done."""
    import numpy as np

    one = forms.pop("_one_step")
    try:
        _, err = proc.communicate(timeout=1800)
        if proc.returncode != 0:
            raise RuntimeError(err[-500:])
        U1 = np.load(path)
        bg = np.load(path + ".bg.npy")
    except Exception as e:  # reported, not hidden
        forms["oracle"] = {"error": str(e)[:300]}
        return forms
    for name, U in one.items():
        forms[name]["rel_err_vs_oracle_one_step"] = max(
            float(np.linalg.norm(U[v] - U1[v]) / np.linalg.norm(U1[v] - bg[v])) for v in range(U.shape[0]))
    forms["oracle"] = "one oracle IMEX-RK2 step from the same initial state (FP64, CPU), same dt and tolerances"
    return forms


def apply_sweep(dg, torch, case_name, reps=10):
    """Throughput of the operator applies on a mesh whose vectors exceed L2 (FP64 and FP32)."""
    from workloads import make_case

    case = make_case(case_name, 0)
    ctx = dg.Context(torch.cuda.current_device())
    mesh = dg.Mesh(ctx, case)
    hbm, src = measured_peaks()
    stream = torch.cuda.current_stream()
    U = torch.empty(mesh.shape(), dtype=torch.float64, device="cuda")
    dg.dg_init_state(ctx, mesh, "inflow", [10.0], U)
    Ubg = torch.empty_like(U)
    dg.dg_background(ctx, mesh, Ubg)
    U += 1e-3 * torch.randn_like(U) * Ubg.abs().clamp(min=1.0)
    Up32 = (U - Ubg).float()
    shp = (mesh.n_cells, mesh.nodes_per_cell)
    p64 = 100.0 * torch.randn(shp, dtype=torch.float64, device="cuda")
    h64 = torch.full(shp, 3.5e5, dtype=torch.float64, device="cuda")
    p32, h32 = p64.float(), h64.float()
    out = {}

    def timeit(fn):
        fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    n = mesh.n_nodes
    for prec, name, s_b in ((dg.DG_FP64, "fp64", 8), (dg.DG_FP32, "fp32", 4)):
        peak = ALU_PEAK_TFLOPS[name]
        Uin = U if prec == dg.DG_FP64 else Up32
        R = torch.empty_like(Uin)
        t = timeit(lambda: dg.dg_apply_explicit(ctx, mesh, Uin, R, prec, dg.DG_TERMS_FULL))
        fl, by = algorithmic(case.dim, case.degree, n, "explicit", s_b)
        out["explicit_" + name] = {"ms": t, "dof_per_s": mesh.n_dof / (t / 1e3), "alg_gbs": by / (t / 1e3) / 1e9,
                                   "hbm_frac": by / (t / 1e3) / 1e9 / hbm, "tflops": fl / (t / 1e3) / 1e12,
                                   "alu_frac": fl / (t / 1e3) / 1e12 / peak}
        pp, hh = (p64, h64) if prec == dg.DG_FP64 else (p32, h32)
        Ap = torch.empty_like(pp)
        t = timeit(lambda: dg.dg_apply_implicit(ctx, mesh, hh, pp, Ap, 1.0, prec))
        fl, by = algorithmic(case.dim, case.degree, n, "helmholtz", s_b)
        out["helmholtz_" + name] = {"ms": t, "dof_per_s": n / (t / 1e3), "alg_gbs": by / (t / 1e3) / 1e9,
                                    "hbm_frac": by / (t / 1e3) / 1e9 / hbm, "tflops": fl / (t / 1e3) / 1e12,
                                    "alu_frac": fl / (t / 1e3) / 1e12 / peak}
    out["workload"] = "%s: %d cells, degree %d, %d DoF (vectors larger than L2)" % (
        case_name, mesh.n_cells, case.degree, mesh.n_dof)
    out["hbm_peak_gbs"] = hbm
    out["peaks"] = "HBM %s (%.0f GB/s); FP64 %.3f and FP32 %.1f TFLOP/s %s (FMA-throughput probe)" % (
        src, hbm, ALU_PEAK_TFLOPS["fp64"], ALU_PEAK_TFLOPS["fp32"], ALU_PEAK_SOURCE)
    mesh.close()
    ctx.close()
    return out


def ensemble_bench(dg, torch, n_members=64, steps=10, inner_tol=1e-6):
    """64 uneven 2D members (16x8..128x64 base, 0-2 levels, degree 2-5), FP32-refined: one
    dg_batch_step per ensemble step, then the same step as a captured batch plan (CUDA graph)."""
    from workloads.cases import member2d

    ctx = dg.Context(torch.cuda.current_device())
    cases = [member2d(1000 + i) for i in range(n_members)]
    opts = dg.solver_opts(tol=1e-12, precision=dg.DG_FP32, inner_tol=inner_tol)
    meshes = [dg.Mesh(ctx, c) for c in cases]
    states = [dg.State(ctx, m, opts) for m in meshes]
    for c, m, st in zip(cases, meshes, states):
        kind, params = dg.api.init_params(c)
        dg.dg_init_state(ctx, m, kind, params, st.U)
    dts = [c.dt for c in cases]
    dg.dg_batch_step(ctx, meshes, states, dts, opts)  # warm-up
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    iters = 0
    for _ in range(steps):
        res = dg.dg_batch_step(ctx, meshes, states, dts, opts)
        iters += sum(r["gmres_iters"] for r in res)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    # the same step captured once as a CUDA graph (members on parallel branches), then replayed
    t0 = time.perf_counter()
    plan = dg.BatchPlan(ctx, meshes, states, dts, opts)
    capture_ms = (time.perf_counter() - t0) * 1e3
    plan.step()  # warm-up
    torch.cuda.synchronize()
    n0 = dg.dg_launch_count(ctx)
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    giters = 0
    for _ in range(steps):
        res = plan.step()
        giters += sum(r["gmres_iters"] for r in res)
    g1.record(stream)
    torch.cuda.synchronize()
    gms = g0.elapsed_time(g1)
    kernels_per_step = (dg.dg_launch_count(ctx) - n0) / steps
    plan.close()
    kap = {}
    for c, st in zip(cases, states):
        kap.setdefault("r%d" % c.degree, []).append(spectrum_of(st))
    kappa_by_degree = {k: {"min": min(v), "max": max(v), "members": len(v)} for k, v in sorted(kap.items())}
    dof = sum(m.n_dof for m in meshes)
    out = {"workload": "%d 2D members (base 16x8..128x64, 0-2 levels, degree 2-5), %d DoF in all, "
                       "FP32 Krylov + FP64 residual, one CUDA-graph replay per ensemble step" % (n_members, dof),
           "member_steps_per_s": n_members * steps / (gms / 1e3), "dof_steps_per_s": dof * steps / (gms / 1e3),
           "ms_per_ensemble_step": gms / steps, "gmres_iters_per_member_step": giters / (n_members * steps),
           "graph_capture_ms": capture_ms, "kernels_per_ensemble_step": kernels_per_step,
           "helmholtz_kappa_by_degree": kappa_by_degree,
           "without_graph": {"ms_per_ensemble_step": ms / steps,
                             "member_steps_per_s": n_members * steps / (ms / 1e3),
                             "gmres_iters_per_member_step": iters / (n_members * steps)}}
    for st in states:
        st.close()
    for m in meshes:
        m.close()
    ctx.close()
    return out


def serving_bench(dg, torch, n_requests=24, rate=20.0, dof_hi=5e6, steps_lo=10, steps_hi=500, budget=160e9,
                  inner_tol=1e-6):
    """The serving stream: Poisson arrivals, 2D/3D, degree 2-5, DoF 1e4-5e6 log-uniform, 10-500 steps,
    FP64 or FP32-refined; the first n_requests requests of the seeded trace."""
    from workloads.cases import serving_trace

    trace = serving_trace(7, n_requests, rate, 1e4, dof_hi, steps_lo, steps_hi)
    ctx = dg.Context(torch.cuda.current_device())
    sv = dg.Server(ctx, int(budget))
    t0 = time.perf_counter()
    ids = []
    for (t_arr, case, steps, prec) in trace:
        now = time.perf_counter() - t0
        if t_arr > now:
            time.sleep(t_arr - now)
        o = dg.solver_opts(tol=1e-10, precision=dg.DG_FP64 if prec == "fp64" else dg.DG_FP32, inner_tol=inner_tol)
        ids.append((sv.submit(case, steps, opts=o), case, steps))
    for rid, _, _ in ids:
        sv.wait(rid, 900)
    infos = [sv.poll(rid) for rid, _, _ in ids]
    ok = [i for i in infos if i["state"] == "done"]
    from paper_2408_08129_gb300._binding import DG_STATUS
    failed = [{"status": DG_STATUS.get(i["status"], i["status"]), "dim": c.dim, "degree": c.degree, "dof": c.n_dof,
               "steps": s, "precision": p, "steps_done": i["steps_done"], "init": c.init["kind"]}
              for i, (_, c, s), (_, _, _, p) in zip(infos, ids, trace) if i["state"] != "done"]
    lat = sorted(i["t_finish"] - i["t_submit"] for i in ok)
    t_first = min(i["t_submit"] for i in infos)
    t_last = max(i["t_finish"] for i in infos)
    span = t_last - t_first
    steps_total = sum(s for _, _, s in ids)
    dof_steps = sum(c.n_dof * s for _, c, s in ids)
    stats = sv.stats()
    sv.close()
    ctx.close()

    def pct(q):
        return lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))] if lat else None

    return {"workload": "%d requests, Poisson %.0f/s, 2D/3D, degree 2-5, DoF 1e4-%.0e log-uniform, %d-%d steps, "
                        "FP64 or FP32-refined 50/50, %.0f GB budget (the first %d requests of the seeded stream; "
                        "the full ranges of DoF and steps, fewer requests to keep the bench within minutes)"
                        % (n_requests, rate, dof_hi, steps_lo, steps_hi, budget / 1e9, n_requests),
            "dof_steps_total": dof_steps,
            "completed": len(ok), "failed": failed, "p50_s": pct(0.5), "p99_s": pct(0.99), "makespan_s": span,
            "member_steps_per_s": steps_total / span, "dof_steps_per_s": dof_steps / span,
            "ticks": stats["ticks"]}


METRIC = "DG apply DoF/s fp64 vs fp32, %HBM peak; ensemble steps/s, p50/p99 latency"
CONFIG = {
    "hill2d": {
        "workload": "hill2d: 2D x-z flow over a seeded Gaussian hill, 64x32 base quads over 40x20 km, "
                    "two 2:1 refinement levels near the ground (2912 cells), degree 4, FP64, "
                    "constant-N atmosphere + 10 m/s inflow; IMEX-RK2 steps, 3 Picard iterations per implicit "
                    "stage, Helmholtz solves to relative residual 1e-12",
        "dof": 291200,
        "l2": "flushed between timed steps (256 MB write)",
    },
    "bubble2d": {
        "workload": "bubble2d: 16x8 conforming quads, degree 2, FP64 warm bubble; IMEX-RK2 steps",
        "dof": 4608,
        "l2": "flushed between timed steps (256 MB write)",
    },
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="hill2d", choices=sorted(CONFIG))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sweep", action="store_true", help="skip the operator-apply sweep on the large 3D mesh")
    ap.add_argument("--sweep-workload", default="hill3d_big")
    ap.add_argument("--sweep-only", action="store_true", help="run only the operator-apply sweep")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the ensemble and serving measurements")
    ap.add_argument("--krylov", default="auto", choices=["auto", "gmres", "gmres_cgs2", "cg", "chebyshev"],
                    help="linear solver of the timed steps (auto: autotuned among GMRES and Chebyshev; "
                         "the other forms are timed beside it)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"],
                    help="fp32 = FP32 Krylov iterations inside FP64 refinement")
    ap.add_argument("--no-forms", action="store_true", help="skip the FP32-refined and other-solver comparisons")
    ap.add_argument("--inner-tol", type=float, default=1e-6,
                    help="FP32-refined forms: residual reduction of each FP32 inner cycle")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    import paper_2408_08129_gb300 as dg
    from workloads import make_case

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    try:
        peaks = measure_alu_peaks(dg, torch)
    except Exception as e:  # the nominal figures stay, and the line says so
        peaks = {"error": str(e)[:200]}
    if args.sweep_only:
        print(json.dumps({"alu_peaks": peaks, "applies": apply_sweep(dg, torch, args.sweep_workload)}))
        return
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")

    case = make_case(args.workload, 0)
    ctx = dg.Context(local)
    mesh = dg.Mesh(ctx, case)
    kry = {"auto": dg.DG_KRYLOV_AUTO, "gmres": dg.DG_KRYLOV_GMRES, "gmres_cgs2": dg.DG_KRYLOV_GMRES_CGS2,
           "cg": dg.DG_KRYLOV_CG, "chebyshev": dg.DG_KRYLOV_CHEBYSHEV}[args.krylov]
    prec = dg.DG_FP64 if args.precision == "fp64" else dg.DG_FP32
    opts = dg.solver_opts(tol=1e-12, picard=3, restart=30, krylov=kry, precision=prec, inner_tol=args.inner_tol)
    state = dg.State(ctx, mesh, opts)
    init = case.init
    if init["kind"] == "bubble":
        dg.dg_init_state(ctx, mesh, "bubble", [init["amp"], init["radius"], init["xc"], init["zc"]], state.U)
    else:
        dg.dg_init_state(ctx, mesh, "inflow", [init.get("u0", 10.0)], state.U)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        dg.imex_rk2_step(ctx, mesh, state, case.dt, opts)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    U_start = state.download()
    dg.dg_profile_reset(ctx)
    dg.dg_profile_enable(ctx, True)
    launches0 = dg.dg_launch_count(ctx)
    times = []
    stats = []
    clk = Clocks(os.path.join(tempfile.gettempdir(), "dg_bench_clocks_%d.csv" % rank))
    with clk:
        for _ in range(args.steps):
            flush.zero_()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev0.record(stream)
            stats.append(dg.imex_rk2_step(ctx, mesh, state, case.dt, opts))
            ev1.record(stream)
            torch.cuda.synchronize()
            times.append(ev0.elapsed_time(ev1))
    launches = dg.dg_launch_count(ctx) - launches0
    prof = dg.dg_profile_read(ctx)
    dg.dg_profile_enable(ctx, False)
    total_ms = sum(times)
    if world > 1:
        total_ms = max_over_ranks(total_ms, dist, "cuda")
        dist.barrier()
    dof = mesh.n_dof
    value = whole_job_value(world, dof, args.steps, total_ms)

    U64 = state.download()
    # a few more (untimed) steps with the clocks inside the persistent solves on: per-phase time
    # as seen by block 0, and every CTA's own gradient and divergence passes
    clock_steps = max(1, min(args.steps, 5))
    dg.dg_profile_reset(ctx)
    dg.dg_profile_enable(ctx, 2)
    for _ in range(clock_steps):
        dg.imex_rk2_step(ctx, mesh, state, case.dt, opts)
    phases = dg.dg_profile_read_gmres_phases(ctx)
    cta_passes = cta_pass_summary(*dg.dg_profile_read_cta_passes(ctx), clock_steps)
    dg.dg_profile_enable(ctx, False)
    state.upload(U64)
    kappa = spectrum_of(state)

    Ubg = torch.empty(mesh.shape(), dtype=torch.float64, device="cuda")
    dg.dg_background(ctx, mesh, Ubg)
    Ubg = Ubg.cpu().numpy()
    tuned = mesh.autotuned()  # the headline's choice, before the other forms run
    fp32, cg = None, None
    if not args.no_forms:
        # the FP32-refined form from the same start: FP32 applies + FP32 inner GMRES, FP64 outer residual
        opts32 = dg.solver_opts(tol=1e-12, picard=3, restart=30, precision=dg.DG_FP32, inner_tol=args.inner_tol)
        state.upload(U_start)
        for _ in range(args.warmup):  # untimed: lazy loading and the autotuner's first FP32 solve
            dg.imex_rk2_step(ctx, mesh, state, case.dt, opts32)
        state.upload(U_start)
        times32, its32 = [], 0
        for _ in range(args.steps):
            flush.zero_()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev0.record(stream)
            its32 += dg.imex_rk2_step(ctx, mesh, state, case.dt, opts32)["gmres_iters"]
            ev1.record(stream)
            torch.cuda.synchronize()
            times32.append(ev0.elapsed_time(ev1))
        U32 = state.download()
        rel_full = max(np.linalg.norm(U32[v] - U64[v]) / np.linalg.norm(U64[v]) for v in range(mesh.n_vars))
        rel_dev = max(np.linalg.norm(U32[v] - U64[v]) / max(np.linalg.norm(U64[v] - Ubg[v]), 1e-300)
                      for v in range(mesh.n_vars))
        fp32 = {"ms_per_step": sum(times32) / args.steps,
                "value": world * dof * args.steps / (sum(times32) / 1e3),
                "speedup_vs_fp64": sum(times) / sum(times32),
                "inner_iters_per_step": its32 / args.steps,
                "rel_err_vs_fp64_full_state": rel_full,
                "rel_err_vs_fp64_deviation": rel_dev,
                "solver": mesh.autotuned()["fp32"]["form"]}
        # other Krylov forms from the same start: GMRES with classical Gram-Schmidt twice per step, and
        # conjugate gradients (the Helmholtz operator is self-adjoint in the w J inner product)
        cg = {}
        for name, prec, kry in (("gmres_fp64", dg.DG_FP64, dg.DG_KRYLOV_GMRES),
                                ("gmres_fp32_refined", dg.DG_FP32, dg.DG_KRYLOV_GMRES),
                                ("gmres_cgs2_fp64", dg.DG_FP64, dg.DG_KRYLOV_GMRES_CGS2),
                                ("cg_fp64", dg.DG_FP64, dg.DG_KRYLOV_CG),
                                ("cg_fp32_refined", dg.DG_FP32, dg.DG_KRYLOV_CG),
                                ("chebyshev_fp64", dg.DG_FP64, dg.DG_KRYLOV_CHEBYSHEV),
                                ("chebyshev_fp32_refined", dg.DG_FP32, dg.DG_KRYLOV_CHEBYSHEV)):
            o = dg.solver_opts(tol=1e-12, picard=3, restart=30, precision=prec, inner_tol=args.inner_tol, krylov=kry,
                               fused=-1 if kry == dg.DG_KRYLOV_GMRES else 1)
            state.upload(U_start)
            for _ in range(args.warmup):
                dg.imex_rk2_step(ctx, mesh, state, case.dt, o)
            state.upload(U_start)
            tms, its = [], 0
            for _ in range(args.steps):
                flush.zero_()
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                ev0.record(stream)
                its += dg.imex_rk2_step(ctx, mesh, state, case.dt, o)["gmres_iters"]
                ev1.record(stream)
                torch.cuda.synchronize()
                tms.append(ev0.elapsed_time(ev1))
            Uc = state.download()
            cg[name] = {"ms_per_step": sum(tms) / args.steps, "value": world * dof * args.steps / (sum(tms) / 1e3),
                        "speedup_vs_headline": sum(times) / sum(tms), "iters_per_step": its / args.steps,
                        "rel_err_vs_headline_deviation": max(
                            np.linalg.norm(Uc[v] - U64[v]) / max(np.linalg.norm(U64[v] - Ubg[v]), 1e-300)
                            for v in range(mesh.n_vars))}
            # one more (untimed) step with the per-phase clock of the persistent solve on
            dg.dg_profile_reset(ctx)
            dg.dg_profile_enable(ctx, 2)
            dg.imex_rk2_step(ctx, mesh, state, case.dt, o)
            ph = dg.dg_profile_read_gmres_phases(ctx)
            dg.dg_profile_enable(ctx, False)
            cg[name]["phase_us_per_iteration"] = {k: round(1e3 * v / max(1, ph["iterations"]), 3) for k, v in ph.items()
                                                  if k not in ("iterations", "second_passes") and v > 0}
    state.upload(U64)

    # end to end through the C ABI with host buffers: upload, step, download per step
    host = torch.empty(mesh.shape(), dtype=torch.float64, pin_memory=True).numpy()
    host[:] = state.download()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        state.upload(host)
        dg.imex_rk2_step(ctx, mesh, state, case.dt, opts)
        host[:] = state.download()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": world * dof * args.steps / e2e_s, "unit": "DoF/s",
           "h2d_bytes_per_step": int(host.nbytes), "d2h_bytes_per_step": int(host.nbytes)}

    # the oracle's hill3d step for the precision forms, in the background while the GPU sections run
    oracle_proc, oracle_path = None, None
    if rank == 0 and not args.no_sweep:
        oracle_path = os.path.join(tempfile.gettempdir(), "dg_bench_oracle_hill3d_%d.npy" % os.getpid())
        oracle_proc = start_oracle_step("hill3d", oracle_path, max(1, (os.cpu_count() or 2) // 2))

    # roofline of the dominant operator class inside the timed region
    cats = {k: v for k, v in prof.items()
            if k in ("explicit", "helmholtz", "grad", "div", "krylov", "gmres") and v["count"]}
    dom = max(cats, key=lambda k: cats[k]["ms"])
    avg_ms = cats[dom]["ms"] / cats[dom]["count"]
    hbm, peak_src = measured_peaks()
    n = mesh.n_nodes
    helm_flops, helm_bytes = algorithmic(case.dim, case.degree, n, "helmholtz")
    expl_flops, expl_bytes = algorithmic(case.dim, case.degree, n, "explicit")
    iters = sum(s["gmres_iters"] for s in stats)
    solves = sum(s["solves"] for s in stats)
    traffic_key = (args.workload, dom, args.precision)
    if dom == "gmres":
        # one launch = one whole solve; it = mean iterations per solve.  GMRES: per iteration
        # one Helmholtz mat-vec and Gram-Schmidt twice over the k+1 basis vectors (two dots +
        # two axpys, 8 (k+1) flops/node), plus the residual mat-vec.  Chebyshev: per iteration
        # one mat-vec and the three-vector update (8 flops/node), plus the residual mat-vec.
        it = iters / max(1, solves)
        form = (tuned[args.precision]["form"] or "") if args.krylov == "auto" else args.krylov
        if "chebyshev" in form:
            flops = (it + 1) * helm_flops + n * 8.0 * it
            name = "gmres_persistent_kernel (persistent Chebyshev solve)"
            traffic_key = (args.workload, "chebyshev", args.precision)
        else:
            flops = (it + 1) * helm_flops + n * (4.0 * it * (it + 1) + 4.0 * it)
            name = "gmres_persistent_kernel (persistent GMRES solve)"
            traffic_key = (args.workload, "gmres", args.precision)
    elif dom == "explicit":
        flops = expl_flops
        name = "explicit apply (face + cell kernels)"
    else:
        flops = helm_flops
        name = dom
    achieved = flops / (avg_ms / 1e3) / 1e12
    pk = ALU_PEAK_TFLOPS[args.precision]
    roof = {"kernel": name, "bound": "alu", "achieved": achieved, "peak": pk, "unit": "TFLOP/s",
            "frac": achieved / pk,
            "peak_source": "%s %s FMA throughput (dg_peak_fma probe at start-up)" % (ALU_PEAK_SOURCE, args.precision),
            "traffic": NCU_TRAFFIC_BYTES.get(traffic_key), "traffic_unit": "bytes per launch",
            "avg_launch_us": avg_ms * 1e3, "launches": cats[dom]["count"],
            "hbm_peak_gbs": hbm, "hbm_peak_source": peak_src}

    line = {
        "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic", "config": dict(CONFIG[args.workload], replicas=world, precision=args.precision, krylov=args.krylov),
        "roofline": roof,
        "breakdown_ms_per_step": {k: v["ms"] / args.steps for k, v in prof.items()},
        "gmres_phase_us_per_iteration": {k: 1e3 * v / max(1, phases["iterations"]) for k, v in phases.items()
                                         if k not in ("iterations", "second_passes")},
        "cta_pass_us_per_step": cta_passes,
        "gmres_iters_per_step": statistics.mean(s["gmres_iters"] for s in stats),
        "helmholtz_kappa": kappa,
        "autotuned_solver": tuned,
        "fp32_refined": fp32,
        "other_krylov_forms": cg,
        "e2e": e2e, "gpu_launches": launches, "alu_peaks": peaks,
        "clocks": clk.summary(local),
    }
    forms3d = None
    if rank == 0 and not args.no_sweep:
        line["applies"] = apply_sweep(dg, torch, args.sweep_workload)
        forms3d = precision_forms_3d(dg, torch, inner_tol=args.inner_tol)
        line["paper_pair"] = paper_pair(dg, torch)
    if rank == 0 and not args.no_ensemble:
        line["ensemble"] = ensemble_bench(dg, torch, inner_tol=args.inner_tol)
        line["serving"] = serving_bench(dg, torch, inner_tol=args.inner_tol)
    if forms3d is not None:
        line["precision_forms_3d"] = oracle_errors(forms3d, oracle_proc, oracle_path)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample(args.workload, 10.0)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
