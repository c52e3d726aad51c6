"""Ensemble steps: many uneven members in one batched step equal each member stepped alone.

The batched launch gives every member its own share of CTAs, so its dot
products are cut into different chunks than in a solo solve; the results agree
to the Krylov tolerance, not bit for bit.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from workloads.cases import member2d  # noqa: E402


@pytest.fixture(scope="module")
def dg():
    import paper_2408_08129_gb300 as m

    return m


@pytest.fixture(scope="module")
def ctx(dg):
    return dg.Context(0)


def _init(dg, ctx, mesh, case, state):
    init = case.init
    if init["kind"] == "bubble":
        dg.dg_init_state(ctx, mesh, "bubble", [init["amp"], init["radius"], init["xc"], init["zc"]], state.U)
    else:
        dg.dg_init_state(ctx, mesh, "inflow", [init["u0"]], state.U)


def _rel_dev(a, b, bg):
    return max(np.linalg.norm(a[v] - b[v]) / max(np.linalg.norm(b[v] - bg[v]), 1e-300) for v in range(a.shape[0]))


@pytest.mark.parametrize("precision,krylov", [("fp64", 0), ("fp32", 0), ("fp64", 1), ("fp32", 1), ("fp64", 3),
                                             ("fp32", 3)])
def test_batch_equals_alone(dg, ctx, precision, krylov):
    prec = dg.DG_FP64 if precision == "fp64" else dg.DG_FP32
    opts = dg.solver_opts(tol=1e-12, precision=prec, inner_tol=1e-4, krylov=krylov, fused=1)
    seeds = [1000, 1003, 1004, 1005, 1007, 1008, 1011, 1006]  # degrees 2..5, 16x8 .. 64x32, 0-2 levels
    cases = [member2d(s) for s in seeds]
    alone, meshes, states = [], [], []
    for case in cases:
        mesh = dg.Mesh(ctx, case)
        st = dg.State(ctx, mesh, opts)
        _init(dg, ctx, mesh, case, st)
        for _ in range(2):
            dg.imex_rk2_step(ctx, mesh, st, case.dt, opts)
        alone.append(st.download())
        _init(dg, ctx, mesh, case, st)
        meshes.append(mesh)
        states.append(st)
    for _ in range(2):
        res = dg.dg_batch_step(ctx, meshes, states, [c.dt for c in cases], opts)
        assert all(r["status"] == 0 for r in res)
    for case, mesh, st, ref in zip(cases, meshes, states, alone):
        bg = torch.empty(mesh.shape(), dtype=torch.float64, device="cuda")
        dg.dg_background(ctx, mesh, bg)
        err = _rel_dev(st.download(), ref, bg.cpu().numpy())
        assert err < 1e-9, (case.degree, case.base, err)


def test_batch_rejects_shared_mesh(dg, ctx):
    case = member2d(1007)
    mesh = dg.Mesh(ctx, case)
    a, b = dg.State(ctx, mesh), dg.State(ctx, mesh)
    with pytest.raises(dg.DGError, match="share a mesh"):
        dg.dg_batch_step(ctx, [mesh, mesh], [a, b], [case.dt, case.dt])


def test_batch_member_matches_oracle(dg, ctx):
    """One batched step of a small member against the CPU oracle."""
    from oracle.dg import DG
    from oracle.imex import Stepper

    case = member2d(1007)
    other = member2d(1011)
    ref = DG(case)
    U0 = ref.state()
    meshes = [dg.Mesh(ctx, case), dg.Mesh(ctx, other)]
    opts = dg.solver_opts(tol=1e-12)
    states = [dg.State(ctx, meshes[0], opts), dg.State(ctx, meshes[1], opts)]
    states[0].upload(U0)
    _init(dg, ctx, meshes[1], other, states[1])
    dg.dg_batch_step(ctx, meshes, states, [case.dt, other.dt], opts)
    Ur = Stepper(ref, tol=1e-12).step(U0, case.dt)
    assert _rel_dev(states[0].download(), Ur, ref.Ubg) < 1e-10


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_plan_replays_equal_batch_steps(dg, ctx, precision):
    """A captured batch plan computes bit for bit what dg_batch_step computes, step after step."""
    prec = dg.DG_FP64 if precision == "fp64" else dg.DG_FP32
    opts = dg.solver_opts(tol=1e-12, precision=prec, inner_tol=1e-4)
    seeds = [1000, 1003, 1004, 1005, 1007, 1008, 1011, 1006]
    cases = [member2d(s) for s in seeds]
    dts = [c.dt for c in cases]
    ma = [dg.Mesh(ctx, c) for c in cases]
    mb = [dg.Mesh(ctx, c) for c in cases]
    sa = [dg.State(ctx, m, opts) for m in ma]
    sb = [dg.State(ctx, m, opts) for m in mb]
    for c, m, st in zip(cases, ma, sa):
        _init(dg, ctx, m, c, st)
    for c, m, st in zip(cases, mb, sb):
        _init(dg, ctx, m, c, st)
    plan = dg.BatchPlan(ctx, mb, sb, dts, opts)
    for _ in range(3):
        ra = dg.dg_batch_step(ctx, ma, sa, dts, opts)
        n0 = dg.dg_launch_count(ctx)
        rb = plan.step()
        assert dg.dg_launch_count(ctx) > n0  # the graph's kernels are counted
        assert [r["gmres_iters"] for r in ra] == [r["gmres_iters"] for r in rb]
        assert all(r["status"] == 0 for r in rb)
    for a, b in zip(sa, sb):
        assert np.array_equal(a.download(), b.download())
    plan.close()


def test_plan_rejects_multi_kernel_solves(dg, ctx):
    case = member2d(1007)
    mesh = dg.Mesh(ctx, case)
    st = dg.State(ctx, mesh)
    with pytest.raises(dg.DGError, match="persistent solve"):
        dg.BatchPlan(ctx, [mesh], [st], [case.dt], dg.solver_opts(fused=0, krylov=dg.DG_KRYLOV_GMRES))
