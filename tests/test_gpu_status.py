"""Error statuses of the step entry points, provoked without faulting the GPU.

* DG_ENOTCONV: a Helmholtz solve capped at one iteration misses its tolerance,
  for every solver form (and the reported residual is the final one).
* DG_ENONFINITE: a state uploaded from the host with a NaN gives a non-finite
  step result; the Krylov loops stay bounded by max_iters.
* DG_ETIMEOUT: the batched launch's bounded barrier runs out when one member
  is told it has one CTA more than the launch gives it (a host-side test hook:
  the wait simply expires after a few milliseconds and the kernel returns);
  the same context then runs a clean batched step that matches the oracle.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.dg import DG  # noqa: E402
from oracle.imex import Stepper  # noqa: E402
from workloads import make_case  # noqa: E402
from workloads.cases import member2d  # noqa: E402

DG_ENOTCONV, DG_ENONFINITE, DG_ETIMEOUT = -4, -5, -8


@pytest.fixture(scope="module")
def dg():
    import paper_2408_08129_gb300 as m

    return m


@pytest.fixture(scope="module")
def ctx(dg):
    return dg.Context(0)


@pytest.mark.parametrize("krylov,fused", [("chebyshev", 1), ("gmres", 1), ("gmres", 0), ("cg", 1),
                                          ("gmres_cgs2", 1)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_not_converged_status(dg, ctx, krylov, fused, precision):
    kry = {"chebyshev": dg.DG_KRYLOV_CHEBYSHEV, "gmres": dg.DG_KRYLOV_GMRES, "cg": dg.DG_KRYLOV_CG,
           "gmres_cgs2": dg.DG_KRYLOV_GMRES_CGS2}[krylov]
    prec = dg.DG_FP64 if precision == "fp64" else dg.DG_FP32
    case = make_case("bubble2d", 0)
    ref = DG(case)
    mesh = dg.Mesh(ctx, case)
    opts = dg.solver_opts(tol=1e-12, max_iters=1, max_refine=1, krylov=kry, fused=fused, precision=prec)
    st = dg.State(ctx, mesh, opts)
    st.upload(ref.state())
    stats = dg.imex_rk2_step(ctx, mesh, st, case.dt, opts, raise_on_error=False)
    assert stats["status"] == DG_ENOTCONV, stats
    assert "tolerance" in dg.api.last_error()
    assert stats["max_rel_residual"] > 1e-12  # the final residual, not a converged one
    # the same state and mesh still step cleanly with the normal cap
    ok = dg.solver_opts(tol=1e-12, krylov=kry, fused=fused, precision=prec)
    st.upload(ref.state())
    assert dg.imex_rk2_step(ctx, mesh, st, case.dt, ok)["status"] == 0


def test_non_finite_status(dg, ctx):
    case = make_case("bubble2d", 0)
    ref = DG(case)
    mesh = dg.Mesh(ctx, case)
    opts = dg.solver_opts(tol=1e-12, max_iters=50)
    st = dg.State(ctx, mesh, opts)
    U = ref.state()
    U[0, 5, 3] = np.nan
    st.upload(U)
    stats = dg.imex_rk2_step(ctx, mesh, st, case.dt, opts, raise_on_error=False)
    assert stats["status"] == DG_ENONFINITE, stats
    assert not np.isfinite(st.download()).all()
    with pytest.raises(dg.DGError, match="non-finite"):
        st.upload(U)
        dg.imex_rk2_step(ctx, mesh, st, case.dt, opts)
    # a finite state on the same objects steps cleanly
    st.upload(ref.state())
    assert dg.imex_rk2_step(ctx, mesh, st, case.dt, opts)["status"] == 0


def test_batched_barrier_timeout_then_clean_step(dg, ctx):
    cases = [member2d(s) for s in (1003, 1007)]  # both degree 4: one batched launch
    opts = dg.solver_opts(tol=1e-12, krylov=dg.DG_KRYLOV_CHEBYSHEV, fused=1)
    meshes = [dg.Mesh(ctx, c) for c in cases]
    states = [dg.State(ctx, m, opts) for m in meshes]
    refs = [DG(c) for c in cases]
    U0 = [r.state() for r in refs]
    for st, u in zip(states, U0):
        st.upload(u)
    dts = [c.dt for c in cases]
    try:
        dg.dg_batch_barrier_test(ctx, 5e-3, 1)
        res = dg.dg_batch_step(ctx, meshes, states, dts, opts, raise_on_error=False)
        assert [r["status"] for r in res] == [DG_ETIMEOUT, DG_ETIMEOUT], res
        assert "barrier" in dg.api.last_error()
    finally:
        dg.dg_batch_barrier_test(ctx, 2.0, -1)
    for st, u in zip(states, U0):
        st.upload(u)
    res = dg.dg_batch_step(ctx, meshes, states, dts, opts)
    assert all(r["status"] == 0 for r in res)
    for st, ref, u, c in zip(states, refs, U0, cases):
        Ur = Stepper(ref, tol=1e-12).step(u, c.dt)
        err = max(np.linalg.norm((st.download() - Ur)[v]) / np.linalg.norm((Ur - ref.Ubg)[v]) for v in range(4))
        assert err < 1e-9, err


def test_barrier_test_hook_validates(dg, ctx):
    for bad in ((0.0, -1), (20.0, -1), (1.0, -2)):
        with pytest.raises(dg.DGError):
            dg.dg_batch_barrier_test(ctx, *bad)
