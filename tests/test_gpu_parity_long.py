"""CUDA path vs the FP64 CPU oracle on the full workloads, over many steps.

* hill2d (64x32 base quads, two 2:1 levels near the ground, degree 4, 291,200
  DoF): 100 FP64 IMEX-RK2 steps within 1e-10 of the oracle (relative L2 of the
  deviation from the hydrostatic background, per variable), and 10 steps of the
  FP32-refined form (FP32 Krylov iterations inside FP64 iterative refinement)
  within the 1e-8 of that form.
* hill3d (32x32x16 base hexahedra, one 2:1 level, degree 3, 7.5 M DoF): one
  step in FP64 and one in the FP32-refined form against one oracle step, held
  to the step bars of the two forms (1e-10 and 1e-8).  A step holds six
  Helmholtz solves stopped at relative residual 1e-12; on this mesh one step
  measures about 1.4e-11.

The oracle trajectories are computed once per module (about two minutes of
host time for hill2d, one and a half for the hill3d step).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.dg import DG  # noqa: E402
from oracle.imex import Stepper  # noqa: E402
from workloads import make_case  # noqa: E402


@pytest.fixture(scope="module")
def dg():
    import paper_2408_08129_gb300 as m

    return m


@pytest.fixture(scope="module")
def ctx(dg):
    return dg.Context(0)


def _dev_err(U, Ur, Ubg):
    """Largest per-variable relative L2 error of the deviation from the background."""
    return max(np.linalg.norm((U - Ur)[v]) / np.linalg.norm((Ur - Ubg)[v]) for v in range(U.shape[0]))


@pytest.fixture(scope="module")
def hill2d_oracle():
    case = make_case("hill2d", 0)
    ref = DG(case)
    st = Stepper(ref, tol=1e-12)
    U = ref.state()
    traj = {0: U}
    for k in range(1, 101):
        U = st.step(U, case.dt)
        if k in (10, 100):
            traj[k] = U
    return case, ref, traj


def _gpu_steps(dg, ctx, case, U0, n, opts):
    mesh = dg.Mesh(ctx, case)
    st = dg.State(ctx, mesh, opts)
    st.upload(U0)
    worst = 0.0
    for _ in range(n):
        s = dg.imex_rk2_step(ctx, mesh, st, case.dt, opts)
        worst = max(worst, s["max_rel_residual"])
    U = st.download()
    st.close()
    mesh.close()
    return U, worst


def test_hill2d_100_fp64_steps_match_oracle(dg, ctx, hill2d_oracle):
    case, ref, traj = hill2d_oracle
    U, res = _gpu_steps(dg, ctx, case, traj[0], 100, dg.solver_opts(tol=1e-12))
    assert res <= 1e-12
    err = _dev_err(U, traj[100], ref.Ubg)
    assert err < 1e-10, err


def test_hill2d_10_fp32_refined_steps_match_oracle(dg, ctx, hill2d_oracle):
    case, ref, traj = hill2d_oracle
    opts = dg.solver_opts(tol=1e-12, precision=dg.DG_FP32, inner_tol=1e-6)
    U, res = _gpu_steps(dg, ctx, case, traj[0], 10, opts)
    assert res <= 1e-12
    err = _dev_err(U, traj[10], ref.Ubg)
    assert err < 1e-8, err


@pytest.fixture(scope="module")
def hill3d_oracle():
    case = make_case("hill3d", 0)
    ref = DG(case)
    U0 = ref.state()
    U1 = Stepper(ref, tol=1e-12).step(U0, case.dt)
    return case, ref, U0, U1


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-8)])
def test_hill3d_step_matches_oracle(dg, ctx, hill3d_oracle, precision, tol):
    case, ref, U0, U1 = hill3d_oracle
    prec = dg.DG_FP64 if precision == "fp64" else dg.DG_FP32
    U, res = _gpu_steps(dg, ctx, case, U0, 1, dg.solver_opts(tol=1e-12, precision=prec, inner_tol=1e-6))
    assert res <= 1e-12
    err = _dev_err(U, U1, ref.Ubg)
    assert err < tol, err
