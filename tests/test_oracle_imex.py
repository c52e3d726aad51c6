"""Pins of the oracle's IMEX-RK2 integrator, pressure loop and GMRES (no GPU)."""

import math

import numpy as np
import pytest

from oracle.dg import DG
from oracle.imex import A_EX, A_IM, B, Stepper, gmres
from workloads import make_case, tiny_case

STRAT = dict(kind="stratified", N=0.01, T_ref=293.15, p_ref=1e5)


def test_tableau_order_conditions():
    """ARK2: consistent rows, sum b = 1, b.c = b.ct = 1/2, stiffly accurate implicit part."""
    c = A_EX.sum(axis=1)
    ct = A_IM.sum(axis=1)
    assert np.allclose(c, ct)
    assert np.allclose(c, [0.0, 2.0 - math.sqrt(2.0), 1.0])
    assert abs(B.sum() - 1.0) < 1e-15
    assert abs(B @ c - 0.5) < 1e-15 and abs(B @ ct - 0.5) < 1e-15
    assert np.allclose(A_IM[2], B)
    assert np.allclose(np.triu(A_EX), 0.0)
    assert np.allclose(np.triu(A_IM, 1), 0.0)


def test_gmres_matches_direct_solve():
    """GMRES on the assembled Helmholtz operator agrees with a dense LU solve."""
    case = tiny_case(2, 2, refine=[(0, 0)], hill=dict(kind="gauss", hc=300.0, half_width=700.0, xc=1.5e3), atmosphere=STRAT)
    dg = DG(case)
    K, nc = dg.mesh.K, dg.mesh.nc
    N = K * nc
    h = 1e5 * (1 + 0.1 * np.random.default_rng(0).random((K, nc)))
    A = np.stack([dg.helmholtz(np.eye(N)[j].reshape(K, nc), h, 50.0).ravel() for j in range(N)], axis=1)
    b = np.random.default_rng(1).standard_normal(N)
    x, it, rel = gmres(lambda q: A @ q, b, np.zeros(N), 1e-13, restart=10)
    exact = np.linalg.solve(A, b)
    assert rel <= 1e-13 and it > 10  # restarted at least once
    assert np.abs(x - exact).max() < 1e-11 * np.abs(exact).max()
    assert np.linalg.norm(b - A @ x) < 1e-12 * np.linalg.norm(b)


@pytest.mark.parametrize("dim", [2, 3])
def test_rest_state_preserved_by_a_step(dim):
    ext = (3e3, 2e3) if dim == 2 else (2e3, 2e3, 2e3)
    hill = dict(kind="gauss", hc=200.0, half_width=600.0, xc=ext[0] / 2, yc=ext[1] / 2)
    case = tiny_case(dim, 2, refine=[(0, 0, 0)[:dim]], hill=hill, atmosphere=STRAT)
    dg = DG(case)
    U1 = Stepper(dg).step(dg.Ubg, case.dt)
    for v in range(dg.V):
        assert np.abs(U1[v] - dg.Ubg[v]).max() <= 1e-12 * np.abs(dg.Ubg[v]).max() + 1e-9


def test_mass_conserved_over_steps():
    case = tiny_case(2, 3, base=(6, 4), extent=(6e3, 4e3), refine=[(2, 1)],
                     hill=dict(kind="gauss", hc=300.0, half_width=800.0, xc=3e3), atmosphere=STRAT)
    dg = DG(case)
    st = Stepper(dg)
    U = dg.state("inflow")
    m0 = dg.conservation(U)[0]
    for _ in range(3):
        U = st.step(U, case.dt)
    assert abs(dg.conservation(U)[0] - m0) < 1e-14 * m0


def test_second_order_in_time():
    """Warm bubble on a fixed mesh over four case steps: the error against a run
    with 256 steps shrinks by ~4 per halving of dt once dt is below the case's
    acoustic-Courant-1 step (16 -> 32 steps)."""
    case = make_case("bubble2d", 0, degree=2, base=(8, 4))
    dg = DG(case)
    U0 = dg.state()
    T = 4 * case.dt

    def run(n):
        st = Stepper(dg, picard=3, tol=1e-14)
        U = U0.copy()
        for _ in range(n):
            U = st.step(U, T / n)
        return U

    ref = run(256)
    e16 = np.abs(run(16) - ref).max(axis=(1, 2))
    e32 = np.abs(run(32) - ref).max(axis=(1, 2))
    orders = np.log2(e16 / e32)
    assert np.all(orders > 1.8) and np.all(orders < 2.4), orders
