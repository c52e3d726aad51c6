"""Pins of the oracle's DG operators against invariants and exact calculus (no GPU).

Each check is chosen so that a plausible slip in the oracle (a flipped face
sign, a transposed derivative matrix, a wrong subface index or normal, a
dropped source or metric term) breaks at least one of them.
"""

import numpy as np
import pytest

from oracle import physics as ph
from oracle.dg import DG
from workloads import tiny_case

STRAT = dict(kind="stratified", N=0.01, T_ref=293.15, p_ref=1e5)


def _hill(dim, ext):
    return dict(kind="gauss", hc=300.0, half_width=700.0, xc=ext[0] / 2, yc=ext[1] / 2)


def _mid_refined(dim, r, hill=True, atm=None, periodic=None):
    base = (4, 4) if dim == 2 else (3, 3, 3)
    ext = (4e3, 4e3) if dim == 2 else (3e3, 3e3, 3e3)
    return tiny_case(
        dim, r, base=base, extent=ext, refine=[(1, 1, 1)[:dim]],
        hill=_hill(dim, ext) if hill else None, atmosphere=atm or STRAT, periodic=periodic,
    )


def _uniform_state(dg, dim):
    U = np.zeros((dg.V, dg.mesh.K, dg.mesh.nc))
    vel = np.array([10.0, -3.0, 2.0][:dim])
    U[0] = 1.2
    U[1:1 + dim] = 1.2 * vel[:, None, None]
    U[-1] = 1e5 / 0.4 + 0.5 * 1.2 * vel @ vel
    return U


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("curved", [False, True])
def test_free_stream_preserved(dim, curved):
    """g = 0, no background, uniform state: R = 0 in every cell not touching a wall."""
    case = _mid_refined(dim, 3, hill=curved, atm=dict(kind="none"))
    dg = DG(case, gravity=0.0)
    U = _uniform_state(dg, dim)
    R = dg.explicit(U, "full")
    wall = {c for c, _ in dg.mesh.walls}
    inner = [k for k in range(dg.mesh.K) if k not in wall]
    assert len(inner) > 0 and len(dg.mesh.subs) > 0
    scale = 1e5 * 10 / 250.0
    assert np.abs(R[:, inner]).max() < 1e-11 * scale


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("terms", ["full", "imex"])
def test_hydrostatic_rest_is_steady(dim, terms):
    """R(U_bg) = 0 to round-off, with curved cells and 2:1 faces (reference-state subtraction)."""
    dg = DG(_mid_refined(dim, 3))
    R = dg.explicit(dg.Ubg, terms)
    assert np.abs(R).max() < 1e-9


@pytest.mark.parametrize("dim", [2, 3])
def test_mass_and_energy_conservation(dim):
    """sum w J R_rho = 0; with g = 0 also sum w J R_E = 0 (periodic + walls + 2:1 faces)."""
    dg = DG(_mid_refined(dim, 3))
    U = dg.state("random", seed=3)
    R = dg.explicit(U, "full")
    wJ = dg.mesh.wJ
    assert abs(np.sum(wJ * R[0])) < 1e-13 * np.sum(wJ * np.abs(R[0]))
    dg0 = DG(_mid_refined(dim, 3), gravity=0.0)
    R = dg0.explicit(U, "full")
    assert abs(np.sum(wJ * R[-1])) < 1e-13 * np.sum(wJ * np.abs(R[-1]))
    # the IMEX-explicit part conserves mass too
    R = dg.explicit(U, "imex")
    assert abs(np.sum(wJ * R[0])) < 1e-13 * np.sum(wJ * np.abs(R[0]))


def _poly_momentum(X, dim, deg):
    x, z = X[0], X[-1]
    if deg >= 3:
        mx, my, mz = 1e-10 * x ** 2 * z + 1.0, 1e-10 * x * z ** 2, 2e-10 * z ** 3 - 3e-10 * x ** 3
    else:
        mx, my, mz = 1e-6 * x * z + 1.0, 1e-6 * x * z, 3e-6 * z ** 2 - 2e-6 * x ** 2
    return [mx, my, mz] if dim == 3 else [mx, mz]


def _poly_div(X, dim, deg):
    x, z = X[0], X[-1]
    if deg >= 3:
        return 2e-10 * x * z + 6e-10 * z ** 2
    return 1e-6 * z + 6e-6 * z


@pytest.mark.parametrize("dim,refined,deg", [(2, False, 3), (2, True, 2), (3, False, 3), (3, True, 2)])
def test_continuity_residual_is_minus_divergence(dim, refined, deg):
    """Uniform rho, polynomial m on an affine mesh: R_rho = -div m at every node.

    Exact for degree r on conforming meshes and degree r-1 across 2:1 faces
    (where the collocated subface quadrature sees a product of degree 2r-1).
    """
    r = 3
    case = tiny_case(
        dim, r, base=(4, 4) if dim == 2 else (3, 3, 3), extent=(4e3, 4e3) if dim == 2 else (3e3,) * 3,
        refine=[(1, 1, 1)[:dim]] if refined else [], periodic=(False,) * dim, atmosphere=dict(kind="none"),
    )
    dg = DG(case, gravity=0.0)
    X = dg.mesh.X
    U = np.zeros((dg.V, dg.mesh.K, dg.mesh.nc))
    U[0] = 1.0
    m = _poly_momentum(X, dim, deg)
    for a in range(dim):
        U[1 + a] = m[a]
    U[-1] = 2.5e5
    # walls reflect m.n, which is not zero here, so only cells away from walls are exact
    R = dg.explicit(U, "full")
    wall = {c for c, _ in dg.mesh.walls}
    inner = [k for k in range(dg.mesh.K) if k not in wall]
    exact = -_poly_div(X, dim, deg)
    assert np.abs(R[0][inner] - exact[inner]).max() < 1e-12 * np.abs(exact).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_gradient_exact_for_degree_r(dim):
    """Strong-form gradient of a degree-r polynomial is exact, also across 2:1 faces and at walls."""
    r = 3
    case = _mid_refined(dim, r, hill=False, periodic=(False,) * dim)
    dg = DG(case)
    X = dg.mesh.X
    x, z = X[0], X[-1]
    p = x ** 3 + 3 * x * z ** 2 - z ** 3 + (x * X[1] * z if dim == 3 else 0)
    g = dg.grad(p)
    ex = [3 * x ** 2 + 3 * z ** 2 + (X[1] * z if dim == 3 else 0)]
    if dim == 3:
        ex.append(x * z)
    ex.append(6 * x * z - 3 * z ** 2 + (x * X[1] if dim == 3 else 0))
    for b in range(dim):
        assert np.abs(g[b] - ex[b]).max() < 1e-12 * np.abs(ex[0]).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_divergence_exact(dim):
    """Weak-form divergence with f.n = 0 on the walls: exact for degree r-1 across 2:1 faces."""
    r = 3
    case = _mid_refined(dim, r, hill=False, periodic=(False,) * dim)
    dg = DG(case)
    X = dg.mesh.X
    f = np.zeros((dim,) + X[0].shape)
    ext = case.extent
    f[0] = X[0] * (ext[0] - X[0])
    f[-1] = X[-1] * (ext[-1] - X[-1])
    dv = dg.div(f)
    exact = ext[0] - 2 * X[0] + ext[-1] - 2 * X[-1]
    assert np.abs(dv - exact).max() < 1e-12 * np.abs(exact).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_helmholtz_mass_weighted_symmetric_positive(dim):
    """Dense assembly: M A is symmetric positive definite (D = -G^T) for any h > 0,
    on curved cells with 2:1 faces and walls; A itself is not symmetric."""
    case = tiny_case(dim, 2, hill=_hill(dim, (3e3, 2e3) if dim == 2 else (2e3, 2e3)), refine=[(0, 0, 0)[:dim]], atmosphere=STRAT)
    dg = DG(case)
    K, nc = dg.mesh.K, dg.mesh.nc
    N = K * nc
    h = 1e5 * (1.0 + 0.1 * np.random.default_rng(0).random((K, nc)))
    A = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        A[:, j] = dg.helmholtz(e.reshape(K, nc), h, 3.0).ravel()
    MA = dg.mesh.wJ.ravel()[:, None] * A
    assert np.abs(MA - MA.T).max() < 1e-13 * np.abs(MA).max()
    assert np.linalg.eigvalsh(0.5 * (MA + MA.T)).min() > 0
    assert np.abs(A - A.T).max() > 1e-6 * np.abs(A).max()
    # the p/(gamma-1) part alone
    assert np.allclose(np.diag(dg.helmholtz(np.eye(N)[0].reshape(K, nc), h, 0.0).ravel()[:1]), 1 / 0.4)


def test_rusanov_consistency_and_wall_flux():
    """F*(U, U) = F(U).n; the wall flux carries no mass and no energy."""
    rng = np.random.default_rng(1)
    d = 3
    U = np.zeros((5, 7))
    U[0] = 1.0 + 0.1 * rng.random(7)
    U[1:4] = rng.standard_normal((3, 7))
    U[4] = 2.5e5
    n = rng.standard_normal((3, 7))
    n /= np.linalg.norm(n, axis=0)
    pb = np.full(7, 9e4)
    for terms in ("full", "imex"):
        F = ph.physical_flux(U, pb, d, terms)
        assert np.allclose(ph.rusanov(U, U, n, pb, d, terms), np.sum(F * n[None], axis=1))
        W = ph.rusanov(U, ph.wall_ghost(U, n, d), n, pb, d, terms)
        assert np.abs(W[0]).max() < 1e-12 and np.abs(W[4]).max() < 1e-6
