"""Pins of the oracle's Euler flux (Eq. (1), Sec. 2) and of the Rusanov speed (no GPU).

The free stream, the hydrostatic rest state and energy conservation hold for
any flux form, so they cannot tell a correct energy or momentum flux from a
wrong one.  These checks can:

1. Smooth polynomial states on affine meshes: every variable's residual equals
   the analytic -div F + S, with the divergence worked out by hand from the
   product rule on Eq. (1) (uniform density, linear velocity and pressure), not
   from the oracle's flux function.  The fluxes are then polynomials of degree
   3, which the DG operator differentiates exactly.
2. The Rusanov speed equals the spectral radius of the flux Jacobian
   d(F.n)/dU, taken by central differences of the oracle's flux, and the
   Jacobian's eigenvalues are the characteristic speeds of the Euler system,
   u.n (d times) and u.n -/+ c.  For the IMEX-explicit flux (continuity,
   advection, kinetic-energy flux) every eigenvalue is u.n.
3. Two constant states meeting at one face: the residual at the face nodes is
   the Rusanov flux of the two states through the face, and zero elsewhere.

Mistakes are planted in copies of the oracle's functions, on the CPU, to show
that each check fails for the slip it guards against.
"""

import numpy as np
import pytest

from oracle import physics as ph
from oracle.dg import DG
from workloads import tiny_case

GAM = 1.4
GRAV = 9.81


# ---------------------------------------------------------------- 1. exact divergence


def _affine_case(dim, r, refined):
    base = (4, 4) if dim == 2 else (4, 4, 4)
    ext = (4e3, 4e3) if dim == 2 else (4e3,) * 3
    return tiny_case(dim, r, base=base, extent=ext, refine=[(1, 1, 1)[:dim]] if refined else [],
                     periodic=(False,) * dim, atmosphere=dict(kind="none"))


def _linear_fields(X, dim):
    """rho0, velocity u = u0 + A x, pressure p = p0 + b.x (x relative to the domain's corner)."""
    rho0 = 1.1
    u0 = np.array([12.0, -4.0, 3.0])[:dim]
    A = np.array([[2.0, -1.0, 0.7], [0.5, 1.5, -0.8], [-1.2, 0.9, -2.5]])[:dim, :dim] / 1e3 * 3.0
    p0 = 9.5e4
    b = np.array([2.0, -3.5, 1.5])[:dim]
    x = np.stack([X[a] for a in range(dim)])  # (d, K, Nc)
    u = u0[:, None, None] + np.einsum("ab,bkq->akq", A, x)
    p = p0 + np.einsum("b,bkq->kq", b, x)
    return rho0, u, p, A, b


def _state(rho0, u, p, dim):
    U = np.zeros((dim + 2,) + p.shape)
    U[0] = rho0
    U[1:1 + dim] = rho0 * u
    U[dim + 1] = p / (GAM - 1.0) + 0.5 * rho0 * np.sum(u * u, axis=0)
    return U


def _exact_residual(rho0, u, p, A, b, dim, terms, g):
    """-div F + S of Eq. (1) by the product rule, for uniform rho, u = u0 + A x, p = p0 + b.x.

    div u = tr A, d u_a / d x_b = A[a, b], grad(|u|^2 / 2) = A^T u.
      continuity   div(rho u)            = rho tr A
      momentum a   div(rho u_a u) + d_a p = rho ((A u)_a + u_a tr A) + b_a      (p only if full)
      energy       div((rho E + p) u)    = u.grad(rho E + p) + (rho E + p) tr A,
                   grad(rho E + p)       = gamma/(gamma-1) b + rho A^T u
      IMEX energy  div(k rho u)          = rho (u.grad k + k tr A), k = |u|^2/2
      sources      momentum z: -rho g (full); energy: -g rho w (both)
    """
    trA = np.trace(A)
    Au = np.einsum("ab,bkq->akq", A, u)
    ATu = np.einsum("ba,bkq->akq", A, u)
    k = 0.5 * np.sum(u * u, axis=0)
    R = np.zeros((dim + 2,) + p.shape)
    R[0] = -rho0 * trA
    for a in range(dim):
        R[1 + a] = -rho0 * (Au[a] + u[a] * trA)
        if terms == "full":
            R[1 + a] -= b[a]
    if terms == "full":
        H = GAM / (GAM - 1.0) * p + rho0 * k  # rho E + p
        gradH = GAM / (GAM - 1.0) * b[:, None, None] + rho0 * ATu
        R[dim + 1] = -(np.sum(u * gradH, axis=0) + H * trA)
        R[dim] -= rho0 * g
    else:
        R[dim + 1] = -rho0 * (np.sum(u * ATu, axis=0) + k * trA)
    R[dim + 1] -= g * rho0 * u[dim - 1]
    return R


def _divergence_errors(dim, r, refined, terms):
    """Per-variable max |R - exact| over cells that touch no wall, relative to the scale of one
    discrete derivative of that variable's flux, max |F_v| / h (h the smallest cell edge), with
    |F_v| bounded by hand: rho |u| (mass), p + rho |u|^2 (momentum), (rho E + p) |u| (energy).
    Rounding leaves a few 1e-13 of that scale; each planted mistake below leaves 1e-4 or more."""
    case = _affine_case(dim, r, refined)
    dg = DG(case, gravity=GRAV)
    X = dg.mesh.X
    rho0, u, p, A, b = _linear_fields(X, dim)
    U = _state(rho0, u, p, dim)
    R = dg.explicit(U, terms)
    exact = _exact_residual(rho0, u, p, A, b, dim, terms, GRAV)
    wall = {c for c, _ in dg.mesh.walls}
    inner = [k for k in range(dg.mesh.K) if k not in wall]
    assert len(inner) > 0
    if refined:  # the coarse side of a 2:1 face must be among the checked cells
        assert any(s[2] in inner for s in dg.mesh.subs) and any(s[0] in inner for s in dg.mesh.subs)
    speed = np.sqrt(np.sum(u * u, axis=0))
    flux = [rho0 * speed] + [p + rho0 * speed ** 2] * dim + [(GAM / (GAM - 1.0) * p + 0.5 * rho0 * speed ** 2) * speed]
    h = case.min_edge()
    return [float(np.abs(R[v][inner] - exact[v][inner]).max() / (np.abs(flux[v]).max() / h))
            for v in range(dim + 2)]


# degree r conforming; degree r-1 across 2:1 faces (collocated subface quadrature), so r = 4 there
DIV_CASES = [(2, 3, False), (2, 4, True), (3, 3, False), (3, 4, True)]


@pytest.mark.parametrize("dim,r,refined", DIV_CASES)
@pytest.mark.parametrize("terms", ["full", "imex"])
def test_every_variable_residual_is_exact_divergence(dim, r, refined, terms):
    errs = _divergence_errors(dim, r, refined, terms)
    assert max(errs) < 1e-12, errs


def _mutant_flux(kind):
    base = ph.physical_flux

    def flux(U, pbar, d, terms):
        F = base(U, pbar, d, terms)
        rho, m, E = ph.split(U, d)
        u = m / rho
        if kind == "energy_without_p" and terms == "full":
            for b in range(d):
                F[1 + d, b] = E * u[b]  # E u written for (E + p) u
        elif kind == "momentum_without_1_over_rho":
            for a in range(d):
                for b in range(d):
                    F[1 + a, b] += m[a] * m[b] - m[a] * u[b]
        elif kind == "momentum_without_pressure" and terms == "full":
            p = ph.pressure(U, d)
            for a in range(d):
                F[1 + a, a] -= p - pbar
        elif kind == "kinetic_flux_without_half" and terms == "imex":
            for b in range(d):
                F[1 + d, b] *= 2.0
        return F

    return flux


@pytest.mark.parametrize("kind,terms,var", [
    ("energy_without_p", "full", "energy"),
    ("momentum_without_1_over_rho", "full", "momentum"),
    ("momentum_without_1_over_rho", "imex", "momentum"),
    ("momentum_without_pressure", "full", "momentum"),
    ("kinetic_flux_without_half", "imex", "energy"),
])
def test_divergence_pin_catches_planted_flux_mistakes(monkeypatch, kind, terms, var):
    monkeypatch.setattr(ph, "physical_flux", _mutant_flux(kind))
    errs = _divergence_errors(2, 3, False, terms)
    rows = [1, 2] if var == "momentum" else [3]
    assert max(errs[v] for v in rows) > 1e-6, errs


def test_divergence_pin_catches_planted_source_mistake(monkeypatch):
    base = ph.source

    def source(U, rhobar, d, terms, g):
        S = base(U, rhobar, d, terms, g)
        S[1 + d] = -S[1 + d]  # energy source -g m_z with the wrong sign
        return S

    monkeypatch.setattr(ph, "source", source)
    assert _divergence_errors(2, 3, False, "full")[3] > 1e-6


# ---------------------------------------------------------------- 2. Rusanov speed


def _random_states(d, n, seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.5, 1.5, n)
    u = rng.normal(0.0, 40.0, (d, n))
    p = rng.uniform(5e4, 1.2e5, n)
    U = np.zeros((d + 2, n))
    U[0] = rho
    U[1:1 + d] = rho * u
    U[d + 1] = p / (GAM - 1.0) + 0.5 * rho * np.sum(u * u, axis=0)
    nv = rng.normal(size=(d, n))
    nv /= np.linalg.norm(nv, axis=0)
    return U, u, p, rho, nv


def _jacobian_eigs(flux, U, nv, d, terms, j):
    """Eigenvalues of d(F.n)/dU at state j by central differences of the flux."""
    V = d + 2
    Jm = np.zeros((V, V))
    pb = np.zeros(1)
    for c in range(V):
        hstep = 1e-6 * max(abs(U[c, j]), 1.0)
        Up = U[:, j:j + 1].copy()
        Um = U[:, j:j + 1].copy()
        Up[c] += hstep
        Um[c] -= hstep
        Fp = np.sum(flux(Up, pb, d, terms) * nv[None, :, j:j + 1], axis=1)[:, 0]
        Fm = np.sum(flux(Um, pb, d, terms) * nv[None, :, j:j + 1], axis=1)[:, 0]
        Jm[:, c] = (Fp - Fm) / (2.0 * hstep)
    return np.linalg.eigvals(Jm)


def _speed_errors(flux, speed, d, terms, n=24, seed=2):
    """Largest relative mismatch of (eigenvalues vs characteristic speeds, speed vs spectral radius)."""
    U, u, p, rho, nv = _random_states(d, n, seed)
    un = np.sum(u * nv, axis=0)
    c = np.sqrt(GAM * p / rho)
    lam = speed(U, nv, d, terms)
    e_eig, e_rad = 0.0, 0.0
    for j in range(n):
        ev = _jacobian_eigs(flux, U, nv, d, terms, j)
        if terms == "full":
            expect = np.sort(np.r_[[un[j]] * d, un[j] - c[j], un[j] + c[j]])
        else:  # rho E enters no IMEX-explicit flux: eigenvalue 0, and u.n (d+1 times, defective)
            expect = np.sort(np.r_[[un[j]] * (d + 1), 0.0])
        scale = abs(un[j]) + c[j]
        e_eig = max(e_eig, np.abs(np.sort(ev.real) - expect).max() / scale, np.abs(ev.imag).max() / scale)
        e_rad = max(e_rad, abs(lam[j] - np.abs(ev).max()) / scale)
    return e_eig, e_rad


@pytest.mark.parametrize("d", [2, 3])
def test_rusanov_speed_is_spectral_radius_of_flux_jacobian(d):
    e_eig, e_rad = _speed_errors(ph.physical_flux, ph.wave_speed, d, "full")
    assert e_eig < 1e-6 and e_rad < 1e-6, (e_eig, e_rad)


@pytest.mark.parametrize("d", [2, 3])
def test_imex_speed_is_advective_speed(d):
    # The IMEX-explicit flux (no pressure) has the eigenvalues u.n, d+1 times in one Jordan
    # block, and 0 (no flux depends on rho E); the spectral radius is |u.n|.  The defective
    # eigenvalue of the finite-difference Jacobian scatters by about (1e-10)^(1/(d+1)).
    e_eig, e_rad = _speed_errors(ph.physical_flux, ph.wave_speed, d, "imex")
    assert e_eig < 2e-2 and e_rad < 2e-2, (e_eig, e_rad)


def test_speed_pin_catches_planted_mistakes():
    def speed_c2(U, n, d, terms):  # c^2 written for c
        rho, m, E = ph.split(U, d)
        return np.abs(np.sum(m * n, axis=0) / rho) + GAM * ph.pressure(U, d) / rho

    def speed_no_advection(U, n, d, terms):  # |u.n| dropped
        return np.sqrt(GAM * ph.pressure(U, d) / U[0])

    assert _speed_errors(ph.physical_flux, speed_c2, 2, "full")[1] > 1e-2
    assert _speed_errors(ph.physical_flux, speed_no_advection, 2, "full")[1] > 1e-2
    # a wrong energy flux moves the acoustic eigenvalues off u.n -/+ c
    assert _speed_errors(_mutant_flux("energy_without_p"), ph.wave_speed, 2, "full")[0] > 1e-2


# ---------------------------------------------------------------- 3. two-state jump


def _euler_normal_flux(rho, u, p, n, terms):
    """F(U).n of Eq. (1) from primitive variables (no reference state)."""
    un = float(u @ n)
    k = 0.5 * float(u @ u)
    if terms == "full":
        E = p / (GAM - 1.0) + rho * k
        return np.r_[rho * un, rho * u * un + p * n, (E + p) * un]
    return np.r_[rho * un, rho * u * un, rho * k * un]


def _conserved(rho, u, p):
    return np.r_[rho, rho * u, p / (GAM - 1.0) + 0.5 * rho * float(u @ u)]


@pytest.mark.parametrize("terms", ["full", "imex"])
def test_two_state_jump_gives_rusanov_flux(terms):
    """Left column of cells in state L, right column in state R, periodic in x and z, g = 0.

    Volume terms of a constant state vanish except at face nodes; along z the
    columns are uniform, so only the x-faces carry a jump.  For a face node of
    a cell of width hx, with outward normal n, the residual is
    2/(w_end hx) (F_own.n - F*(U_own, U_other, n)) with the Rusanov flux
    F* = 1/2 (F_own + F_other).n - 1/2 lam (U_other - U_own),
    lam = max(|u.n| + c) (full) or max |u.n| (IMEX-explicit terms).
    """
    r = 2
    ext = (2e3, 2e3)
    case = tiny_case(2, r, base=(2, 2), extent=ext, refine=[], periodic=(True, True), atmosphere=dict(kind="none"))
    dg = DG(case, gravity=0.0)
    m = dg.mesh
    states = {0: (1.2, np.array([15.0, 4.0]), 1.0e5), 1: (0.9, np.array([-6.0, -9.0]), 0.8e5)}
    U = np.zeros((4, m.K, m.nc))
    col = np.array([int(case.ijk[c, 0]) for c in range(m.K)])
    for c in range(m.K):
        U[:, c, :] = _conserved(*states[col[c]])[:, None]
    R = dg.explicit(U, terms)
    hx = ext[0] / 2
    w_end = 1.0 / 3.0  # GLL weight of an end node for r = 2
    i0 = m.mi[:, 0]
    for c in range(m.K):
        own, other = states[col[c]], states[1 - col[c]]
        for q in range(m.nc):
            if i0[q] not in (0, r):
                expect = np.zeros(4)
            else:
                n = np.array([1.0, 0.0]) if i0[q] == r else np.array([-1.0, 0.0])
                Fo = _euler_normal_flux(*own, n, terms)
                Ft = _euler_normal_flux(*other, n, terms)
                sp = [abs(float(s[1] @ n)) + (np.sqrt(GAM * s[2] / s[0]) if terms == "full" else 0.0)
                      for s in (own, other)]
                Fs = 0.5 * (Fo + Ft) - 0.5 * max(sp) * (_conserved(*other) - _conserved(*own))
                expect = 2.0 / (w_end * hx) * (Fo - Fs)
            scale = np.abs(expect).max() if np.abs(expect).max() > 0 else 1.0
            assert np.abs(R[:, c, q] - expect).max() <= 1e-12 * max(scale, 1e3), (c, q, R[:, c, q], expect)
