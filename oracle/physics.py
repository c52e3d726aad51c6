"""Pointwise physics of Eq. (1): ideal gas, fluxes, gravity, background state (test oracle).

Conserved variables, in this order: rho, the d momentum components
(vertical last), rho E.  Pressure from the ideal-gas law with total energy
rho E = p / (gamma - 1) + rho |u|^2 / 2 (Sec. 2: rho E = rho e + rho k).
"""

import numpy as np

GRAV = 9.81  # Sec. 2
R_GAS = 287.0  # Sec. 2
GAMMA = 1.4  # Sec. 3.1


def background(atm, z):
    """Hydrostatic background (rho_bar, p_bar) at heights z.

    * ``none``: no reference state (used for free-stream checks with g = 0).
    * ``isothermal``: p = p_ref exp(-g z / (R T0)), rho = p / (R T0).
    * ``stratified``: the constant-N atmosphere of Sec. 3.1.  The printed
      pressure formula lacks a factor g in front of g/N^2 (it is not
      dimensionless as printed); with Gamma = (gamma-1)/gamma and
      rho_ref = p_ref / (R T_ref) it reads
      p = p_ref {1 - (g^2/N^2) Gamma (rho_ref/p_ref) [1 - exp(-N^2 z/g)]}^(1/Gamma),
      rho = rho_ref (p/p_ref)^(1/gamma) exp(-N^2 z / g).
    """
    z = np.asarray(z, dtype=np.float64)
    if atm["kind"] == "none":  # no reference state: p' = p, rho' = rho
        return np.zeros_like(z), np.zeros_like(z)
    if atm["kind"] == "isothermal":
        t0, pref = atm["T0"], atm["p_ref"]
        p = pref * np.exp(-GRAV * z / (R_GAS * t0))
        return p / (R_GAS * t0), p
    if atm["kind"] == "stratified":
        n2, tref, pref = atm["N"] ** 2, atm["T_ref"], atm["p_ref"]
        cap_gamma = (GAMMA - 1.0) / GAMMA
        rho_ref = pref / (R_GAS * tref)
        s = np.exp(-n2 * z / GRAV)
        p = pref * (1.0 - (GRAV ** 2 / n2) * cap_gamma * (rho_ref / pref) * (1.0 - s)) ** (1.0 / cap_gamma)
        rho = rho_ref * (p / pref) ** (1.0 / GAMMA) * s
        return rho, p
    raise ValueError(atm["kind"])


def split(U, d):
    rho = U[0]
    m = U[1:1 + d]
    E = U[1 + d]
    return rho, m, E


def pressure(U, d):
    rho, m, E = split(U, d)
    return (GAMMA - 1.0) * (E - 0.5 * np.sum(m * m, axis=0) / rho)


def physical_flux(U, pbar, d, terms):
    """Flux tensor F[v, b] of the selected terms.

    ``full``: all of Eq. (1): rho u, m u + p' I, (rho E + p) u, with the
    momentum flux written with p' = p - p_bar (reference-state subtraction;
    the matching source is -(rho - rho_bar) g k).
    ``imex``: only the terms the IMEX split keeps explicit (continuity,
    momentum advection and the kinetic-energy flux k m, k = |u|^2/2); the
    pressure gradient, buoyancy and enthalpy flux are implicit.
    """
    rho, m, E = split(U, d)
    u = m / rho
    shape = (d + 2, d) + rho.shape
    F = np.zeros(shape)
    for b in range(d):
        F[0, b] = m[b]
        for a in range(d):
            F[1 + a, b] = m[a] * u[b]
    if terms == "full":
        p = pressure(U, d)
        for a in range(d):
            F[1 + a, a] += p - pbar
        for b in range(d):
            F[1 + d, b] = (E + p) * u[b]
    elif terms == "imex":
        kin = 0.5 * np.sum(u * u, axis=0)
        for b in range(d):
            F[1 + d, b] = kin * m[b]
    else:
        raise ValueError(terms)
    return F


def source(U, rhobar, d, terms, g):
    """Gravity: momentum -(rho - rho_bar) g k (full only), energy -g m_z (both)."""
    rho, m, E = split(U, d)
    S = np.zeros_like(U)
    if terms == "full":
        S[d] = -(rho - rhobar) * g
    S[1 + d] = -g * m[d - 1]
    return S


def wave_speed(U, n, d, terms):
    """|u.n| (+ c for the full system): the Rusanov dissipation speed."""
    rho, m, E = split(U, d)
    un = np.abs(np.sum(m * n, axis=0) / rho)
    if terms == "full":
        p = pressure(U, d)
        return un + np.sqrt(GAMMA * p / rho)
    return un


def rusanov(UL, UR, n, pbar, d, terms):
    """Rusanov normal flux 1/2 (F_L + F_R).n - 1/2 lambda (U_R - U_L)."""
    FL = physical_flux(UL, pbar, d, terms)
    FR = physical_flux(UR, pbar, d, terms)
    FnL = np.sum(FL * n[None], axis=1)
    FnR = np.sum(FR * n[None], axis=1)
    lam = np.maximum(wave_speed(UL, n, d, terms), wave_speed(UR, n, d, terms))
    return 0.5 * (FnL + FnR) - 0.5 * lam[None] * (UR - UL)


def wall_ghost(U, n, d):
    """Mirror state for a slip wall: m+ = m- - 2 (m-.n) n, rho and rho E copied."""
    G = U.copy()
    mn = np.sum(U[1:1 + d] * n, axis=0)
    G[1:1 + d] = U[1:1 + d] - 2.0 * mn[None] * n
    return G
