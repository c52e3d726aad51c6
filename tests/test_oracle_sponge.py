"""Oracle pins of the Rayleigh damping layer below the top boundary.

The layer is a reading (the paper's non-reflecting boundaries are described
elsewhere): a source -tau(z) (U - U_ref) in the top `depth` metres, tau rising
as sin^2 from 0 to `rate`, added to the explicit tendencies.  The pins use
properties that do not restate that formula: where the layer is the only
process acting, each node's perturbation is multiplied per step by the
stability function of the explicit tableau, R(z) = 1 + z b^T (I - z A)^-1 1,
at z = -tau dt, with tau = 0 below the layer, the full rate at the top and half
of it at mid-depth (sin^2(pi/4) = 1/2); and the reference state is a steady
state.
"""

import dataclasses

import numpy as np

from oracle.dg import DG
from oracle.imex import A_EX, B, Stepper
from workloads.cases import tiny_case

STRAT = dict(kind="stratified", N=0.01, T_ref=293.15, p_ref=1e5)


def _stability(z):
    return 1.0 + z * (B @ np.linalg.solve(np.eye(3) - z * A_EX, np.ones(3)))


def test_stability_function_of_the_tableau():
    # second order: R(z) = 1 + z + z^2/2 + O(z^3)
    for z in (-1e-2, -1e-3):
        assert abs(_stability(z) - (1 + z + z * z / 2)) < 2 * abs(z) ** 3


def test_layer_alone_damps_a_density_perturbation_by_the_explicit_stability_function():
    """Flat ground, g = 0, the background at rest plus a random density perturbation: mass, momentum
    and energy fluxes all vanish (no velocity, p' = 0), so only the layer acts, node by node."""
    case = tiny_case(2, 3, base=(3, 4), extent=(3e3, 4e3), refine=[(1, 1)], atmosphere=STRAT)
    rate, dt = 0.05, 2.0
    case = dataclasses.replace(case, sponge=dict(depth=2e3, rate=rate))
    dg = DG(case, gravity=0.0)
    rng = np.random.default_rng(0)
    U0 = dg.Ubg.copy()
    drho = 1e-3 * dg.rhobar * (1.0 + rng.random(dg.rhobar.shape))
    U0[0] += drho
    U1 = Stepper(dg, tol=1e-13).step(U0, dt)
    ratio = (U1[0] - dg.rhobar) / drho
    z = dg.mesh.X[-1]
    below = z <= 2e3 + 1e-6
    top = np.abs(z - 4e3) < 1e-6
    mid = np.abs(z - 3e3) < 1e-6
    assert below.any() and top.any() and mid.any()
    assert np.abs(ratio[below] - 1.0).max() < 1e-12
    assert np.abs(ratio[top] - _stability(-rate * dt)).max() < 1e-12
    assert np.abs(ratio[mid] - _stability(-0.5 * rate * dt)).max() < 1e-12
    # in between: between R(-rate dt) and 1, and higher nodes are damped at least as much
    assert np.all(ratio <= 1.0 + 1e-12) and np.all(ratio >= _stability(-rate * dt) - 1e-12)
    order = np.argsort(z.ravel())
    assert np.all(np.diff(ratio.ravel()[order]) <= 1e-12)
    # nothing else moves
    assert np.abs(U1[1:3]).max() < 1e-9
    assert np.abs(U1[3] - U0[3]).max() < 1e-6


def test_reference_state_is_steady():
    """Flat ground, gravity on, the hydrostatic background carrying the reference inflow u0 on a
    conforming mesh: the damping vanishes on it and the discrete operator keeps it, so a step
    leaves it unchanged.  (Across 2:1 faces the coarse polynomial of rho_bar u0 differs from the
    fine nodes' values by the interpolation error, a discretisation effect of order 1e-7 here.)"""
    u0 = 10.0
    case = tiny_case(2, 3, base=(4, 4), extent=(4e3, 4e3), refine=(), atmosphere=STRAT)
    case = dataclasses.replace(case, sponge=dict(depth=1.5e3, rate=0.1, u0=u0))
    dg = DG(case)
    U = dg.Ubg.copy()
    U[1] = dg.rhobar * u0
    U[3] += 0.5 * dg.rhobar * u0 * u0
    assert np.abs(dg.damping(U)).max() == 0.0
    U1 = Stepper(dg, tol=1e-13).step(U, 1.0)
    scale = [np.abs(U[0]).max(), np.abs(U[1]).max(), np.abs(U[1]).max(), np.abs(U[3]).max()]
    for v in range(4):
        assert np.abs(U1[v] - U[v]).max() <= 1e-12 * scale[v], v


def test_no_layer_no_change():
    case = tiny_case(2, 2, atmosphere=STRAT)
    assert DG(case).tau is None
    off = dataclasses.replace(case, sponge=dict(depth=0.0, rate=1.0))
    assert DG(off).tau is None


def test_lateral_layer_damps_by_distance_to_the_lateral_boundaries():
    """Lateral layers alone (no top layer), flat ground, g = 0, the background at rest plus a density
    perturbation: each node's perturbation is multiplied per step by R(-tau dt), tau = the rate on
    the lateral boundaries, half of it at half the width in from them, and nothing beyond the width
    (2D: x only; 3D: the nearer of the x and y boundaries)."""
    for dim in (2, 3):
        base = (4, 3) if dim == 2 else (4, 4, 2)
        ext = (4e3, 3e3) if dim == 2 else (4e3, 4e3, 2e3)
        case = tiny_case(dim, 2, base=base, extent=ext, refine=[], atmosphere=STRAT,
                         periodic=(True,) * (dim - 1) + (False,))
        rate, dt, w = 0.05, 2.0, 1e3
        case = dataclasses.replace(case, sponge=dict(lateral_width=w, lateral_rate=rate))
        dg = DG(case, gravity=0.0)
        U0 = dg.Ubg.copy()
        drho = 1e-3 * dg.rhobar
        U0[0] += drho
        U1 = Stepper(dg, tol=1e-13).step(U0, dt)
        ratio = (U1[0] - dg.rhobar) / drho
        X = dg.mesh.X
        dist = np.min([np.minimum(X[a], ext[a] - X[a]) for a in range(dim - 1)], axis=0)
        edge = np.abs(dist) < 1e-6
        half = np.abs(dist - 0.5 * w) < 1e-6
        inner = dist >= w - 1e-6
        assert edge.any() and half.any() and inner.any()
        assert np.abs(ratio[edge] - _stability(-rate * dt)).max() < 1e-12
        assert np.abs(ratio[half] - _stability(-0.5 * rate * dt)).max() < 1e-12
        assert np.abs(ratio[inner] - 1.0).max() < 1e-12
