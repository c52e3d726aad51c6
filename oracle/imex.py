"""IMEX-RK2 time step with a pressure fixed-point loop and GMRES (test oracle).

Sec. 2: continuity is explicit, energy and momentum are coupled implicitly
(the pressure terms are stiff at low Mach number), with a second-order
IMEX Runge-Kutta method.  Sec. 3.2: each implicit stage runs a fixed-point
loop on the pressure in which GMRES solves a non-symmetric linear system.

Readings (the paper cites the method only):

* Tableau: ARK2(2,3,2) of Giraldo, Kelly and Constantinescu (2013),
  gamma = 1 - 1/sqrt(2), delta = 1/(2 sqrt(2)), a32 = (3 + 2 sqrt(2)) / 6,
  explicit A = [[0,0,0],[2 gamma,0,0],[1-a32,a32,0]],
  implicit At = [[0,0,0],[gamma,gamma,0],[delta,delta,gamma]],
  b = (delta, delta, gamma).  The implicit tableau is stiffly accurate, so
  the step result is the last stage plus the explicit correction
  dt sum_j (b_j - A[2, j]) E_j.
* Implicit terms: momentum -grad p' - rho' g k, energy -div(h m) with the
  specific enthalpy h = gamma p / ((gamma-1) rho).  Substituting the
  momentum stage equation into the energy one gives the Helmholtz problem
  p'/(gamma-1) - (dt at_ii)^2 div_h(h grad_h p') = rhs, with h and the
  kinetic energy lagged by the fixed-point loop.
* A Rayleigh damping layer below the top (a reading; see DG.damping) is an
  explicit source, added to the explicit tendencies.
* GMRES(m) with classical Gram-Schmidt applied twice, Givens rotations,
  relative tolerance on ||b - A x|| / ||b||, previous iterate as initial guess.
"""

import math

import numpy as np

from . import physics as ph

SQ2 = math.sqrt(2.0)
G_ = 1.0 - 1.0 / SQ2
D_ = 1.0 / (2.0 * SQ2)
A32 = (3.0 + 2.0 * SQ2) / 6.0
A_EX = np.array([[0.0, 0.0, 0.0], [2.0 * G_, 0.0, 0.0], [1.0 - A32, A32, 0.0]])
A_IM = np.array([[0.0, 0.0, 0.0], [G_, G_, 0.0], [D_, D_, G_]])
B = np.array([D_, D_, G_])


def gmres(apply, b, x0, tol, restart=30, max_iter=2000):
    """Restarted GMRES; returns (x, iterations, relative residual estimate)."""
    bnorm = float(np.linalg.norm(b))
    x = x0.copy()
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0
    it = 0
    rel = 1.0
    while it < max_iter:
        r = b - apply(x)
        beta = float(np.linalg.norm(r))
        rel = beta / bnorm
        if rel <= tol:
            break
        m = restart
        Q = np.zeros((m + 1,) + b.shape)
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        Q[0] = r / beta
        k_done = 0
        for k in range(m):
            w = apply(Q[k])
            # classical Gram-Schmidt, twice
            h = np.array([np.vdot(Q[j], w) for j in range(k + 1)])
            w = w - np.tensordot(h, Q[: k + 1], axes=1)
            h2 = np.array([np.vdot(Q[j], w) for j in range(k + 1)])
            w = w - np.tensordot(h2, Q[: k + 1], axes=1)
            h = h + h2
            hn = float(np.linalg.norm(w))
            H[: k + 1, k] = h
            H[k + 1, k] = hn
            if hn > 0.0:
                Q[k + 1] = w / hn
            # apply previous rotations, then a new one zeroing H[k+1, k]
            for j in range(k):
                t = cs[j] * H[j, k] + sn[j] * H[j + 1, k]
                H[j + 1, k] = -sn[j] * H[j, k] + cs[j] * H[j + 1, k]
                H[j, k] = t
            den = math.hypot(H[k, k], H[k + 1, k])
            cs[k], sn[k] = H[k, k] / den, H[k + 1, k] / den
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            it += 1
            k_done = k + 1
            rel = abs(g[k + 1]) / bnorm
            if rel <= tol or it >= max_iter or hn == 0.0:
                break
        y = np.linalg.solve(np.triu(H[:k_done, :k_done]), g[:k_done])
        x = x + np.tensordot(y, Q[:k_done], axes=1)
        if rel <= tol:
            break
    return x, it, rel


class Stepper:
    """IMEX-RK2 integrator of one oracle discretisation."""

    def __init__(self, dg, picard=3, tol=1e-12, restart=30, max_iter=5000):
        self.dg = dg
        self.picard = picard
        self.tol = tol
        self.restart = restart
        self.max_iter = max_iter
        self.iters = []

    def implicit_terms(self, U, pprime, h):
        """dU/dt of the implicit terms: (0, -grad p' - rho' g k, -div(h m))."""
        dg, d = self.dg, self.dg.d
        I = np.zeros_like(U)
        I[1:1 + d] = -dg.grad(pprime)
        I[d] -= (U[0] - dg.rhobar) * dg.g
        I[1 + d] = -dg.div(h[None] * U[1:1 + d])
        return I

    def step(self, U, dt):
        dg, d = self.dg, self.dg.d
        gm1 = ph.GAMMA - 1.0
        # the damping layer (if any) is an explicit source
        E = [dg.explicit(U, "imex") + dg.damping(U)]
        p0 = dg.pprime(U)
        I = [self.implicit_terms(U, p0, dg.enthalpy(U))]
        p_prev = p0
        Ui = U
        for i in (1, 2):
            aii = A_IM[i, i]
            ex = sum(A_EX[i, j] * E[j] for j in range(i))
            im = sum(A_IM[i, j] * I[j] for j in range(i))
            rho = U[0] + dt * ex[0]
            mhat = U[1:1 + d] + dt * (ex[1:1 + d] + im[1:1 + d])
            mhat[d - 1] -= dt * aii * (rho - dg.rhobar) * dg.g
            Ehat = U[1 + d] + dt * (ex[1 + d] + im[1 + d])
            alpha = (dt * aii) ** 2
            p = p_prev
            mk = mhat
            for _ in range(self.picard):
                h = ph.GAMMA * (dg.pbar + p) / (gm1 * rho)
                kin = 0.5 * np.sum(mk * mk, axis=0) / rho ** 2
                rhs = Ehat - dg.pbar / gm1 - rho * kin - dt * aii * dg.div(h[None] * mhat)
                p, its, _ = gmres(lambda q: dg.helmholtz(q, h, alpha), rhs, p, self.tol, self.restart, self.max_iter)
                self.iters.append(its)
                gp = dg.grad(p)
                mk = mhat - dt * aii * gp
            Ui = np.empty_like(U)
            Ui[0] = rho
            Ui[1:1 + d] = mk
            Ui[1 + d] = (dg.pbar + p) / gm1 + 0.5 * np.sum(mk * mk, axis=0) / rho
            E.append(dg.explicit(Ui, "imex") + dg.damping(Ui))
            if i == 1:
                Ii = np.zeros_like(U)
                Ii[1:1 + d] = -gp
                Ii[d] -= (rho - dg.rhobar) * dg.g
                Ii[1 + d] = -dg.div(h[None] * mk)
                I.append(Ii)
            p_prev = p
        return Ui + dt * sum((B[j] - A_EX[2, j]) * E[j] for j in range(3))
