"""Matrix-free DG operators of the IMEX-DG Euler solver, written out densely (test oracle).

Weak form per cell K and nodal test function l_i (Sec. 2: DG on
non-conforming meshes; readings: GLL collocation, Rusanov flux):

  w_i J_i dU_i/dt = sum_q w_q sum_a (d l_i/d xi^a)(q) Ft^a(U_q)
                    - sum_faces sum_f W_f |N_f| l_i(x_f) F*(U-, U+, n_f)
                    + w_i J_i S(U_i)

with the contravariant flux Ft^a = sum_b (J d xi^a/d x_b) F_b.  Element
derivatives are the dense Kronecker matrices of ``Mesh.Da``.  On a 2:1 face
the flux lives on the fine face's GLL points with the fine side's normal;
the coarse trace there is the coarse polynomial (of the perturbation about
the hydrostatic background) evaluated at those points, and the coarse
residual receives the same flux through the values of its basis functions
at those points, so the two sides exchange exactly the same flux.

The implicit operators use centred fluxes:

  grad_h p = M^-1 G p,  G_b p = w_i sum_a Ja^a_b (D_a p)_i + sum W |N| ({p} - p_own) n_b l_i
  div_h f  = M^-1 D f,  D f   = -sum_q w_q sum_a (d l_i/d xi^a) Ja^a.f + sum W |N| {f}.n l_i

(gradient in strong form, divergence in weak form, so that D = -G^T holds
exactly), with {p} = p- and {f}.n = 0 on walls, and the Helmholtz operator
of the pressure stage  A p = p/(gamma-1) - alpha div_h(h grad_h p).
"""

import numpy as np

from . import physics as ph
from .mesh import Mesh


class DG:
    """Oracle discretisation of one case: background, face tables and operators."""

    def __init__(self, case, gravity=None):
        self.case = case
        self.mesh = m = Mesh(case)
        self.d = m.d
        self.V = m.d + 2
        self.g = case.gravity if gravity is None else gravity
        z = m.X[m.d - 1]
        self.rhobar, self.pbar = ph.background(case.atmosphere, z)
        self.Ubg = np.zeros((self.V, m.K, m.nc))
        self.Ubg[0] = self.rhobar
        self.Ubg[self.V - 1] = self.pbar / (ph.GAMMA - 1.0)
        self._sponge(getattr(case, "sponge", None), z)
        self._faces()

    # ------------------------------------------------------------------ damping layer
    def _sponge(self, sp, z):
        """Rayleigh damping layers below the top boundary and along the lateral boundaries.

        The paper's runs use non-reflecting top and lateral boundaries whose
        method it defers to earlier work; this reading relaxes the state towards
        a reference state in the top ``depth`` metres of physical height, with
        the rate rising as sin^2 from 0 at z_d = H - depth to ``rate`` at the top
        (the usual profile of upper absorbing layers), and likewise within
        ``lateral_width`` metres of the lateral domain boundaries (distance to
        the nearest one, rising to ``lateral_rate`` at the boundary); where both
        act, the larger rate applies.  The reference state is the hydrostatic
        background carrying the uniform x-velocity ``u0``.
        """
        self.tau = None
        sp = sp or {}
        top = sp.get("depth", 0.0) > 0.0 and sp.get("rate", 0.0) > 0.0
        lat = sp.get("lateral_width", 0.0) > 0.0 and sp.get("lateral_rate", 0.0) > 0.0
        if not (top or lat):
            return
        tau = np.zeros_like(z)
        if top:
            depth, rate = sp["depth"], sp["rate"]
            H = self.case.extent[self.d - 1]
            frac = np.clip((z - (H - depth)) / depth, 0.0, 1.0)
            tau = rate * np.sin(0.5 * np.pi * frac) ** 2
        if lat:
            w, rate_l = sp["lateral_width"], sp["lateral_rate"]
            X = self.mesh.X
            dist = np.full_like(z, np.inf)
            for a in range(self.d - 1):
                dist = np.minimum(dist, np.minimum(X[a], self.case.extent[a] - X[a]))
            frac = np.clip((w - np.maximum(dist, 0.0)) / w, 0.0, 1.0)
            tau = np.maximum(tau, rate_l * np.sin(0.5 * np.pi * frac) ** 2)
        self.tau = tau
        u0 = sp.get("u0", 0.0)
        self.Uref = self.Ubg.copy()
        self.Uref[1] = self.rhobar * u0
        self.Uref[self.V - 1] = self.pbar / (ph.GAMMA - 1.0) + 0.5 * self.rhobar * u0 * u0

    def damping(self, U):
        """Tendency of the damping layer, -tau (U - U_ref) (zero without a layer)."""
        if self.tau is None:
            return np.zeros_like(U)
        return -self.tau[None] * (U - self.Uref)

    # ------------------------------------------------------------------ tables
    def _faces(self):
        m = self.mesh
        fn = [m.face_nodes(lf) for lf in range(2 * m.d)]
        fw = [m.face_weights(lf) for lf in range(2 * m.d)]
        if m.conf:
            cm, lfm, cp, lfp = (np.array(v) for v in zip(*m.conf))
            self.cf_m, self.cf_p = cm, cp
            self.cf_fm = np.array([fn[l] for l in lfm])
            self.cf_fp = np.array([fn[l] for l in lfp])
            self.cf_W = np.array([fw[l] for l in lfm])
            self.cf_N = np.stack([m.face_normal(c, l) for c, l in zip(cm, lfm)], axis=1)  # (d, F, NF)
        else:
            self.cf_m = np.zeros(0, int)
        if m.walls:
            c, lf = (np.array(v) for v in zip(*m.walls))
            self.w_c = c
            self.w_f = np.array([fn[l] for l in lf])
            self.w_W = np.array([fw[l] for l in lf])
            self.w_N = np.stack([m.face_normal(cc, l) for cc, l in zip(c, lf)], axis=1)
        else:
            self.w_c = np.zeros(0, int)
        if m.subs:
            self.s_f = np.array([s[0] for s in m.subs])
            self.s_c = np.array([s[2] for s in m.subs])
            self.s_ff = np.array([fn[s[1]] for s in m.subs])
            self.s_W = np.array([fw[s[1]] for s in m.subs])
            self.s_N = np.stack([m.face_normal(s[0], s[1]) for s in m.subs], axis=1)
            self.s_L = np.array([m.subface_eval(s[1], s[3], s[4]) for s in m.subs])  # (F, NF, Nc)
        else:
            self.s_f = np.zeros(0, int)

    @staticmethod
    def _unit(N):
        nrm = np.sqrt(np.sum(N * N, axis=0))
        return N / nrm[None], nrm

    def _volume(self, Fb, sign):
        """sign * sum_q w_q sum_a D_a[q, i] (sum_b Ja^a_b F_b)_q for F of shape (V, d, K, Nc)."""
        m = self.mesh
        V = Fb.shape[0]
        out = np.zeros((V, m.K, m.nc))
        for a in range(m.d):
            Ft = np.einsum("bkq,vbkq->vkq", m.Ja[a], Fb)
            out += (Ft.reshape(V * m.K, m.nc) @ (m.Da[a] * m.w[:, None])).reshape(V, m.K, m.nc)
        return sign * out

    @staticmethod
    def _scatter(out, cells, nodes, vals):
        for v in range(out.shape[0]):
            np.add.at(out[v], (cells[:, None], nodes), vals[v])

    def _scatter_coarse(self, out, vals):
        contrib = np.einsum("fkj,vfk->vfj", self.s_L, vals)
        for v in range(out.shape[0]):
            np.add.at(out[v], self.s_c, contrib[v])

    def coarse_trace(self, X, with_background):
        """Coarse polynomial at the fine face points of every subface."""
        Xc = X[:, self.s_c]
        if with_background:
            Xc = Xc - self.Ubg[:, self.s_c]
        T = np.einsum("fkj,vfj->vfk", self.s_L, Xc)
        if with_background:
            T = T + self.Ubg[:, self.s_f[:, None], self.s_ff]
        return T

    # ------------------------------------------------------------------ explicit
    def explicit(self, U, terms="full"):
        """dU/dt of the selected terms ('full' Euler or the IMEX-explicit part)."""
        m, d = self.mesh, self.d
        F = ph.physical_flux(U, self.pbar, d, terms)
        vol = self._volume(F, +1.0)
        if len(self.cf_m):
            UL = U[:, self.cf_m[:, None], self.cf_fm]
            UR = U[:, self.cf_p[:, None], self.cf_fp]
            n, nrm = self._unit(self.cf_N)
            pb = self.pbar[self.cf_m[:, None], self.cf_fm]
            Fs = ph.rusanov(UL, UR, n, pb, d, terms) * (self.cf_W * nrm)[None]
            self._scatter(vol, self.cf_m, self.cf_fm, -Fs)
            self._scatter(vol, self.cf_p, self.cf_fp, Fs)
        if len(self.w_c):
            UL = U[:, self.w_c[:, None], self.w_f]
            n, nrm = self._unit(self.w_N)
            pb = self.pbar[self.w_c[:, None], self.w_f]
            Fs = ph.rusanov(UL, ph.wall_ghost(UL, n, d), n, pb, d, terms) * (self.w_W * nrm)[None]
            self._scatter(vol, self.w_c, self.w_f, -Fs)
        if len(self.s_f):
            UF = U[:, self.s_f[:, None], self.s_ff]
            UC = self.coarse_trace(U, True)
            n, nrm = self._unit(self.s_N)
            pb = self.pbar[self.s_f[:, None], self.s_ff]
            Fs = ph.rusanov(UF, UC, n, pb, d, terms) * (self.s_W * nrm)[None]
            self._scatter(vol, self.s_f, self.s_ff, -Fs)
            self._scatter_coarse(vol, Fs)
        return vol / m.wJ[None] + ph.source(U, self.rhobar, d, terms, self.g)

    # ------------------------------------------------------------------ implicit pieces
    def grad(self, p):
        """Nodal DG gradient M^-1 G p in strong form; p of shape (K, Nc) -> (d, K, Nc).

        w_i J_i g_b,i = w_i sum_a Ja^a_b,i (D_a p)_i + sum_faces W |N| n_b (p^ - p_own) l_i
        with the centred trace p^ = {p} (p^ = p- on walls).  This is the exact
        negative adjoint of the weak divergence below (D = -G^T), also on
        curved cells and 2:1 faces, so M A is symmetric positive definite.
        """
        m, d = self.mesh, self.d
        dp = [p @ m.Da[a].T for a in range(d)]  # (D_a p) at nodes
        out = np.zeros((d, m.K, m.nc))
        for b in range(d):
            for a in range(d):
                out[b] += m.Ja[a, b] * dp[a]
        out = out * m.w[None, None, :]
        if len(self.cf_m):
            pm = p[self.cf_m[:, None], self.cf_fm]
            pp = p[self.cf_p[:, None], self.cf_fp]
            ph_ = 0.5 * (pm + pp)
            self._scatter(out, self.cf_m, self.cf_fm, self.cf_N * (self.cf_W * (ph_ - pm))[None])
            self._scatter(out, self.cf_p, self.cf_fp, -self.cf_N * (self.cf_W * (ph_ - pp))[None])
        if len(self.s_f):
            pf = p[self.s_f[:, None], self.s_ff]
            pc = self.coarse_trace(p[None], False)[0]
            ph_ = 0.5 * (pf + pc)
            self._scatter(out, self.s_f, self.s_ff, self.s_N * (self.s_W * (ph_ - pf))[None])
            self._scatter_coarse(out, -self.s_N * (self.s_W * (ph_ - pc))[None])
        return out / m.wJ[None]

    def div(self, f):
        """Nodal DG divergence M^-1 D f with centred traces; f of shape (d, K, Nc) -> (K, Nc)."""
        m, d = self.mesh, self.d
        out = self._volume(f[None], -1.0)
        if len(self.cf_m):
            fh = 0.5 * (f[:, self.cf_m[:, None], self.cf_fm] + f[:, self.cf_p[:, None], self.cf_fp])
            Fs = np.sum(fh * self.cf_N, axis=0)[None] * self.cf_W[None]
            self._scatter(out, self.cf_m, self.cf_fm, Fs)
            self._scatter(out, self.cf_p, self.cf_fp, -Fs)
        if len(self.s_f):
            fc = self.coarse_trace(f, False)
            fh = 0.5 * (f[:, self.s_f[:, None], self.s_ff] + fc)
            Fs = np.sum(fh * self.s_N, axis=0)[None] * self.s_W[None]
            self._scatter(out, self.s_f, self.s_ff, Fs)
            self._scatter_coarse(out, -Fs)
        return out[0] / m.wJ

    def helmholtz(self, p, h, alpha):
        """A p = p/(gamma-1) - alpha div_h(h grad_h p)."""
        return p / (ph.GAMMA - 1.0) - alpha * self.div(h[None] * self.grad(p))

    # ------------------------------------------------------------------ helpers
    def pprime(self, U):
        return ph.pressure(U, self.d) - self.pbar

    def enthalpy(self, U):
        return ph.GAMMA * ph.pressure(U, self.d) / ((ph.GAMMA - 1.0) * U[0])

    def conservation(self, U):
        """Total mass and total energy: sum over nodes of w J rho and w J rho E."""
        wJ = self.mesh.wJ
        return float(np.sum(wJ * U[0])), float(np.sum(wJ * U[self.V - 1]))

    # ------------------------------------------------------------------ initial states
    def state(self, kind=None, seed=0, amp=1.0):
        """Initial state of the case: rest, bubble, inflow (the case's own) or seeded noise."""
        from workloads import noise  # seeded random numbers only

        case, d = self.case, self.d
        init = dict(case.init)
        if kind is not None:
            init["kind"] = kind
        U = self.Ubg.copy()
        X = self.mesh.X
        if init["kind"] == "rest":
            pass
        elif init["kind"] == "bubble":
            # Delta theta = A cos^2(pi r / (2 R)) inside r < R, added at constant pressure.
            rr = (X[0] - init["xc"]) ** 2 + (X[d - 1] - init["zc"]) ** 2
            if d == 3:
                rr = rr + (X[1] - init.get("yc", 0.5 * case.extent[1])) ** 2
            rb = np.sqrt(rr)
            dth = np.where(rb < init["radius"], init["amp"] * np.cos(0.5 * np.pi * rb / init["radius"]) ** 2, 0.0)
            exner = (self.pbar / case.atmosphere["p_ref"]) ** ((ph.GAMMA - 1.0) / ph.GAMMA)
            T = self.pbar / (ph.R_GAS * self.rhobar) + dth * exner
            U[0] = self.pbar / (ph.R_GAS * T)
        elif init["kind"] == "inflow":
            u0 = init.get("u0", 10.0)
            U[1] = self.rhobar * u0
            U[d + 1] = U[d + 1] + 0.5 * self.rhobar * u0 * u0
        elif init["kind"] == "random":
            nz = noise(seed, self.V, self.mesh.K, self.mesh.nc)
            U[0] = U[0] * (1.0 + 0.01 * amp * nz[0])
            for a in range(d):
                U[1 + a] = 5.0 * amp * nz[1 + a]
            U[d + 1] = U[d + 1] * (1.0 + 0.01 * amp * nz[d + 1])
        else:
            raise ValueError(init["kind"])
        return U
