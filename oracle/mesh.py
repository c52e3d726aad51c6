"""Connectivity and geometry of the non-conforming terrain-following mesh (test oracle).

Connectivity is found by dictionary look-up of tree leaves: across each face
a cell meets either a leaf of its own level (conforming face), a leaf one
level coarser (this cell is the fine side of a 2:1 face), a refined cell
(this cell is the coarse side; the subfaces are recorded from the fine
cells), or the domain boundary (slip wall unless the axis is periodic).
The paper's meshes are refined both horizontally and vertically with no
hanging nodes in the DG sense (Sec. 2; Sec. 3.1 meshes).

Geometry reading (the paper defers the mesh map to earlier work):
terrain-following (Gal-Chen) map z = zeta + h(x, y) (1 - zeta / H) with the
horizontal coordinates unchanged; every base cell is isoparametric of degree
r (the map sampled at its GLL nodes), and every refined cell takes the
positions of its GLL nodes from its base cell's polynomial, so that 2:1
faces are watertight.  Metric terms J grad(xi^a) come from nodal
derivatives of that polynomial (2D: rotated derivatives; 3D: cross
products, which satisfy the discrete metric identities because x and y are
affine in each cell).
"""

import itertools
import math

import numpy as np

from . import gll as _gll


def node_multi_index(d, n):
    """(Nc, d) integer node coordinates, axis 0 fastest."""
    idx = np.array(list(itertools.product(range(n), repeat=d)))[:, ::-1]
    return idx


def hill_height(hill, x, y=None):
    """Orography h(x[, y]): Gaussian (configs), bell (Sec. 3.1 profile), parabola, none."""
    kind = hill["kind"]
    if kind == "none":
        return np.zeros_like(x)
    if kind == "gauss":
        r2 = (x - hill["xc"]) ** 2
        if y is not None:
            r2 = r2 + (y - hill["yc"]) ** 2
        return hill["hc"] * np.exp(-math.log(2.0) * r2 / hill["half_width"] ** 2)
    if kind == "bell":
        q = 1.0 + ((x - hill["xc"]) / hill["half_width"]) ** 2
        if y is not None:
            q = q + ((y - hill["yc"]) / hill["half_width"]) ** 2
        return hill["hc"] / q ** 1.5
    if kind == "parabola":
        s = 1.0 - ((x - hill["xc"]) / hill["half_width"]) ** 2
        if y is not None:
            s = s - ((y - hill["yc"]) / hill["half_width"]) ** 2
        return hill["hc"] * s
    raise ValueError(kind)


class Mesh:
    """Oracle mesh: faces, subfaces, walls, nodal coordinates and metrics."""

    def __init__(self, case):
        self.case = case
        self.d = d = case.dim
        self.r = r = case.degree
        self.n = n = r + 1
        self.nc = n ** d
        self.K = case.n_cells
        self.xi, self.w1 = _gll.gll(r)
        self.mi = node_multi_index(d, n)
        # tensor weights at nodes
        self.w = np.prod(self.w1[self.mi], axis=1)
        self._connect()
        self._geometry()

    # ------------------------------------------------------------------ topology
    def face_nodes(self, lf):
        a, side = divmod(lf, 2)
        return np.nonzero(self.mi[:, a] == (self.r if side else 0))[0]

    def _connect(self):
        case, d = self.case, self.d
        leaf = {}
        for c in range(self.K):
            leaf[(int(case.levels[c]), tuple(int(v) for v in case.ijk[c]))] = c
        internal = set()
        for (l, ijk) in leaf:
            cc = ijk
            for ll in range(l - 1, -1, -1):
                cc = tuple(v // 2 for v in cc)
                internal.add((ll, cc))
        conf, walls, subs = [], [], []
        for (l, ijk), c in leaf.items():
            for a in range(d):
                for side in (0, 1):
                    lf = 2 * a + side
                    nmax = case.base[a] * 2 ** l
                    nb = list(ijk)
                    nb[a] += 1 if side else -1
                    if nb[a] < 0 or nb[a] >= nmax:
                        if not case.periodic[a]:
                            walls.append((c, lf))
                            continue
                        nb[a] %= nmax
                    nb = tuple(nb)
                    if (l, nb) in leaf:
                        if side == 1:
                            conf.append((c, lf, leaf[(l, nb)], lf - 1))
                    elif l > 0 and (l - 1, tuple(v // 2 for v in nb)) in leaf:
                        cc = leaf[(l - 1, tuple(v // 2 for v in nb))]
                        s = tuple(ijk[t] % 2 for t in range(d) if t != a)
                        subs.append((c, lf, cc, 2 * a + (1 - side), s))
                    elif (l, nb) in internal:
                        pass  # coarse side: recorded by the fine cells
                    else:
                        raise ValueError("mesh is not 2:1 balanced")
        self.conf = conf
        self.walls = walls
        self.subs = subs

    # ------------------------------------------------------------------ geometry
    def _geometry(self):
        case, d, n, r = self.case, self.d, self.n, self.r
        xi = self.xi
        H = case.extent[d - 1]
        hb = np.asarray(case.extent) / np.asarray(case.base)
        X = np.zeros((d, self.K, self.nc))
        cache = {}
        for c in range(self.K):
            l = int(case.levels[c])
            ijk = case.ijk[c]
            base_ijk = ijk // (2 ** l)
            lo_b = base_ijk * hb
            # physical coordinates at the base cell's GLL nodes
            comp_b = lo_b[None, :] + (xi[self.mi] + 1.0) * 0.5 * hb[None, :]
            Xb = comp_b.copy()
            hx = hill_height(case.hill, comp_b[:, 0], comp_b[:, 1] if d == 3 else None)
            zeta = comp_b[:, d - 1]
            Xb[:, d - 1] = zeta + hx * (1.0 - zeta / H)
            # interpolation from the base cell's nodes to this cell's GLL nodes,
            # which depends only on the cell's level and position in its base cell
            key = (l, tuple(int(v) for v in ijk - base_ijk * 2 ** l))
            B = cache.get(key)
            if B is None:
                off = np.array(key[1], dtype=np.float64)
                ref = -1.0 + (2.0 * off[None, :] + xi[self.mi] + 1.0) / 2 ** l
                B = np.ones((self.nc, self.nc))
                for a in range(d):
                    La = _gll.lagrange_eval(xi, ref[:, a])  # [node of c, 1D index]
                    B *= La[:, self.mi[:, a]]
                cache[key] = B
            X[:, c, :] = (B @ Xb).T
        self.X = X
        # nodal derivative matrices D_a[q, i] = d l_i / d xi^a at node q
        D1 = _gll.derivative_matrix(r)
        self.Da = []
        for a in range(d):
            M = np.ones((self.nc, self.nc))
            for b in range(d):
                if b == a:
                    M *= D1[self.mi[:, None, b], self.mi[None, :, b]]
                else:
                    M *= (self.mi[:, None, b] == self.mi[None, :, b])
            self.Da.append(M)
        # dX[a][b] = d x_b / d xi^a at nodes
        dX = np.einsum("aqi,bki->abkq", np.array(self.Da), X)
        Ja = np.zeros((d, d, self.K, self.nc))
        if d == 2:
            J = dX[0, 0] * dX[1, 1] - dX[1, 0] * dX[0, 1]
            Ja[0, 0], Ja[0, 1] = dX[1, 1], -dX[1, 0]
            Ja[1, 0], Ja[1, 1] = -dX[0, 1], dX[0, 0]
        else:
            t = [dX[a] for a in range(3)]  # t[a][b]: tangent vector along xi^a
            cross = lambda u, v: np.array([u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]])
            Ja[0] = cross(t[1], t[2])
            Ja[1] = cross(t[2], t[0])
            Ja[2] = cross(t[0], t[1])
            J = np.sum(t[0] * Ja[0], axis=0)
        if np.any(J <= 0):
            raise ValueError("non-positive Jacobian")
        self.J = J
        self.Ja = Ja
        self.wJ = self.w[None, :] * J

    # ------------------------------------------------------------------ face data
    def face_normal(self, c, lf):
        """Outward J grad(xi^a) on face lf of cell c: (d, NF) = |N| n."""
        a, side = divmod(lf, 2)
        f = self.face_nodes(lf)
        return (2 * side - 1) * self.Ja[a, :, c, f].T

    def face_weights(self, lf):
        a = lf // 2
        f = self.face_nodes(lf)
        tang = [b for b in range(self.d) if b != a]
        return np.prod(self.w1[self.mi[f][:, tang]], axis=1)

    def subface_eval(self, lf_fine, lf_coarse, s):
        """L[k, j]: coarse basis j at fine face node k of subface s (2:1 faces)."""
        a = lf_fine // 2
        f = self.face_nodes(lf_fine)
        pts = np.zeros((len(f), self.d))
        ti = 0
        for b in range(self.d):
            if b == a:
                pts[:, b] = 1.0 if lf_coarse % 2 == 1 else -1.0
            else:
                pts[:, b] = 0.5 * (self.xi[self.mi[f, b]] + (2 * s[ti] - 1))
                ti += 1
        L = np.ones((len(f), self.nc))
        for b in range(self.d):
            Lb = _gll.lagrange_eval(self.xi, pts[:, b])
            L *= Lb[:, self.mi[:, b]]
        return L
