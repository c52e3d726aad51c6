"""Pins of the oracle's mesh: counts, connectivity, geometry and metric identities (no GPU)."""

import math

import numpy as np
import pytest

from oracle.mesh import Mesh
from workloads import make_case, tiny_case


def test_config_cell_counts():
    """Refinement rules give the cell counts of the workload descriptions."""
    c1 = make_case("bubble2d", 0)
    assert c1.n_cells == 128 and c1.n_dof == 4608
    c2 = make_case("hill2d", 0)
    assert c2.n_cells == 2912
    assert np.bincount(c2.levels).tolist() == [1856, 672, 384]
    assert c2.n_dof == 291200
    c3 = make_case("hill3d", 0)
    assert c3.n_cells == 23552 and c3.n_dof == 7536640


def _faces_cover(case):
    """Every cell face is a wall, one conforming face, one fine subface, or 2^(d-1) subfaces."""
    m = Mesh(case)
    d = case.dim
    cover = {}
    for (c, lf) in m.walls:
        cover[(c, lf)] = cover.get((c, lf), 0) + 2 ** (d - 1)
    for (cm, lfm, cp, lfp) in m.conf:
        for key in ((cm, lfm), (cp, lfp)):
            cover[key] = cover.get(key, 0) + 2 ** (d - 1)
    for (cf, lff, cc, lfc, s) in m.subs:
        cover[(cf, lff)] = cover.get((cf, lff), 0) + 2 ** (d - 1)
        cover[(cc, lfc)] = cover.get((cc, lfc), 0) + 1
    assert len(cover) == case.n_cells * 2 * d
    assert all(v == 2 ** (d - 1) for v in cover.values())
    return m


@pytest.mark.parametrize("dim", [2, 3])
def test_connectivity_watertight(dim):
    case = tiny_case(dim, 2, base=(4, 3) if dim == 2 else (3, 3, 2), refine=[(1, 1, 0)[:dim], (2, 0, 0)[:dim]])
    m = _faces_cover(case)
    assert len(m.subs) > 0


def test_connectivity_hill2d_has_lateral_and_vertical_hanging_faces():
    m = _faces_cover(make_case("hill2d", 0))
    axes = {lf // 2 for (_, lf, _, _, _) in m.subs}
    assert axes == {0, 1}


def _parabola_case(dim, r):
    hill = dict(kind="parabola", hc=200.0, half_width=4e3, xc=1.5e3 if dim == 2 else 1e3, yc=1e3)
    return tiny_case(dim, r, hill=hill, refine=[(0, 0, 0)[:dim]])


@pytest.mark.parametrize("dim", [2, 3])
def test_volume_exact_for_polynomial_terrain(dim):
    """sum w J = integral of (H - h) over the footprint, exactly, for a degree-2 hill."""
    case = _parabola_case(dim, 3)
    m = Mesh(case)
    H = case.extent[-1]
    hc, a = case.hill["hc"], case.hill["half_width"]
    if dim == 2:
        L, xc = case.extent[0], case.hill["xc"]
        # integral of hc (1 - ((x - xc)/a)^2) over [0, L]
        ih = hc * (L - ((L - xc) ** 3 + xc ** 3) / (3 * a * a))
        exact = L * H - ih
    else:
        Lx, Ly = case.extent[0], case.extent[1]
        xc, yc = case.hill["xc"], case.hill["yc"]
        ix = ((Lx - xc) ** 3 + xc ** 3) / 3
        iy = ((Ly - yc) ** 3 + yc ** 3) / 3
        ih = hc * (Lx * Ly - (ix * Ly + iy * Lx) / (a * a))
        exact = Lx * Ly * H - ih
    assert abs(m.wJ.sum() - exact) < 1e-9 * exact


@pytest.mark.parametrize("dim", [2, 3])
def test_discrete_metric_identities(dim):
    """sum_a D_a (J grad xi^a)_b = 0 at every node on curved, refined meshes."""
    hill = dict(kind="gauss", hc=300.0, half_width=700.0, xc=1.5e3 if dim == 2 else 1e3, yc=1e3)
    case = tiny_case(dim, 4, hill=hill, refine=[(0, 0, 0)[:dim]])
    m = Mesh(case)
    scale = np.abs(m.Ja).max()
    for b in range(dim):
        s = sum(m.Ja[a, b] @ m.Da[a].T for a in range(dim))
        assert np.abs(s).max() < 1e-12 * scale * case.n_cells


@pytest.mark.parametrize("dim", [2, 3])
def test_faces_geometrically_watertight(dim):
    """Both sides of every face see the same points: conforming nodes and 2:1 subface points."""
    hill = dict(kind="gauss", hc=300.0, half_width=700.0, xc=1.5e3 if dim == 2 else 1e3, yc=1e3)
    case = tiny_case(dim, 3, hill=hill, refine=[(0, 0, 0)[:dim]])
    m = Mesh(case)
    for (cm, lfm, cp, lfp) in m.conf:
        a = lfm // 2
        xm = m.X[:, cm, m.face_nodes(lfm)]
        xp = m.X[:, cp, m.face_nodes(lfp)]
        diff = xm - xp
        if case.periodic[a]:
            # periodic wrap: differ by a multiple of the extent along axis a only
            diff[a] = np.mod(diff[a] + 1.0, case.extent[a]) - 1.0
        assert np.abs(diff).max() < 1e-9
    for (cf, lff, cc, lfc, s) in m.subs:
        L = m.subface_eval(lff, lfc, s)
        xf = m.X[:, cf, m.face_nodes(lff)]
        xc = m.X[:, cc, :] @ L.T
        diff = xf - xc
        a = lff // 2
        if case.periodic[a]:
            diff[a] = np.mod(diff[a] + 1.0, case.extent[a]) - 1.0
        assert np.abs(diff).max() < 1e-9


def test_subface_interpolation_zero_jump():
    """Coarse polynomial of degree <= r evaluated on each subface equals the fine trace."""
    case = tiny_case(3, 3, refine=[(0, 0, 0)], periodic=(False, False, False))
    m = Mesh(case)
    X = m.X
    f = lambda x: 1.0 + x[0] ** 3 - 2 * x[0] * x[1] * x[2] / 1e3 + x[2] ** 2
    for (cf, lff, cc, lfc, s) in m.subs:
        L = m.subface_eval(lff, lfc, s)
        assert np.allclose(L @ f(X[:, cc]), f(X[:, cf][:, m.face_nodes(lff)]), rtol=1e-12, atol=1e-6)
