"""Caller-built geometry and face tables in dg_mesh_create (meshes generated elsewhere).

* Round trip: the face tables and node coordinates a mesh exports, handed back
  to dg_mesh_create, give the same mesh -- the same tables, coordinates and
  operator applies bit for bit, and the same IMEX-RK2 step.
* Caller coordinates are used: a flat-terrain description with the node
  coordinates of a hill mesh (built by the CPU oracle) applies the operator of
  the hill mesh, matching the oracle's.
* Broken inputs are rejected: a face missing or listed twice, a subface at the
  wrong position, a conforming face between non-neighbours, a wall inside the
  domain, coordinates that leave a gap at a face, a non-finite coordinate.
"""

import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.dg import DG  # noqa: E402
from workloads import make_case, tiny_case  # noqa: E402

STRAT = dict(kind="stratified", N=0.01, T_ref=293.15, p_ref=1e5)
DG_EINVAL, DG_EUNBALANCED = -1, -6


@pytest.fixture(scope="module")
def dg():
    import paper_2408_08129_gb300 as m

    return m


@pytest.fixture(scope="module")
def ctx(dg):
    return dg.Context(0)


def _tiny(dim, r, hill=True):
    base = (5, 3) if dim == 2 else (3, 3, 2)
    ext = (5e3, 3e3) if dim == 2 else (3e3, 3e3, 2e3)
    h = dict(kind="gauss", hc=250.0, half_width=900.0, xc=ext[0] / 2, yc=ext[1] / 2) if hill else None
    return tiny_case(dim, r, base=base, extent=ext, refine=[(1, 1, 0)[:dim], (3, 0, 0)[:dim]], hill=h,
                     atmosphere=STRAT)


def _applies(dg, ctx, mesh, ref):
    U = torch.from_numpy(ref.state("random", seed=4)).cuda()
    R = torch.empty_like(U)
    dg.dg_apply_explicit(ctx, mesh, U, R)
    rng = np.random.default_rng(2)
    shp = (mesh.n_cells, mesh.nodes_per_cell)
    p = torch.from_numpy(100.0 * rng.standard_normal(shp)).cuda()
    h = torch.from_numpy(3.5e5 * (1.0 + 0.05 * rng.random(shp))).cuda()
    Ap = torch.empty_like(p)
    dg.dg_apply_implicit(ctx, mesh, h, p, Ap, 2.0)
    torch.cuda.synchronize()
    return R.cpu().numpy(), Ap.cpu().numpy()


@pytest.mark.parametrize("name", ["tiny2d", "tiny3d", "hill2d"])
def test_round_trip_is_bit_identical(dg, ctx, name):
    case = {"tiny2d": lambda: _tiny(2, 3), "tiny3d": lambda: _tiny(3, 2), "hill2d": lambda: make_case("hill2d", 0)}[name]()
    ref = DG(case)
    m1 = dg.Mesh(ctx, case)
    faces, X = m1.faces(), m1.coords()
    m2 = dg.Mesh(ctx, case, node_xyz=X, faces=faces)
    for a, b in zip(faces, m2.faces()):
        assert np.array_equal(a, b)
    assert np.array_equal(X, m2.coords())
    for a, b in zip(_applies(dg, ctx, m1, ref), _applies(dg, ctx, m2, ref)):
        assert np.array_equal(a, b)
    opts = dg.solver_opts(tol=1e-12, krylov=dg.DG_KRYLOV_CHEBYSHEV, fused=1)
    out = []
    for m in (m1, m2):
        st = dg.State(ctx, m, opts)
        st.upload(ref.state())
        dg.imex_rk2_step(ctx, m, st, case.dt, opts)
        out.append(st.download())
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("dim,r", [(2, 3), (3, 2)])
def test_caller_coordinates_are_used(dg, ctx, dim, r):
    hill_case = _tiny(dim, r, hill=True)
    flat_case = dataclasses.replace(hill_case, hill=dict(kind="none"))
    ref = DG(hill_case)  # the oracle builds the hill geometry itself
    mesh = dg.Mesh(ctx, flat_case, node_xyz=ref.mesh.X)
    U0 = ref.state("random", seed=9)
    U = torch.from_numpy(U0).cuda()
    R = torch.empty_like(U)
    dg.dg_apply_explicit(ctx, mesh, U, R)
    torch.cuda.synchronize()
    Rref = ref.explicit(U0, "full")
    err = max(np.linalg.norm(R.cpu().numpy()[v] - Rref[v]) / np.linalg.norm(Rref[v]) for v in range(dim + 2))
    assert err < 1e-12, err


def _expect_reject(dg, ctx, case, status, match, **kw):
    with pytest.raises(dg.DGError, match=match) as e:
        dg.Mesh(ctx, case, **kw)
    assert e.value.status == status


def test_broken_inputs_rejected(dg, ctx):
    case = _tiny(2, 3)
    m = dg.Mesh(ctx, case)
    conf, subs, walls = m.faces()
    X = m.coords()
    n = case.degree + 1
    _expect_reject(dg, ctx, case, DG_EUNBALANCED, "watertight", faces=(conf[1:], subs, walls))
    _expect_reject(dg, ctx, case, DG_EUNBALANCED, "twice", faces=(np.vstack([conf, conf[:1]]), subs, walls))
    bad = subs.copy()
    bad[0, 3] ^= 1
    _expect_reject(dg, ctx, case, DG_EUNBALANCED, "position", faces=(conf, bad, walls))
    bad = conf.copy()
    bad[0, 2] = m.n_cells - 1 if bad[0, 2] != m.n_cells - 1 else 0
    _expect_reject(dg, ctx, case, DG_EUNBALANCED, "neighbours", faces=(bad, subs, walls))
    inner = conf[:1, :2].copy()
    _expect_reject(dg, ctx, case, DG_EUNBALANCED, "boundary", faces=(conf, subs, np.vstack([walls, inner])))
    # move one node of a conforming face (not a corner) up by 1 m: a gap opens at the face
    c, lf = int(conf[0, 0]), int(conf[0, 1])
    a, side = lf >> 1, lf & 1
    node = ((n - 1) * side + n) if a == 0 else (1 + n * (n - 1) * side)
    Xb = X.copy()
    Xb[-1, c, node] += 1.0
    _expect_reject(dg, ctx, case, DG_EUNBALANCED, "watertight", node_xyz=Xb)
    Xb = X.copy()
    Xb[0, 0, 0] = np.nan
    _expect_reject(dg, ctx, case, DG_EINVAL, "non-finite", node_xyz=Xb)
