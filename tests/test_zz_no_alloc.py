"""dg_apply_implicit_noalloc: the Helmholtz operator for callers that cannot allocate.

It must give the result of dg_apply_implicit bit for bit (same kernels, the
gradient scratch taken from the library's fixed 4 MiB array instead of the
mesh), call after call, on a 2D and a refined 3D mesh, and reject meshes whose
scratch would not fit.  Collected last on purpose.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("name", ["hill2d", "tiny3d"])
def test_noalloc_matches_allocating_entry_point_twice(name):
    import paper_2408_08129_gb300 as dg
    from workloads import make_case, tiny_case

    ctx = dg.Context(0)
    if name == "tiny3d":
        case = tiny_case(3, 3, base=(3, 3, 2), extent=(3e3, 3e3, 2e3), refine=[(1, 1, 0), (0, 2, 1)],
                         hill=dict(kind="gauss", hc=250.0, half_width=900.0, xc=1.5e3, yc=1.5e3),
                         atmosphere=dict(kind="stratified", N=0.01, T_ref=293.15, p_ref=1e5))
    else:
        case = make_case(name, 0)
    mesh = dg.Mesh(ctx, case)
    rng = np.random.default_rng(3)
    shp = (mesh.n_cells, mesh.nodes_per_cell)
    alpha = (0.3 * case.dt) ** 2
    for prec, dt in ((dg.DG_FP64, torch.float64), (dg.DG_FP32, torch.float32)):
        for call in range(2):
            p = torch.from_numpy(100.0 * rng.standard_normal(shp)).to(dt).cuda()
            h = torch.from_numpy(3.5e5 * (1.0 + 0.05 * rng.random(shp))).to(dt).cuda()
            ref = torch.empty_like(p)
            out = torch.full_like(p, float("nan"))
            dg.dg_apply_implicit(ctx, mesh, h, p, ref, alpha, prec)
            dg.dg_apply_implicit_noalloc(ctx, mesh, h, p, out, alpha, prec)
            torch.cuda.synchronize()
            assert torch.equal(out, ref), (prec, call, _rel(out.double(), ref.double()))


def test_noalloc_rejects_meshes_beyond_the_static_scratch():
    import paper_2408_08129_gb300 as dg
    from workloads import make_case

    ctx = dg.Context(0)
    mesh = dg.Mesh(ctx, make_case("hill3d", 0))
    shp = (mesh.n_cells, mesh.nodes_per_cell)
    p = torch.zeros(shp, dtype=torch.float64, device="cuda")
    with pytest.raises(dg.DGError, match="too large"):
        dg.dg_apply_implicit_noalloc(ctx, mesh, p, p, torch.empty_like(p), 1.0)
