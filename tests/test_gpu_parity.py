"""CUDA path vs the FP64 CPU oracle, element by element, through the C ABI.

Tolerances: FP64 operator applies <= 1e-12 relative L2 per variable; IMEX-RK2
steps <= 1e-10 relative L2 after 100 steps of the warm-bubble case; integer
connectivity bit-exact.  Cases span several CTAs and ragged tails (cell
counts that are not multiples of the cells-per-CTA of any degree), degrees
1..5, 2D and 3D, conforming and 2:1 faces, flat and curved cells.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.dg import DG  # noqa: E402
from oracle.imex import Stepper  # noqa: E402
from workloads import make_case, tiny_case  # noqa: E402

STRAT = dict(kind="stratified", N=0.01, T_ref=293.15, p_ref=1e5)


@pytest.fixture(scope="module")
def dg():
    import paper_2408_08129_gb300 as m

    return m


@pytest.fixture(scope="module")
def ctx(dg):
    return dg.Context(0)


def _tiny(dim, r, curved=True, refine=True, periodic=None):
    base = (5, 3) if dim == 2 else (3, 3, 2)
    ext = (5e3, 3e3) if dim == 2 else (3e3, 3e3, 2e3)
    hill = dict(kind="gauss", hc=250.0, half_width=900.0, xc=ext[0] / 2, yc=ext[1] / 2) if curved else None
    ref = [(1, 1, 0)[:dim], (3, 0, 0)[:dim]] if refine else []
    return tiny_case(dim, r, base=base, extent=ext, refine=ref, hill=hill, atmosphere=STRAT, periodic=periodic)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _per_var_rel(a, b):
    return max(_rel(a[v], b[v]) for v in range(a.shape[0]))


CASES = [("tiny", 2, r) for r in (1, 2, 3, 4, 5)] + [("tiny", 3, r) for r in (1, 2, 3, 4, 5)] + [
    ("bubble2d", 2, 2), ("hill2d", 2, 4), ("hill3d", 3, 3)]


def _case(name, dim, r):
    if name == "tiny":
        return _tiny(dim, r)
    return make_case(name, 0)


@pytest.mark.parametrize("name,dim,r", CASES)
def test_connectivity_bit_exact(dg, ctx, name, dim, r):
    case = _case(name, dim, r)
    mesh = dg.Mesh(ctx, case)
    ref = DG(case).mesh
    conf, subs, walls = mesh.faces()
    rconf = np.array(sorted(ref.conf)).reshape(-1, 4)
    assert np.array_equal(np.array(sorted(map(tuple, conf))).reshape(-1, 4), rconf)
    rs = sorted((f, lf, c, sum(b << i for i, b in enumerate(s))) for (f, lf, c, _, s) in ref.subs)
    assert np.array_equal(np.array(sorted(map(tuple, subs))).reshape(-1, 4), np.array(rs).reshape(-1, 4))
    assert np.array_equal(np.array(sorted(map(tuple, walls))).reshape(-1, 2), np.array(sorted(ref.walls)).reshape(-1, 2))
    assert np.abs(mesh.coords() - ref.X).max() < 1e-9


@pytest.mark.parametrize("name,dim,r", CASES)
@pytest.mark.parametrize("terms", ["full", "imex"])
def test_explicit_apply_fp64(dg, ctx, name, dim, r, terms):
    case = _case(name, dim, r)
    ref = DG(case)
    mesh = dg.Mesh(ctx, case)
    U0 = ref.state("random", seed=7)
    U = torch.from_numpy(U0).cuda()
    R = torch.empty_like(U)
    dg.dg_apply_explicit(ctx, mesh, U, R, dg.DG_FP64, dg.DG_TERMS_FULL if terms == "full" else dg.DG_TERMS_IMEX_EXPLICIT)
    torch.cuda.synchronize()
    err = _per_var_rel(R.cpu().numpy(), ref.explicit(U0, terms))
    assert err < 1e-12, err


@pytest.mark.parametrize("name,dim,r", CASES)
def test_implicit_operators_fp64(dg, ctx, name, dim, r):
    case = _case(name, dim, r)
    ref = DG(case)
    mesh = dg.Mesh(ctx, case)
    rng = np.random.default_rng(11)
    shp = (ref.mesh.K, ref.mesh.nc)
    p0 = 100.0 * rng.standard_normal(shp)
    h0 = 3.5e5 * (1.0 + 0.05 * rng.random(shp))
    f0 = rng.standard_normal((dim,) + shp)
    p, h, f = (torch.from_numpy(a).cuda() for a in (p0, h0, f0))
    g = torch.empty((dim,) + shp, dtype=torch.float64, device="cuda")
    dv = torch.empty(shp, dtype=torch.float64, device="cuda")
    Ap = torch.empty(shp, dtype=torch.float64, device="cuda")
    dg.dg_apply_grad(ctx, mesh, p, g)
    torch.cuda.synchronize()
    assert _per_var_rel(g.cpu().numpy(), ref.grad(p0)) < 1e-12
    dg.dg_apply_grad(ctx, mesh, p, g, h=h)
    torch.cuda.synchronize()
    assert _per_var_rel(g.cpu().numpy(), h0[None] * ref.grad(p0)) < 1e-12
    dg.dg_apply_div(ctx, mesh, f, dv)
    torch.cuda.synchronize()
    assert _rel(dv.cpu().numpy(), ref.div(f0)) < 1e-12
    alpha = (0.3 * case.dt) ** 2
    dg.dg_apply_implicit(ctx, mesh, h, p, Ap, alpha)
    torch.cuda.synchronize()
    assert _rel(Ap.cpu().numpy(), ref.helmholtz(p0, h0, alpha)) < 1e-12


@pytest.mark.parametrize("name,dim,r", CASES)
def test_implicit_operators_fp32(dg, ctx, name, dim, r):
    """FP32 gradient, divergence and Helmholtz operator (one launch per operator; on these
    meshes, affine in x and y, the metric terms are recomputed from the nodal heights) against
    the FP64 oracle, to FP32 accuracy."""
    case = _case(name, dim, r)
    ref = DG(case)
    mesh = dg.Mesh(ctx, case)
    rng = np.random.default_rng(12)
    shp = (ref.mesh.K, ref.mesh.nc)
    p0 = 100.0 * rng.standard_normal(shp)
    h0 = 3.5e5 * (1.0 + 0.05 * rng.random(shp))
    f0 = rng.standard_normal((dim,) + shp)
    p, h, f = (torch.from_numpy(a).float().cuda() for a in (p0, h0, f0))
    p0, h0, f0 = (a.astype(np.float32).astype(np.float64) for a in (p0, h0, f0))  # the same inputs
    g = torch.empty((dim,) + shp, dtype=torch.float32, device="cuda")
    dv = torch.empty(shp, dtype=torch.float32, device="cuda")
    Ap = torch.empty(shp, dtype=torch.float32, device="cuda")
    dg.dg_apply_grad(ctx, mesh, p, g, h=h, precision=dg.DG_FP32)
    dg.dg_apply_div(ctx, mesh, f, dv, precision=dg.DG_FP32)
    alpha = (0.3 * case.dt) ** 2
    dg.dg_apply_implicit(ctx, mesh, h, p, Ap, alpha, precision=dg.DG_FP32)
    torch.cuda.synchronize()
    e = [_per_var_rel(g.double().cpu().numpy(), h0[None] * ref.grad(p0)),
         _rel(dv.double().cpu().numpy(), ref.div(f0)),
         _rel(Ap.double().cpu().numpy(), ref.helmholtz(p0, h0, alpha))]
    assert max(e) < 2e-5, e


@pytest.mark.parametrize("name,dim,r", [("tiny", 2, 1), ("tiny", 2, 4), ("tiny", 3, 2), ("tiny", 3, 3),
                                        ("bubble2d", 2, 2), ("hill2d", 2, 4), ("hill3d", 3, 3)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cell_partitions_give_identical_operators(dg, ctx, name, dim, r, precision):
    """The balanced cell partition (on small meshes, cost-balanced batches of at most CPB consecutive
    cells, one per CTA of a persistent solve, one cell each on the tiny meshes; on hill3d, the
    uniform batches in a cost-balanced order over the CTAs) changes only which CTA computes which
    cell: gradient, divergence and Helmholtz operator are bitwise equal to those on the uniform
    batches, and match the oracle."""
    case = _case(name, dim, r)
    ref = DG(case)
    mesh = dg.Mesh(ctx, case)
    if name == "hill3d":
        assert mesh.n_batches[1] == mesh.n_batches[0] > 0
    else:
        assert mesh.n_batches[1] > mesh.n_batches[0] > 0
    rng = np.random.default_rng(13)
    shp = (ref.mesh.K, ref.mesh.nc)
    p0 = 100.0 * rng.standard_normal(shp)
    h0 = 3.5e5 * (1.0 + 0.05 * rng.random(shp))
    f0 = rng.standard_normal((dim,) + shp)
    dt = torch.float64 if precision == "fp64" else torch.float32
    prec = dg.DG_FP64 if precision == "fp64" else dg.DG_FP32
    p, h, f = (torch.from_numpy(a).to(dt).cuda() for a in (p0, h0, f0))
    alpha = (0.3 * case.dt) ** 2
    out = []
    for part in (0, 1, 0):
        mesh.set_partition(part)
        g = torch.empty((dim,) + shp, dtype=dt, device="cuda")
        dv = torch.empty(shp, dtype=dt, device="cuda")
        Ap = torch.empty(shp, dtype=dt, device="cuda")
        dg.dg_apply_grad(ctx, mesh, p, g, h=h, precision=prec)
        dg.dg_apply_div(ctx, mesh, f, dv, precision=prec)
        dg.dg_apply_implicit(ctx, mesh, h, p, Ap, alpha, precision=prec)
        torch.cuda.synchronize()
        out.append([x.double().cpu().numpy() for x in (g, dv, Ap)])
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
    for a, b in zip(out[0], out[2]):
        assert np.array_equal(a, b)
    if precision == "fp64":
        assert _per_var_rel(out[1][0], h0[None] * ref.grad(p0)) < 1e-12
        assert _rel(out[1][1], ref.div(f0)) < 1e-12
        assert _rel(out[1][2], ref.helmholtz(p0, h0, alpha)) < 1e-12
    with pytest.raises(dg.DGError):
        mesh.set_partition(2)


@pytest.mark.parametrize("krylov", ["chebyshev", "gmres", "cg"])
def test_persistent_solves_on_balanced_partition(dg, ctx, krylov):
    """Two IMEX-RK2 steps of hill2d with the persistent solves (and every implicit pass) on the
    cost-balanced cell batches match the oracle as on the uniform ones."""
    case = make_case("hill2d", 0)
    ref = DG(case)
    mesh = dg.Mesh(ctx, case)
    mesh.set_partition(1)
    st = dg.State(ctx, mesh)
    st.upload(ref.state())
    kry = {"chebyshev": dg.DG_KRYLOV_CHEBYSHEV, "gmres": dg.DG_KRYLOV_GMRES, "cg": dg.DG_KRYLOV_CG}[krylov]
    opts = dg.solver_opts(tol=1e-12, fused=1, krylov=kry)
    for _ in range(2):
        dg.imex_rk2_step(ctx, mesh, st, case.dt, opts)
    assert mesh.autotuned()["fp64"]["partition"] == "balanced"
    S = Stepper(ref, tol=1e-12)
    Ur = S.step(S.step(ref.state(), case.dt), case.dt)
    assert _per_var_rel(st.download() - ref.Ubg, Ur - ref.Ubg) < 1e-10


@pytest.mark.parametrize("name,dim,r", [("tiny", 2, 3), ("tiny", 3, 2), ("hill2d", 2, 4)])
def test_conservation_sums(dg, ctx, name, dim, r):
    case = _case(name, dim, r)
    ref = DG(case)
    mesh = dg.Mesh(ctx, case)
    U0 = ref.state("random", seed=5)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    dg.dg_conservation(ctx, mesh, torch.from_numpy(U0).cuda(), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    exp = np.array(ref.conservation(U0))
    assert np.all(np.abs(got - exp) <= 1e-13 * np.abs(exp))


def test_background_and_initial_states(dg, ctx):
    case = make_case("bubble2d", 0)
    ref = DG(case)
    mesh = dg.Mesh(ctx, case)
    U = torch.empty(mesh.shape(), dtype=torch.float64, device="cuda")
    dg.dg_background(ctx, mesh, U)
    assert _per_var_rel(U.cpu().numpy()[[0, 3]], ref.Ubg[[0, 3]]) < 1e-14
    init = case.init
    dg.dg_init_state(ctx, mesh, "bubble", [init["amp"], init["radius"], init["xc"], init["zc"]], U)
    assert _per_var_rel(U.cpu().numpy()[[0, 3]], ref.state()[[0, 3]]) < 1e-14
    case2 = make_case("hill2d", 0)
    ref2 = DG(case2)
    mesh2 = dg.Mesh(ctx, case2)
    U2 = torch.empty(mesh2.shape(), dtype=torch.float64, device="cuda")
    dg.dg_init_state(ctx, mesh2, "inflow", [10.0], U2)
    assert _per_var_rel(U2.cpu().numpy()[[0, 1, 3]], ref2.state()[[0, 1, 3]]) < 1e-14


def test_apply_is_deterministic(dg, ctx):
    case = make_case("hill2d", 0)
    ref = DG(case)
    mesh = dg.Mesh(ctx, case)
    U = torch.from_numpy(ref.state("random", seed=1)).cuda()
    R1, R2 = torch.empty_like(U), torch.empty_like(U)
    dg.dg_apply_explicit(ctx, mesh, U, R1)
    dg.dg_apply_explicit(ctx, mesh, U, R2)
    torch.cuda.synchronize()
    assert torch.equal(R1, R2)


def test_fp32_explicit_apply_accuracy(dg, ctx):
    """FP32 apply on the perturbation about the FP64 background: single-precision accuracy."""
    case = make_case("hill2d", 0)
    ref = DG(case)
    mesh = dg.Mesh(ctx, case)
    U0 = ref.state()
    Up = torch.from_numpy(U0 - ref.Ubg).float().cuda()
    R = torch.empty_like(Up)
    dg.dg_apply_explicit(ctx, mesh, Up, R, dg.DG_FP32, dg.DG_TERMS_IMEX_EXPLICIT)
    torch.cuda.synchronize()
    Rref = ref.explicit(U0, "imex")
    err = _per_var_rel(R.double().cpu().numpy(), Rref)
    assert err < 1e-4, err


@pytest.mark.parametrize("name,dim,r", CASES)
@pytest.mark.parametrize("terms", ["full", "imex"])
def test_fp32_explicit_apply_all_meshes(dg, ctx, name, dim, r, terms):
    """FP32 explicit apply (perturbation state, FP64 background added inside) against the FP64
    oracle on every parity mesh and both term sets, and its mass balance: each face flux is
    computed once and taken by both sides, so sum w J R_rho vanishes to FP32 rounding."""
    case = _case(name, dim, r)
    ref = DG(case)
    mesh = dg.Mesh(ctx, case)
    U0 = ref.state("random", seed=3)
    Up = torch.from_numpy(U0 - ref.Ubg).float().cuda()
    R = torch.empty_like(Up)
    kind = dg.DG_TERMS_FULL if terms == "full" else dg.DG_TERMS_IMEX_EXPLICIT
    dg.dg_apply_explicit(ctx, mesh, Up, R, dg.DG_FP32, kind)
    torch.cuda.synchronize()
    Rg = R.double().cpu().numpy()
    Rref = ref.explicit(U0, terms)
    err = _per_var_rel(Rg, Rref)
    assert err < 2e-4, err
    wJ = ref.mesh.wJ
    assert abs(np.sum(wJ * Rg[0])) <= 1e-5 * np.sum(np.abs(wJ * Rg[0]))


def _run_steps(dg, ctx, case, n, opts, oracle_tol=1e-12):
    ref = DG(case)
    U0 = ref.state()
    mesh = dg.Mesh(ctx, case)
    st = dg.State(ctx, mesh, opts)
    st.upload(U0)
    stepper = Stepper(ref, tol=oracle_tol)
    Ur = U0
    for _ in range(n):
        dg.imex_rk2_step(ctx, mesh, st, case.dt, opts)
        Ur = stepper.step(Ur, case.dt)
    return st.download(), Ur, ref


# A step holds six Helmholtz solves at relative residual 1e-12, whose solution
# error is the residual times the operator's condition number, so one step is
# held to 1e-11; the 100-step bar is the 1e-10 of the FP64 target.
@pytest.mark.parametrize("nsteps,tol", [(1, 1e-11), (10, 1e-11), (100, 1e-10)])
def test_imex_steps_bubble2d(dg, ctx, nsteps, tol):
    case = make_case("bubble2d", 0)
    opts = dg.solver_opts(tol=1e-12)
    U, Ur, ref = _run_steps(dg, ctx, case, nsteps, opts)
    # compare the deviation from the background, the part the dynamics changes
    err = _per_var_rel(U - ref.Ubg, Ur - ref.Ubg)
    assert err < tol, err


def test_imex_steps_unfused_krylov(dg, ctx):
    """The one-launch-per-kernel GMRES gives the same step as the persistent one."""
    case = make_case("bubble2d", 0)
    U, Ur, ref = _run_steps(dg, ctx, case, 3, dg.solver_opts(tol=1e-12, fused=0))
    assert _per_var_rel(U - ref.Ubg, Ur - ref.Ubg) < 1e-11


def test_imex_steps_hill2d(dg, ctx):
    case = make_case("hill2d", 0)
    opts = dg.solver_opts(tol=1e-12)
    U, Ur, ref = _run_steps(dg, ctx, case, 2, opts)
    err = _per_var_rel(U - ref.Ubg, Ur - ref.Ubg)
    assert err < 1e-10, err


@pytest.mark.parametrize("fused", [1, 0])
@pytest.mark.parametrize("inner_tol", [1e-4, 1e-6])
def test_imex_fp32_refined_step(dg, ctx, fused, inner_tol):
    """FP32 Krylov mat-vecs and basis inside FP64 iterative refinement.

    The FP64 residual at every restart drives each Helmholtz solve to the FP64
    tolerance, so after 10 steps the deviation from the background agrees
    with the FP64 oracle to 1e-8 (the FP32-refined target), whether each FP32
    cycle reduces the residual by 1e-4 or by 1e-6 (the default, near the FP32
    limit).
    """
    case = make_case("bubble2d", 0)
    opts = dg.solver_opts(tol=1e-12, precision=dg.DG_FP32, inner_tol=inner_tol, fused=fused)
    U, Ur, ref = _run_steps(dg, ctx, case, 10, opts)
    assert _per_var_rel(U, Ur) < 1e-10
    assert _per_var_rel(U - ref.Ubg, Ur - ref.Ubg) < 1e-8


def test_rest_state_stays_at_rest(dg, ctx):
    case = _tiny(3, 3)
    ref = DG(case)
    mesh = dg.Mesh(ctx, case)
    st = dg.State(ctx, mesh)
    st.upload(ref.Ubg)
    dg.imex_rk2_step(ctx, mesh, st, case.dt)
    U = st.download()
    assert np.abs(U[1:4]).max() < 1e-9
    assert _rel(U[0], ref.Ubg[0]) < 1e-14 and _rel(U[4], ref.Ubg[4]) < 1e-14


@pytest.mark.parametrize("krylov,forms", [("gmres", ("gmres_persistent", "gmres_multi_kernel")),
                                          ("auto", ("gmres_persistent", "gmres_multi_kernel", "chebyshev"))])
def test_autotuner_times_the_solver_forms(dg, ctx, krylov, forms):
    """krylov = GMRES with fused = -1 times both GMRES forms; krylov = AUTO adds Chebyshev; the
    fastest is kept, and the tuned step still matches the oracle."""
    case = make_case("bubble2d", 0)
    ref = DG(case)
    mesh = dg.Mesh(ctx, case)
    st = dg.State(ctx, mesh)
    st.upload(ref.state())
    assert mesh.autotuned()["fp64"]["form"] is None
    kry = dg.DG_KRYLOV_GMRES if krylov == "gmres" else dg.DG_KRYLOV_AUTO
    opts = dg.solver_opts(tol=1e-12, fused=-1, krylov=kry)
    dg.imex_rk2_step(ctx, mesh, st, case.dt, opts)
    t = mesh.autotuned()["fp64"]
    assert sorted(t["ms"]) == sorted(forms)
    cands = {(f, "uniform"): v for f, v in t["ms"].items()}
    if "balanced" in t["batches"]:  # the cost-balanced cell partition is timed too
        assert sorted(t["ms_balanced"]) == sorted(forms)
        cands.update({(f, "balanced"): v for f, v in t["ms_balanced"].items()})
    assert (t["form"], t["partition"]) == min(cands, key=cands.get)
    dg.imex_rk2_step(ctx, mesh, st, case.dt, opts)
    Ur = Stepper(ref, tol=1e-12).step(Stepper(ref, tol=1e-12).step(ref.state(), case.dt), case.dt)
    assert _per_var_rel(st.download() - ref.Ubg, Ur - ref.Ubg) < 1e-9


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("krylov", ["cg", "gmres_cgs2", "chebyshev"])
def test_imex_steps_other_krylov_forms(dg, ctx, precision, krylov):
    """CG in the w J inner product (M A is SPD), GMRES with classical Gram-Schmidt twice per step
    and Chebyshev iteration on [1/(gamma-1), lmax] reach the same step as the oracle's GMRES."""
    prec = dg.DG_FP64 if precision == "fp64" else dg.DG_FP32
    kry = {"cg": dg.DG_KRYLOV_CG, "gmres_cgs2": dg.DG_KRYLOV_GMRES_CGS2,
           "chebyshev": dg.DG_KRYLOV_CHEBYSHEV}[krylov]
    opts = dg.solver_opts(tol=1e-12, krylov=kry, precision=prec, inner_tol=1e-4, fused=1)
    case = make_case("bubble2d", 0)
    U, Ur, ref = _run_steps(dg, ctx, case, 10, opts)
    assert _per_var_rel(U - ref.Ubg, Ur - ref.Ubg) < 1e-9
    case = make_case("hill2d", 0)
    U, Ur, ref = _run_steps(dg, ctx, case, 2, opts)
    assert _per_var_rel(U - ref.Ubg, Ur - ref.Ubg) < 1e-9


def test_chebyshev_bound_estimate_and_repair(dg, ctx):
    """The power-iteration bound sits just above the Helmholtz spectrum (<= 1.05 x lmax, and above
    the largest Ritz value GMRES finds); a bound set too low is caught: the solve falls back to
    GMRES, still matches the oracle, and the bound is re-estimated on the next solve."""
    case = make_case("bubble2d", 0)
    opts = dg.solver_opts(tol=1e-12, krylov=dg.DG_KRYLOV_CHEBYSHEV, fused=1)
    mesh = dg.Mesh(ctx, case)
    st = dg.State(ctx, mesh, opts)
    assert st.chebyshev_bound() == (0.0, 0.0)
    # a fresh state: estimate on the first solve
    r = DG(case)
    st.upload(r.state())
    dg.imex_rk2_step(ctx, mesh, st, case.dt, opts)
    lmax, alpha = st.chebyshev_bound()
    assert alpha > 0 and lmax > 2.5
    # dense spectrum of the oracle's operator at the initial enthalpy: the bound covers it
    K, nc = r.mesh.K, r.mesh.nc
    h = r.enthalpy(r.state())
    n = K * nc
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = r.helmholtz(e.reshape(K, nc), h, alpha).ravel()
    ev = np.linalg.eigvals(A).real.max()
    assert ev <= lmax <= 1.06 * ev, (ev, lmax)
    # too low a bound: repaired
    st.upload(r.state())
    st.chebyshev_bound((2.6, alpha))
    stats = dg.imex_rk2_step(ctx, mesh, st, case.dt, opts)
    assert stats["status"] == 0
    Uref = Stepper(r, tol=1e-12).step(r.state(), case.dt)
    assert _per_var_rel(st.download() - r.Ubg, Uref - r.Ubg) < 1e-9
    assert st.chebyshev_bound()[0] > 2.6 + 1e-9


@pytest.mark.parametrize("name,nsteps,sponge", [
    ("bubble2d", 10, dict(depth=4e3, rate=0.2, u0=0.0)),
    ("hill2d", 2, dict(depth=8e3, rate=0.5, u0=10.0)),
    ("hill2d", 2, dict(depth=8e3, rate=0.5, u0=10.0, lateral_width=6e3, lateral_rate=0.3)),
    ("hill3d", 1, dict(depth=5e3, rate=0.3, u0=10.0)),
])
def test_imex_steps_with_damping_layer(dg, ctx, name, nsteps, sponge):
    """Rayleigh damping layers below the top (and along the lateral boundaries): the GPU step
    matches the oracle's."""
    import dataclasses

    case = dataclasses.replace(make_case(name, 0), sponge=sponge)
    assert sponge["rate"] * case.dt <= 1.0
    opts = dg.solver_opts(tol=1e-12)
    U, Ur, ref = _run_steps(dg, ctx, case, nsteps, opts)
    assert ref.tau is not None and ref.tau.max() > 0
    assert _per_var_rel(U - ref.Ubg, Ur - ref.Ubg) < 1e-9


def test_bell_hill_nonconforming_step_matches_oracle(dg, ctx):
    """Sec. 3.1's bell-shaped hill on the non-conforming mesh (1972 cells, degree 4, two 2:1 levels,
    top and lateral absorbing layers, dt = 2 s): one FP64 step against the oracle."""
    case = make_case("bell3d_nc", 0)
    U, Ur, ref = _run_steps(dg, ctx, case, 1, dg.solver_opts(tol=1e-12))
    assert ref.tau is not None and ref.tau.max() > 0
    assert _per_var_rel(U - ref.Ubg, Ur - ref.Ubg) < 1e-10


def test_damping_layer_parameters_validated(dg, ctx):
    import dataclasses

    case = make_case("bubble2d", 0)
    for bad in (dict(depth=2e4, rate=0.1), dict(depth=1e3, rate=-1.0), dict(lateral_width=2e4, lateral_rate=0.1),
                dict(lateral_width=1e3, lateral_rate=-0.1)):
        with pytest.raises(dg.DGError, match="sponge"):
            dg.Mesh(ctx, dataclasses.replace(case, sponge=bad))


def test_newton_rsqrt_against_cuda(dg):
    """The solvers' own FP64 1/sqrt (FP32 seed + two Newton steps) against CUDA's 1/sqrt: within
    2 ulp over the whole FP32 exponent range the solvers use it on."""
    rng = np.random.default_rng(5)
    x = torch.from_numpy(10.0 ** rng.uniform(-30, 30, 1 << 16)).cuda()
    y = torch.empty_like(x)
    dg.dg_math_selftest(0, x, y)
    ref = torch.rsqrt(x)
    torch.cuda.synchronize()
    ulp = torch.abs(y - ref) / (torch.abs(ref) * 2.0 ** -52)
    assert float(ulp.max()) <= 2.0
