"""Serving loop: continuous batching, memory-budget admission, host-side fault injection."""

import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from workloads.cases import member2d, request_case  # noqa: E402


@pytest.fixture(scope="module")
def dg():
    import paper_2408_08129_gb300 as m

    return m


@pytest.fixture(scope="module")
def ctx(dg):
    return dg.Context(0)


def _bg(dg, ctx, case):
    mesh = dg.Mesh(ctx, case)
    U = torch.empty(mesh.shape(), dtype=torch.float64, device="cuda")
    dg.dg_background(ctx, mesh, U)
    return U.cpu().numpy()


def _rel_dev(a, b, bg):
    return max(np.linalg.norm(a[v] - b[v]) / max(np.linalg.norm(b[v] - bg[v]), 1e-300) for v in range(a.shape[0]))


def test_result_same_alone_and_in_the_mix(dg, ctx):
    """A request's result alone equals its result when others arrive while it runs."""
    a = member2d(1009)  # 64x32, degree 4
    others = [member2d(1003), request_case(5, 1e4, 1e5), member2d(1011), request_case(9, 1e4, 1e5)]
    opts = dg.solver_opts(tol=1e-12)
    sv = dg.Server(ctx, 40 << 30)
    rid = sv.submit(a, 6, opts=opts)
    sv.wait(rid, 300)
    alone = sv.poll(rid, with_result=True)
    assert alone["state"] == "done" and alone["steps_done"] == 6
    sv.close()

    sv = dg.Server(ctx, 40 << 30)
    rid = sv.submit(a, 6, opts=opts)
    ids = []
    for i, o in enumerate(others):  # arrive while the first member runs, mixed precisions
        time.sleep(0.01)
        prec = dg.DG_FP32 if i % 2 else dg.DG_FP64
        ids.append(sv.submit(o, 3 + i, opts=dg.solver_opts(tol=1e-12, precision=prec)))
    for r in [rid] + ids:
        sv.wait(r, 300)
    mix = sv.poll(rid, with_result=True)
    infos = [sv.poll(r) for r in ids]
    assert all(i["state"] == "done" for i in infos)
    assert mix["state"] == "done"
    assert _rel_dev(mix["U"], alone["U"], _bg(dg, ctx, a)) < 1e-9
    sv.close()


def test_rejections_do_not_disturb_resident_members(dg, ctx):
    a = member2d(1007)
    probe = dg.Server(ctx, 1 << 40)
    fp = probe.poll(probe.submit(a, 1))["footprint_bytes"]
    probe.close()
    sv = dg.Server(ctx, int(1.5 * fp))
    rid = sv.submit(a, 8)
    big = member2d(1001)  # 1.5 M DoF: footprint far above the budget
    with pytest.raises(dg.DGError, match="DG_EBUDGET"):
        sv.submit(big, 5)
    bad = member2d(1011)
    bad.degree = 9  # malformed: degree out of range
    with pytest.raises(dg.DGError, match="DG_EINVAL"):
        sv.submit(bad, 5)
    sv.wait(rid, 300)
    info = sv.poll(rid)
    assert info["state"] == "done" and info["status"] == 0 and info["steps_done"] == 8
    sv.close()


def test_admission_waits_for_memory(dg, ctx):
    """With room for one member at a time, the second is admitted after the first leaves."""
    a, b = member2d(1009), member2d(1010)
    probe = dg.Server(ctx, 1 << 40)
    fp = probe.poll(probe.submit(a, 1))["footprint_bytes"]
    probe.close()
    sv = dg.Server(ctx, int(1.5 * fp))
    ra, rb = sv.submit(a, 4), sv.submit(b, 4)
    sv.wait(ra, 300)
    sv.wait(rb, 300)
    ia, ib = sv.poll(ra), sv.poll(rb)
    assert ia["state"] == ib["state"] == "done"
    assert ia["t_submit"] <= ia["t_admit"] <= ia["t_finish"]
    assert ib["t_admit"] >= ia["t_finish"] - 1e-6
    sv.close()
