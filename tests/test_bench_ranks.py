"""The multi-rank path of bench.py on CPU (gloo, two ranks): every rank runs its own replica, the
job's time is the slowest rank's, and the value counts the replicas of all ranks.  The reference
arm prints on rank 0 only."""

import contextlib
import io
import os
import socket
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 10.0 + 5.0 * rank  # rank 1 is the slower replica
    ms = bench.max_over_ranks(local_ms, dist, "cpu")
    out[rank] = (ms, bench.whole_job_value(world, 1000, 4, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_job_value():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    with mp.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [mp.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    assert res[0] == res[1]
    ms, value = res[0]
    assert ms == 15.0
    assert value == pytest.approx(2 * 1000 * 4 / 0.015)


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    args = types.SimpleNamespace(steps=1, warmup=0, workload="bubble2d", gpus=2)
    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(args)
    assert buf.getvalue() == ""
