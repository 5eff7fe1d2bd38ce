"""Multi-process path of bench.py on CPU: two gloo ranks in spawned processes.

The bench runs one replica of the whole solve per GPU (the subdomains of one
problem are not split over GPUs), takes the slowest rank's time and reports
the units all ranks processed over it.  These tests drive the same helpers
and the reference arm's rank handling with world_size 2 on the gloo backend.
"""
import contextlib
import io
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    try:
        import types

        import torch.distributed as dist

        import bench
        from feti_inputs import mesh
        dist.init_process_group("gloo", rank=rank, world_size=world)
        r, w, local = bench._dist()
        ms = 10.0 * (rank + 1)                       # rank 1 is the slow one
        slowest = bench._max_over_ranks(ms, w, "cpu")
        rate = bench._job_rate(100, w, slowest / 1e3)
        # the reference arm: rank 0 alone runs the oracle and prints one line
        args = types.SimpleNamespace(steps=1, warmup=0)
        out = io.StringIO()
        with contextlib.redirect_stdout(out):
            bench.run_reference(args, mesh.cube_problem(4, (2, 2, 1)), {"workload": "cube 4^3, 4 subdomains"})
        dist.barrier()
        dist.destroy_process_group()
        q.put((r, w, local, slowest, rate, out.getvalue()))
    except Exception as e:  # reported to the parent, which fails the test
        q.put(("error", repr(e)))


def test_two_gloo_ranks_max_time_and_whole_job_rate():
    import json
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = []
    try:
        for _ in procs:
            res.append(q.get(timeout=240))
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    errs = [r for r in res if r[0] == "error"]
    assert not errs, errs
    res.sort()
    assert [r[:3] for r in res] == [(0, 2, 0), (1, 2, 1)]
    for r in res:
        assert r[3] == pytest.approx(20.0)           # both ranks see the slowest time
        assert r[4] == pytest.approx(100 * 2 / 0.020)  # units of both ranks over it
    assert res[1][5] == ""                           # rank 1 prints nothing
    line = json.loads(res[0][5].strip())
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_one_rank_helpers_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench._job_rate(10, 1, 2.0) == 5.0
