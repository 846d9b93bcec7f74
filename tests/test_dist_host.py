"""Host logic of multi-GPU runs, as world_size-2 gloo process groups on the
CPU. With more than one GPU the hot path runs as independent replicas: each
rank applies the program to its own fields, with no collective on the data
path. The whole-job figures take the slowest rank's time over the units all
ranks processed. The reference arm runs on rank 0 alone."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        assert bench._dist() == (ws, rank, rank)
        ms = 10.0 * (rank + 1)                      # rank 1 is the slow one
        slowest = bench._max_over_ranks(ms, dist)
        rate = bench._job_rate(1000, ms, ws, dist)  # 1000 units per rank
        out.put((rank, slowest, rate))
    finally:
        dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank_over_all_units():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, out)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(out.get(timeout=5) for _ in range(ws))
    for rank, slowest, rate in res:
        assert slowest == 20.0                       # max over ranks, seen by every rank
        assert rate == pytest.approx(2 * 1000 / 20e-3)


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench._max_over_ranks(7.5) == 7.5
    assert bench._job_rate(500, 2.0, 1) == pytest.approx(500 / 2e-3)


def _ref_rank(rank, ws, port, out):
    import contextlib
    import io
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    if rank == 0:
        out.put((rank, "skipped"))   # rank 0 would time the oracle for minutes; only the others are checked
        return
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        rc = bench.run_reference(type("A", (), {"steps": 3, "warmup": 3, "gpus": ws})())
    out.put((rank, rc, buf.getvalue()))


def test_reference_arm_other_ranks_exit_without_work():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_ref_rank, args=(r, ws, port, out)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    res = dict((r[0], r[1:]) for r in (out.get(timeout=5) for _ in range(ws)))
    assert res[1] == (0, "")                         # exit 0, nothing printed
