"""The N > 1 path of the benchmark (independent replicas, one map per rank): the timed region
is the maximum over ranks and the whole-job rate counts every rank's scans. Two gloo ranks on
the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws), VBX_BENCH_BACKEND="gloo")
    import bench

    dist, r, n = bench._dist_init()
    local_ms = [120.0, 300.0][r]  # rank 1 is the slower replica
    max_ms, value = bench.whole_job_rate(dist, local_ms, steps=30, ws=n, device="cpu")
    out.put((r, n, max_ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_whole_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, n, max_ms, value in res:
        assert n == 2
        assert max_ms == 300.0  # the slower rank sets the time
        assert value == pytest.approx(2 * 30 / 0.3)  # both ranks' scans over that time


def test_single_process_rate():
    import bench

    max_ms, value = bench.whole_job_rate(None, 250.0, steps=25, ws=1, device="cpu")
    assert max_ms == 250.0 and value == pytest.approx(100.0)
