"""The multi-replica path of bench.py on CPU: two gloo ranks, each with its own
time, must both see the slowest rank's time and the whole-job throughput, and
draw different pseudo-data."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench

    w, r, local = bench.dist_setup()
    dist = bench.dist_init(w, "gloo")
    ms, rate = bench.replica_throughput(dist, 100.0 + 50.0 * rank, 20, w, "cpu")
    dist.barrier()
    q.put((r, ms, rate, bench.replica_seed(11, r)))
    dist.destroy_process_group()


def test_two_replicas_report_max_time_and_total_throughput():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for r, ms, rate, seed in out:
        assert ms == 150.0
        assert abs(rate - 2 * 20 / 0.150) < 1e-9
    assert out[0][3] != out[1][3]
