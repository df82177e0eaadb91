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


def test_reference_arm_under_two_ranks_prints_one_line():
    # launched like the N > 1 runs: rank 0 alone times the oracle and prints
    # the line; rank 1 exits 0 without work
    import json
    import subprocess

    pytest.importorskip("torch")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"), "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    assert lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2 and lines[0]["value"] > 0
