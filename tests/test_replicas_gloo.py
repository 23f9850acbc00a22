"""The replicas form of the benchmark (one independent solve per GPU, no
data-path collective): the whole-job figures are the slowest rank's step time
and the units of all ranks over it.  Checked with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys

    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = [12.0, 15.5][rank]
        units = [1000, 3000][rank]
        q.put((rank, bench.replica_throughput(dist, ms, units)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_slowest_time_and_total_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        ms, units, value = got[r]
        assert ms == 15.5 and units == 4000.0
        assert value == pytest.approx(4000.0 / 0.0155)


def test_single_process_is_its_own_job():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_throughput(None, 10.0, 500) == (10.0, 500.0, 50000.0)


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun every rank but 0 exits at once without work or output."""
    import subprocess
    import sys
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
