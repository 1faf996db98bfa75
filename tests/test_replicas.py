"""Multi-GPU runs are independent replicas (no collective on the data path):
the host logic around them, on CPU with the gloo backend (world size 2)."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    # rank r timed 100 (r + 1) ms for 10 solves
    rate, t = bench.job_rate(torch, dist, "cpu", 10, 100.0 * (rank + 1))
    q.put((rank, rate, t))
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slowest rank's 200 ms; 2 ranks x 10 solves in 0.2 s
    assert [g[0] for g in got] == [0, 1]
    for _, rate, t in got:
        assert t == 200.0 and rate == pytest.approx(100.0)


def test_job_rate_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(torch, None, "cpu", 5, 250.0) == (20.0, 250.0)


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun only rank 0 runs and prints the CPU reference arm."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
