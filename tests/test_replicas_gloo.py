"""The N > 1 path of bench.py is replicas only: each rank runs its own
circuit and the job rate is the summed units over the slowest rank's time.
Checked with two gloo processes on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2111_06868_gb300 import circuits as C

    # each replica draws its own circuit (seed + rank), as bench.py does
    circ = C.config_small(seed=rank)
    seconds = [2.0, 3.0][rank]
    rate, tmax = bench.whole_job_rate(seconds, float(len(circ.gates) * 5), dist, "cpu")
    out[rank] = (rate, tmax, [g.name for g in circ.gates[:12]])
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_rate_and_distinct_circuits():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    (r0, t0, c0), (r1, t1, c1) = out[0], out[1]
    assert t0 == t1 == 3.0                      # slowest rank
    assert r0 == r1 == pytest.approx(2 * 163 * 5 / 3.0)
    assert c0 != c1                             # independent inputs per replica


def test_single_process_rate():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.whole_job_rate(4.0, 10.0) == (2.5, 4.0)
