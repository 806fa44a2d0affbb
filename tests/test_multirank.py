"""The multi-GPU path of bench.py is independent replicas (no collective on
the data path): the host logic that joins them, the maximum of the step
times over the ranks and the whole-job throughput, run with two gloo ranks
on the CPU."""
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


def _rank(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    # rank r was slower on the first timer and faster on the second
    t = bench.max_over_ranks([1.0 + rank, 5.0 - rank, 2.5], device="cpu")
    v = bench.job_value(ws, 1000.0, t[0])
    q.put((rank, t, v))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in out:
        assert t == [2.0, 5.0, 2.5]            # elementwise maximum over both ranks
        assert v == pytest.approx(2 * 1000.0 / 2.0)  # both replicas' units over the slowest time


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 1.5]) == [3.0, 1.5]
    assert bench.job_value(1, 10.0, 2.0) == 5.0
