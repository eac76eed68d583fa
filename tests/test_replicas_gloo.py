"""The multi-process path of bench.py (independent replicas, one per GPU, no
data-path collective): the whole-job figure is the units all ranks processed
over the slowest rank's time.  Checked with two gloo ranks on the CPU."""
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


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units = [3.0e9, 5.0e9][rank]
    secs = [2.0, 4.0][rank]
    v, t = bench.replica_throughput(units, secs, dist, torch.device("cpu"))
    out[rank] = (v, t)
    dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        v, t = out[r]
        assert t == 4.0 and v == pytest.approx(8.0e9 / 4.0, rel=1e-15)


def test_replica_throughput_single_process():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.replica_throughput(6.0, 3.0) == (2.0, 3.0)
