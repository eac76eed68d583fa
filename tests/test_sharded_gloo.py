"""The host side of the user-sharded form with two gloo ranks on the CPU:
each rank holds a contiguous user range of one instance (partition_users),
its shard statistics are combined over the process group
(allreduce_shard_stats: int64 sums of counts and item degrees, maxima of the
bounds, minimum of the sign flag), and int64 fixed-point item sums added over
the ranks equal those of the whole instance exactly -- the property the
per-iteration exchange of the sweep's partial sums rests on.  The shard
statistics are computed here with numpy from each rank's rows (what
dlm_shard_local returns for them); the GPU path is covered by
tests/test_gpu_sharded.py."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def instance():
    sys.path.insert(0, ROOT)
    import synth

    r = synth.recipe_production(I=3000, J=120, seed=61)
    r.deg_sigma, r.deg_max = 1.4, 110
    inst = synth.generate(r)
    deg = np.diff(inst.row_ptr)
    keep = np.ones(inst.I, bool)
    keep[::37] = False  # users without edges: rows of length 0
    rp = np.zeros(inst.I + 1, np.int64)
    np.cumsum(np.where(keep, deg, 0), out=rp[1:])
    idx = np.concatenate([np.arange(inst.row_ptr[u], inst.row_ptr[u + 1]) for u in range(inst.I) if keep[u]])
    a = inst.a[idx].copy()
    a[5] = -0.25  # one negative coefficient
    return rp, inst.col[idx].copy(), inst.c[idx].copy(), a, inst.J


def stats_of(rp, col, c, a, J):
    deg = np.bincount(col, minlength=J).astype(np.int64)
    loc = dict(nnz=int(rp[-1] - rp[0]), active_users=int((np.diff(rp) > 0).sum()),
               max_abs_a=float(np.abs(a).max()) if a.size else 0.0, max_abs_c=float(np.abs(c).max()) if c.size else 0.0,
               a_nonneg=int((a >= 0).all()))
    return loc, deg


def fixed_sums(col, a, J, shift):
    return np.bincount(col, weights=np.rint(a.astype(np.float64) ** 2 * 2.0 ** shift), minlength=J).astype(np.int64)


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import paper_2606_07777_gb300 as dlm

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rp, col, c, a, J = instance()
    u0, u1 = dlm.partition_users(rp, world)[rank]
    e0, e1 = int(rp[u0]), int(rp[u1])
    loc, deg = stats_of(rp[u0:u1 + 1] - rp[u0], col[e0:e1], c[e0:e1], a[e0:e1], J)
    g = dlm.allreduce_shard_stats(loc, deg, None, torch.device("cpu"))
    sums = torch.from_numpy(fixed_sums(col[e0:e1], a[e0:e1], J, 40))
    dist.all_reduce(sums, op=dist.ReduceOp.SUM)
    out[rank] = (g, sums.numpy().tobytes(), (u0, u1, e1 - e0))
    dist.destroy_process_group()


def test_shard_statistics_and_exact_sums_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(180)
        assert p.exitcode == 0
    rp, col, c, a, J = instance()
    loc, deg = stats_of(rp, col, c, a, J)
    want = dict(loc, max_item_degree=int(deg.max()))
    full = fixed_sums(col, a, J, 40)
    for r in range(2):
        g, sums, _ = out[r]
        assert g == want
        assert np.array_equal(np.frombuffer(sums, dtype=np.int64), full)
    # the two user ranges tile the users and split the edges about evenly
    (u0, u1, n0), (v0, v1, n1) = out[0][2], out[1][2]
    assert u0 == 0 and u1 == v0 and v1 == len(rp) - 1 and abs(n0 - n1) <= 110


def test_combine_without_a_process_group():
    sys.path.insert(0, ROOT)
    import paper_2606_07777_gb300 as dlm

    rp, col, c, a, J = instance()
    parts = dlm.partition_users(rp, 3)
    stats = [stats_of(rp[u0:u1 + 1] - rp[u0], col[rp[u0]:rp[u1]], c[rp[u0]:rp[u1]], a[rp[u0]:rp[u1]], J)
             for u0, u1 in parts]
    g = dlm.shard_combine([s[0] for s in stats], [s[1] for s in stats])
    loc, deg = stats_of(rp, col, c, a, J)
    assert g == dict(loc, max_item_degree=int(deg.max()))
