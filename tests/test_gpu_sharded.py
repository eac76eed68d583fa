"""The user-sharded form on one GPU.  K shard handles (contiguous user
ranges balanced by edges, the full capacity vector each) are stepped the
way K ranks would step them: every shard sweeps its users, the K exchange
buffers (exact 64-bit fixed-point partial sums) are added and handed back to
every shard, every shard takes the same update.  With every row's threshold
taken by its own lane (coop_max = 1, on both sides: the warp-cooperative
path's sums run in another order, and whether a row takes it depends on the
other rows of its slice), the iterates and the dual trajectory must be
bit-identical to one handle holding every user, and the
certificate assembled from the shards' summed certificate buffers must
equal that handle's.  (Emulated in one process: the ranks' kernels never
wait on one another, the sums are added between launches.)"""
import numpy as np
import pytest

import oracle
from gpu_cases import mixed_instance, to_device

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def shards_of(dlm, inst, K, kind, z, bf16, cut):
    rp = inst.row_ptr
    dev_rows = []
    for u0, u1 in dlm.partition_users(rp, K):
        e0, e1 = int(rp[u0]), int(rp[u1])
        sub = type(inst)(rp[u0:u1 + 1] - rp[u0], inst.col[e0:e1], inst.c[e0:e1], inst.a[e0:e1], inst.b, inst.J)
        dev_rows.append(to_device(sub, torch, bf16))
    opts = dict(kind=kind, z=z, bf16=bf16, cut=cut)
    stats = [dlm.shard_local(*r, inst.J, **opts) for r in dev_rows]
    g = dlm.shard_combine([s[0] for s in stats], [s[1] for s in stats])
    sums = [dlm.shard_item_sums(*r, g, inst.J, **opts) for r in dev_rows]
    sq = np.sum([s[0] for s in sums], axis=0)
    s1 = np.sum([s[1] for s in sums], axis=0)
    return [dlm.ShardedSolver(*r, inst.J, g, sq, s1, **opts) for r in dev_rows]


def exchange(shards, name):
    total = sum(getattr(s, name) for s in shards)
    for s in shards:
        getattr(s, name).copy_(total)


CASES = [
    (2, oracle.SIMPLEX_LE, 1.0, False, None, None, False),
    (3, oracle.SIMPLEX_LE, 1.0, True, None, None, True),
    (4, oracle.BOX, 0.6, False, None, None, True),
    (2, oracle.SIMPLEX_LE, 1.0, False, None, 1500.0, True),
    (3, oracle.BOX_CUT, 0.5, False, 1.0, None, True),
    (1, oracle.SIMPLEX_EQ, 0.8, False, None, None, False),
]


@pytest.mark.parametrize("K,kind,z,bf16,cut,count,precondition", CASES)
def test_shards_are_bit_identical_to_one_handle(dlm_lib, K, kind, z, bf16, cut, count, precondition):
    inst = mixed_instance(seed=41, I=5000, J=300)
    sched = (1e-1, 1e-3, 0.5, 15)
    T = 80
    one = dlm_lib.Solver(*to_device(inst, torch, bf16), inst.J, kind=kind, z=z, bf16=bf16, cut=cut)
    shards = shards_of(dlm_lib, inst, K, kind, z, bf16, cut)
    for s in [one] + shards:
        if count is not None:
            s.set_count_limit(count)
        s.set_schedule(*sched)
        s.set_options(precondition=precondition, coop_max=1)
    one.step(T)
    for _ in range(T):
        for s in shards:
            s.sweep()
        exchange(shards, "exchange")
        for s in shards:
            s.update()
    want = one.lam().cpu().numpy()
    traj = one.trajectory(0, T)
    for s in shards:
        assert np.array_equal(s.lam().cpu().numpy().view(np.uint32), want.view(np.uint32))
        assert np.array_equal(s.trajectory(0, T), traj)
    # the certificate from the shards' summed buffers
    for s in shards:
        s.cert_sweep()
    exchange(shards, "cert_exchange")
    exchange(shards, "cert_obj")
    ref = one.stats()
    for s in shards:
        st = s.cert_finish()
        assert st.iter == ref.iter == T
        assert abs(st.dual_obj - ref.dual_obj) <= 1e-12 * abs(ref.dual_obj)
        assert abs(st.primal_obj - ref.primal_obj) <= 1e-12 * abs(ref.primal_obj)
        if np.isfinite(ref.rel_gap):
            assert abs(st.rel_gap - ref.rel_gap) <= 1e-10
        assert st.max_viol == ref.max_viol
    one.close()
    for s in shards:
        s.close()


def test_shard_solve_and_single_handle_calls(dlm_lib):
    inst = mixed_instance(seed=42, I=3000, J=200)
    shards = shards_of(dlm_lib, inst, 2, oracle.SIMPLEX_LE, 1.0, False, None)

    def reduce_all(name):
        exchange(shards, name)

    # one shard alone cannot iterate through the single-handle calls
    with pytest.raises(dlm_lib.DlmError) as e:
        dlm_lib.dlm_step(shards[0].h, 1)
    assert e.value.status == dlm_lib.DLM_ERR_UNSUPPORTED
    with pytest.raises(dlm_lib.DlmError) as e:
        dlm_lib.dlm_get_stats(shards[0].h)
    assert e.value.status == dlm_lib.DLM_ERR_UNSUPPORTED
    # drive both shards to a certified gap, checking every 25 iterations
    for s in shards:
        s.set_schedule(1e-1, 1e-2, 0.5, 25)
        s.set_options(precondition=True, restart=True, coop_max=1)
    done = 0
    while True:
        for s in shards:
            s.cert_sweep()
        reduce_all("cert_exchange")
        reduce_all("cert_obj")
        st = [s.cert_finish() for s in shards]
        assert st[0].dual_obj == st[1].dual_obj and st[0].rel_gap == st[1].rel_gap
        if st[0].gamma == 1e-2 and st[0].rel_gap <= 1e-4:
            break
        assert done < 20000
        for _ in range(25):
            for s in shards:
                s.sweep()
            reduce_all("exchange")
            for s in shards:
                s.update()
        done += 25
    lam = shards[0].lam().cpu().numpy().astype(np.float64)
    p = oracle.Problem(inst.row_ptr, inst.col, inst.c.astype(np.float64), inst.a.astype(np.float64), inst.b, inst.J)
    cert = oracle.certify(p, lam, 1e-2)
    assert cert["rel_gap"] <= 1.5e-4 and abs(cert["g"] - st[0].dual_obj) <= 2e-6 * abs(cert["g"])
    for s in shards:
        s.close()
