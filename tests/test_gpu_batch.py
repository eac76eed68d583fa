"""Batches and the mapping tuner.

A batch sweeps several independent instances in one launch per iteration.
Item sums are exact fixed-point sums and each user's x depends only on its own
slice, so a member's iterates must be bit-identical to those of the same
instance run alone (same cooperative threshold), whatever the slice-to-CTA
mapping; and each member must follow the FP64 oracle's accelerated iteration
(Sec. 4.4 with the continuation of App. B.2) within the trajectory tolerance
of the single-instance tests.  The tuner must leave the iteration state as it
found it.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_cases import oracle_problem, to_device, with_empty_users

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

T = 120


def members():
    """Seven seeded production-generator instances of mixed size (one with
    empty users), each with its own schedule and preconditioning flag."""
    out = []
    for k, (r, gamma) in enumerate(synth.recipe_batch(n=7, seed=2024, users_lo=2e3, users_hi=3e4, items_lo=20,
                                                      items_hi=600)):
        inst = synth.generate(r)
        if k == 2:
            inst = with_empty_users(inst, 40, seed=k)
        sched = (gamma, gamma, 0.5, 1 << 30) if k % 2 == 0 else (10 * gamma, gamma, 0.5, 25)
        out.append((inst, sched, k % 3 == 1))
    return out


def make(dlm, inst, sched, precond):
    rp, col, c, a, b = to_device(inst, torch)
    s = dlm.Solver(rp, col, c, a, b, inst.J)
    s.set_schedule(*sched)
    s.set_options(precondition=precond)
    return s


def lam_of(s):
    return s.lam().cpu().numpy()


@pytest.fixture(scope="module")
def cases():
    return members()


@pytest.fixture(scope="module")
def alone(dlm_lib, cases):
    """lam after T iterations of each instance run by its own handle."""
    out = []
    for inst, sched, pre in cases:
        s = make(dlm_lib, inst, sched, pre)
        s.step(T)
        out.append(lam_of(s))
        s.close()
    return out


@pytest.fixture(scope="module")
def alone_traj(dlm_lib, cases):
    """g(y_t), t < T, of each instance run by its own handle."""
    out = []
    for inst, sched, pre in cases:
        s = make(dlm_lib, inst, sched, pre)
        s.step(T)
        out.append(s.trajectory(0, T))
        s.close()
    return out


def test_members_follow_the_oracle(cases, alone):
    for k, (inst, sched, pre) in enumerate(cases):
        p = oracle_problem(inst)
        ref = oracle.fista(p, T, sched[0], sched[1], sched[2], sched[3], precondition=pre, trajectory=False)["lam"]
        err = np.abs(alone[k].astype(np.float64) - ref).max()
        print(f"member {k}: max |dlam| / |lam| = {err / max(np.abs(ref).max(), 1e-6):.3e}")
        assert err <= 1e-5 * max(np.abs(ref).max(), 1e-6), f"member {k}: max err {err:.3e}"


@pytest.mark.parametrize("mapping,threads", [(0, 0), (1, 0), (2, 512), (1, 512), (3, 512), (2, 0)])
def test_batch_is_bit_identical_to_single_handles(dlm_lib, cases, alone, alone_traj, mapping, threads):
    solvers = [make(dlm_lib, *c) for c in cases]
    bt = dlm_lib.Batch(solvers)
    bt.set_options(mapping=mapping, block_threads=threads, graph_iters=7)
    bt.step(T)
    for k, s in enumerate(solvers):
        got = lam_of(s)
        assert np.array_equal(got.view(np.uint32), alone[k].view(np.uint32)), f"member {k} differs"
        assert np.array_equal(s.trajectory(0, T), alone_traj[k]), f"member {k}: dual trajectory differs"
    st = bt.stats()
    assert all(x.status == dlm_lib.DLM_OK and x.iter == T for x in st)
    bt.close()
    for s in solvers:
        s.close()


def test_batch_stats_and_solve(dlm_lib, cases):
    solvers = [make(dlm_lib, *c) for c in cases]
    bt = dlm_lib.Batch(solvers)
    bt.step(30)
    st = bt.stats()
    for k, s in enumerate(solvers):
        one = s.stats()  # same lam, evaluated by the member's own handle
        assert one.iter == st[k].iter == 30
        assert abs(one.dual_obj - st[k].dual_obj) <= 1e-12 * abs(one.dual_obj)
        assert abs(one.primal_obj - st[k].primal_obj) <= 1e-12 * abs(one.primal_obj)
        assert st[k].rel_gap >= -1e-12
    status, fin = bt.solve(1e-2, 20000)
    assert status == dlm_lib.DLM_OK
    for k, x in enumerate(fin):
        assert x.converged == 1 and x.rel_gap <= 1e-2 and x.gamma == cases[k][1][1]
    bt.close()
    for s in solvers:
        s.close()


def test_autotune_keeps_the_state_and_trajectory(dlm_lib, cases):
    inst, sched, pre = cases[3]
    s = make(dlm_lib, inst, sched, pre)
    ref = make(dlm_lib, inst, sched, pre)
    s.step(30)
    ref.step(30)
    lam0, y0, st0 = s.get_state()
    chosen, ms = s.autotune(iters=2)
    lam1, y1, st1 = s.get_state()
    assert torch.equal(lam0, lam1) and torch.equal(y0, y1)
    assert (st0.iter, st0.theta, st0.stage) == (st1.iter, st1.theta, st1.stage)
    assert ms > 0 and chosen.block_threads in (512, 1024) and chosen.mapping in (1, 2, 3)
    assert s.options().coop_max == chosen.coop_max
    ref.set_options(precondition=pre, coop_max=chosen.coop_max, short_rows=chosen.short_rows)
    s.step(40)
    ref.step(40)
    assert torch.equal(s.lam(), ref.lam())
    s.close()
    ref.close()


def test_batch_autotune_keeps_the_state(dlm_lib, cases):
    solvers = [make(dlm_lib, *c) for c in cases]
    bt = dlm_lib.Batch(solvers)
    bt.step(20)
    before = [lam_of(s) for s in solvers]
    chosen, ms = bt.autotune(iters=2)
    assert ms > 0
    for k, s in enumerate(solvers):
        assert np.array_equal(lam_of(s).view(np.uint32), before[k].view(np.uint32))
    assert all(x.iter == 20 for x in bt.stats())
    bt.close()
    for s in solvers:
        s.close()


def test_batch_rejects_bad_members(dlm_lib, cases):
    a = make(dlm_lib, *cases[0])
    b = make(dlm_lib, *cases[1])
    with pytest.raises(dlm_lib.DlmError) as e:
        dlm_lib.Batch([a, b, a])
    assert e.value.status == dlm_lib.DLM_ERR_INVALID_ARG
    inst = cases[1][0]
    rp, col, c, aa, bb = to_device(inst, torch, bf16=True)
    h = dlm_lib.Solver(rp, col, c, aa, bb, inst.J, bf16=True)
    with pytest.raises(dlm_lib.DlmError) as e:
        dlm_lib.Batch([a, h])
    assert e.value.status == dlm_lib.DLM_ERR_INVALID_ARG
    bt = dlm_lib.Batch([a, b])
    with pytest.raises(dlm_lib.DlmError) as e:
        bt.set_options(mapping=4)
    assert e.value.status == dlm_lib.DLM_ERR_INVALID_ARG
    with pytest.raises(dlm_lib.DlmError):
        bt.set_options(block_threads=256)
    bt.close()
    for s in (a, b, h):
        s.close()


@pytest.mark.parametrize("mapping,threads,coop", [(3, 0, 0), (3, 512, 0), (2, 0, 0), (1, 512, 0)])
def test_handle_mappings_are_bit_identical(dlm_lib, cases, alone, mapping, threads, coop):
    for k in (0, 3):
        inst, sched, pre = cases[k]
        s = make(dlm_lib, inst, sched, pre)
        s.set_options(precondition=pre, mapping=mapping, block_threads=threads, coop_max=coop)
        s.step(T)
        assert np.array_equal(lam_of(s).view(np.uint32), alone[k].view(np.uint32)), f"member {k} differs"
        s.close()


def test_wide_scan_batch_is_bit_identical_to_single_handles(dlm_lib, cases):
    # topk = 8 (eight values tracked in the first pass) on every member: the
    # batch (dynamic units) and each handle alone (interleaved slices) agree
    # bit for bit, as with the default scan
    alone8 = []
    for inst, sched, pre in cases:
        s = make(dlm_lib, inst, sched, pre)
        s.set_options(precondition=pre, topk=8)
        s.step(T)
        alone8.append(lam_of(s))
        s.close()
    solvers = [make(dlm_lib, *c) for c in cases]
    for s, c in zip(solvers, cases):
        s.set_options(precondition=c[2], topk=8)
    bt = dlm_lib.Batch(solvers)
    bt.set_options(mapping=3, topk=8)
    bt.step(T)
    for k, s in enumerate(solvers):
        assert np.array_equal(lam_of(s).view(np.uint32), alone8[k].view(np.uint32)), f"member {k} differs"
    bt.close()
    for s in solvers:
        s.close()
