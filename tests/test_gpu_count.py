"""The global count constraint sum x <= M (Sec. 5's example of a new coupling
constraint) on the GPU against the FP64 oracle: one dual evaluation, the
accelerated trajectory, the certificate, batches, and the slack limit.
Tolerances are those of the capacity-only parity tests (FP32 per-edge
arithmetic, exact fixed-point sums)."""
import math

import numpy as np
import pytest

import oracle
from gpu_cases import mixed_instance, oracle_problem, tiny_instance, to_device, x_error_report

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def solver(dlm, inst, kind=oracle.SIMPLEX_LE, M=None, bf16=False):
    rp, col, c, a, b = to_device(inst, torch, bf16)
    s = dlm.Solver(rp, col, c, a, b, inst.J, kind=kind, bf16=bf16)
    if M is not None:
        s.set_count_limit(M)
    return s


def oproblem(inst, kind, M, bf16=False):
    p = oracle_problem(inst, kind, 1.0, bf16)
    return oracle.Problem(p.row_ptr, p.col, p.c, p.a, p.b, p.J, kind, 1.0, M=M)


@pytest.mark.parametrize("kind", [oracle.SIMPLEX_LE, oracle.BOX])
@pytest.mark.parametrize("gamma", [1e-1, 1e-2])
def test_calculate_with_count_dual(dlm_lib, kind, gamma):
    inst = mixed_instance()
    M = 1500.0
    s = solver(dlm_lib, inst, kind, M)
    p = oproblem(inst, kind, M)
    rng = np.random.default_rng(4)
    for mu in (0.0, 0.05, 0.4):
        lam32 = np.append(rng.uniform(0, 1, inst.J), mu).astype(np.float32)
        g, grad, x = s.calculate(torch.from_numpy(lam32).cuda(), gamma)
        lam = lam32.astype(np.float64)
        ref = oracle.sweep(p, lam, gamma)
        # the count dual shifts every u by mu: the x tolerance is that of the
        # capacity-only parity test at the shifted costs
        pc = oracle.Problem(p.row_ptr, p.col, p.c + mu, p.a, p.b, p.J, kind, 1.0)
        dx, tol = x_error_report(x.cpu().numpy(), ref["x"], pc, lam[:-1], gamma)
        assert (dx <= tol).all(), f"mu {mu}: {int((dx > tol).sum())} edges over tolerance, max {dx.max():.3e}"
        gg = grad.cpu().numpy().astype(np.float64)
        assert gg.shape == (inst.J + 1,)
        # sum x is an exact sum of the FP32 x: its error is at most the sum of
        # the per-edge x tolerances, and mu times that enters g
        assert abs(gg[-1] - ref["grad"][-1]) <= tol.sum() + 1e-6
        assert abs(g - ref["g"]) <= 2e-6 * abs(ref["g"]) + mu * tol.sum()
    s.close()


@pytest.mark.parametrize("precondition", [True, False])
def test_trajectory_with_count(dlm_lib, precondition):
    inst = tiny_instance()
    # the capacities admit about 3,700 units of x at the capacity-only
    # optimum; M = 3,000 binds
    M = 3000.0
    s = solver(dlm_lib, inst, oracle.SIMPLEX_LE, M)
    s.set_schedule(1e-2)
    s.set_options(precondition=precondition)
    T = 400
    s.step(T)
    lam = s.lam().cpu().numpy().astype(np.float64)
    p = oproblem(inst, oracle.SIMPLEX_LE, M)
    out = oracle.fista(p, T, 1e-2, precondition=precondition)
    ref = out["lam"]
    assert lam.shape == (inst.J + 1,)
    err = np.abs(lam - ref).max()
    print(f"count precondition={precondition}: max |dlam| / |lam| = {err / max(np.abs(ref).max(), 1e-6):.3e}")
    assert err <= 1e-5 * max(np.abs(ref).max(), 1e-6), f"max err {err:.3e}"
    # the dual objective along the run includes the count term mu (sum x - M)
    g = s.trajectory(0, T)
    assert np.abs(g - out["g_traj"]).max() <= 1e-5 * np.abs(out["g_traj"]).max()
    if precondition:
        assert ref[-1] > 1e-3  # the count row binds
    s.close()


def test_certificate_and_solve_with_count(dlm_lib):
    inst = mixed_instance(seed=8, I=3000, J=300)
    M = 900.0
    s = solver(dlm_lib, inst, oracle.SIMPLEX_LE, M)
    s.set_schedule(1e-1, 1e-2, 0.5, 50)
    s.set_options(precondition=True, gap_every=20, restart=True)
    st = s.solve(1e-4, 20000)
    assert st.status == dlm_lib.DLM_OK and st.rel_gap <= 1e-4
    lam = s.lam().cpu().numpy().astype(np.float64)
    p = oproblem(inst, oracle.SIMPLEX_LE, M)
    cert = oracle.certify(p, lam, 1e-2)
    assert abs(st.dual_obj - cert["g"]) <= 2e-6 * abs(cert["g"])
    assert abs(st.primal_obj - cert["primal"]) <= 2e-6 * abs(cert["primal"])
    assert cert["rel_gap"] <= 1.5e-4
    assert lam[-1] > 0 and oracle.sweep(p, lam, 1e-2, want_x=False)["count"] <= M * (1 + 1e-3)
    s.close()


def test_removed_count_limit_is_bit_identical(dlm_lib):
    inst = tiny_instance()
    a = solver(dlm_lib, inst)
    b = solver(dlm_lib, inst, M=5000.0)
    b.set_count_limit(math.inf)
    for s in (a, b):
        s.set_schedule(1e-2)
        s.set_options(precondition=True)
        s.step(150)
    assert torch.equal(a.lam(), b.lam())
    a.close()
    b.close()


def test_batch_with_count_member_is_bit_identical(dlm_lib):
    insts = [tiny_instance(), mixed_instance(seed=9, I=2500, J=200)]
    limits = [3000.0, None]

    def make():
        out = []
        for inst, M in zip(insts, limits):
            s = solver(dlm_lib, inst, M=M)
            s.set_schedule(1e-2)
            s.set_options(precondition=True)
            out.append(s)
        return out

    alone = make()
    for s in alone:
        s.step(120)
    members = make()
    bt = dlm_lib.Batch(members)
    bt.step(120)
    for s0, s1 in zip(alone, members):
        assert torch.equal(s0.lam(), s1.lam())
    st = bt.stats()
    assert all(x.status == dlm_lib.DLM_OK for x in st)
    bt.close()
    for s in alone + members:
        s.close()


def test_count_limit_rejects_bad_values(dlm_lib):
    s = solver(dlm_lib, tiny_instance())
    for bad in (-1.0, float("nan")):
        with pytest.raises(dlm_lib.DlmError) as e:
            s.set_count_limit(bad)
        assert e.value.status == dlm_lib.DLM_ERR_INVALID_ARG
    s.close()
