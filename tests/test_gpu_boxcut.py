"""The box cut by one budget, {0 <= x_ij <= z, sum_j x_ij <= cut} (the
reading of Table 1's box-cut projection), on the GPU against the FP64
oracle: one dual evaluation at several gammas, the accelerated trajectory,
the certificate, the reduction to the box when the budget is slack (the same
bits), batches of box-cut handles (the same bits as alone), and the
combinations the build does not take."""
import numpy as np
import pytest

import oracle
from gpu_cases import mixed_instance, tiny_instance, to_device, x_error_report

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def solver(dlm, inst, z, cut, bf16=False):
    rp, col, c, a, b = to_device(inst, torch, bf16)
    return dlm.Solver(rp, col, c, a, b, inst.J, kind=dlm.DLM_BOX_CUT, z=z, cut=cut, bf16=bf16)


def oproblem(inst, z, cut):
    return oracle.Problem(inst.row_ptr, inst.col, inst.c.astype(np.float64), inst.a.astype(np.float64), inst.b,
                          inst.J, oracle.BOX_CUT, z, cut=cut)


@pytest.mark.parametrize("z,cut", [(0.3, 0.5), (0.25, 1.5), (1.0, 0.6)])
@pytest.mark.parametrize("gamma", [1e-1, 1e-2, 1e-3])
def test_calculate_matches_oracle(dlm_lib, z, cut, gamma):
    inst = mixed_instance()
    s = solver(dlm_lib, inst, z, cut)
    p = oproblem(inst, z, cut)
    rng = np.random.default_rng(11)
    for scale in (0.3, 1.0, 2.5):
        lam32 = (rng.uniform(0, 1, inst.J) * scale).astype(np.float32)
        lam32[rng.uniform(size=inst.J) < 0.2] = 0.0
        lam = lam32.astype(np.float64)
        g, grad, x = s.calculate(torch.from_numpy(lam32).cuda(), gamma)
        ref = oracle.sweep(p, lam, gamma)
        # the threshold depends on which edges sit at the cap as well as on
        # which are positive: both decisions are taken in FP32
        dx, tol = x_error_report(x.cpu().numpy(), ref["x"], p, lam, gamma, cap=z)
        assert (dx <= tol).all(), f"{int((dx > tol).sum())} edges over tolerance, max {dx.max():.3e}"
        scale_j = np.bincount(p.col, weights=p.a * ref["x"], minlength=p.J) + np.abs(p.b)
        allow = np.bincount(p.col, weights=p.a * np.maximum(tol - 2e-6 * p.z, 0), minlength=p.J)
        dg = np.abs(grad.cpu().numpy().astype(np.float64) - ref["grad"])
        assert (dg <= 2e-6 * scale_j + allow + 1e-6).all(), f"grad max err {dg.max():.3e}"
        assert abs(g - ref["g"]) <= 2e-6 * (abs(ref["g"]) + abs(ref["obj"]) + 1e-9) + float(np.abs(p.c) @ tol)
        if scale == 0.3:  # low prices: the budget binds on some rows or the box on some edges
            sums = np.add.reduceat(ref["x"], p.row_ptr[:-1][np.diff(p.row_ptr) > 0])
            budget, box = (sums > cut * (1 - 1e-9)).any(), (ref["x"] > z * (1 - 1e-12)).any()
            assert budget or box
            if z >= cut:  # the box cannot bind: the inequality simplex of radius cut
                assert budget and not box
    s.close()


def test_slack_budget_gives_the_box_bitwise(dlm_lib):
    inst = mixed_instance(seed=5, I=3000, J=300)
    rp, col, c, a, b = to_device(inst, torch)
    box = dlm_lib.Solver(rp, col, c, a, b, inst.J, kind=dlm_lib.DLM_BOX, z=0.4)
    bc = dlm_lib.Solver(rp, col, c, a, b, inst.J, kind=dlm_lib.DLM_BOX_CUT, z=0.4, cut=1e6)
    lam = torch.from_numpy(np.random.default_rng(2).uniform(0, 1, inst.J).astype(np.float32)).cuda()
    g1, grad1, x1 = box.calculate(lam, 1e-2)
    g2, grad2, x2 = bc.calculate(lam, 1e-2)
    assert torch.equal(x1, x2) and torch.equal(grad1, grad2)
    assert abs(g1 - g2) <= 1e-12 * abs(g1)
    box.close()
    bc.close()


@pytest.mark.parametrize("precondition", [True, False])
def test_trajectory_matches_oracle(dlm_lib, precondition):
    inst = tiny_instance()
    z, cut = 0.3, 0.5
    s = solver(dlm_lib, inst, z, cut)
    s.set_schedule(1e-2)
    s.set_options(precondition=precondition)
    T = 150
    s.step(T)
    lam = s.lam().cpu().numpy().astype(np.float64)
    out = oracle.fista(oproblem(inst, z, cut), T, 1e-2, precondition=precondition)
    ref = out["lam"]
    err = np.abs(lam - ref).max()
    assert err <= 1e-5 * max(np.abs(ref).max(), 1e-6), f"max err {err:.3e}"
    g = s.trajectory(0, T)
    assert np.abs(g - out["g_traj"]).max() <= 1e-5 * np.abs(out["g_traj"]).max()
    assert ref.max() > 1e-3
    s.close()


def test_solve_and_certificate(dlm_lib):
    inst = mixed_instance(seed=12, I=3000, J=300)
    z, cut = 0.35, 0.8
    s = solver(dlm_lib, inst, z, cut)
    s.set_schedule(1e-1, 1e-2, 0.5, 50)
    s.set_options(precondition=True, gap_every=20, restart=True)
    st = s.solve(1e-4, 20000)
    assert st.status == dlm_lib.DLM_OK and st.rel_gap <= 1e-4
    lam = s.lam().cpu().numpy().astype(np.float64)
    p = oproblem(inst, z, cut)
    cert = oracle.certify(p, lam, 1e-2)
    assert abs(st.dual_obj - cert["g"]) <= 2e-6 * abs(cert["g"])
    assert abs(st.primal_obj - cert["primal"]) <= 2e-6 * abs(cert["primal"])
    assert cert["rel_gap"] <= 1.5e-4
    x = s.x().cpu().numpy().astype(np.float64)
    assert (x >= 0).all() and (x <= z * (1 + 1e-6)).all()
    assert (np.add.reduceat(x, inst.row_ptr[:-1][np.diff(inst.row_ptr) > 0]) <= cut * (1 + 1e-5)).all()
    s.close()


def test_unsupported_combinations_and_bad_values(dlm_lib):
    inst = tiny_instance()
    s = solver(dlm_lib, inst, 0.3, 0.5)
    with pytest.raises(dlm_lib.DlmError) as e:
        s.set_count_limit(100.0)
    assert e.value.status == dlm_lib.DLM_ERR_UNSUPPORTED
    rp, col, c, a, b = to_device(inst, torch)
    plain = dlm_lib.Solver(rp, col, c, a, b, inst.J)
    with pytest.raises(dlm_lib.DlmError) as e:  # box-cut members batch only with each other
        dlm_lib.Batch([s, plain])
    assert e.value.status == dlm_lib.DLM_ERR_UNSUPPORTED
    plain.close()
    s.close()
    for bad in (0.0, -1.0, float("inf"), float("nan")):
        with pytest.raises(dlm_lib.DlmError) as e:
            solver(dlm_lib, inst, 0.3, bad)
        assert e.value.status == dlm_lib.DLM_ERR_INVALID_ARG


def test_batch_of_box_cut_members_is_bit_identical(dlm_lib):
    insts = [tiny_instance(), mixed_instance(seed=9, I=2500, J=200)]
    sets = [(0.3, 0.5), (0.25, 0.8)]

    def members():
        out = []
        for inst, (z, cut), pre in zip(insts, sets, (True, False)):
            s = solver(dlm_lib, inst, z, cut)
            s.set_schedule(1e-2)
            s.set_options(precondition=pre)
            out.append(s)
        return out

    alone = members()
    for s in alone:
        s.step(80)
    together = members()
    bt = dlm_lib.Batch(together)
    bt.step(80)
    for s0, s1 in zip(alone, together):
        assert torch.equal(s0.lam(), s1.lam())
    st = bt.stats()
    for x, s0 in zip(st, alone):
        assert x.status == dlm_lib.DLM_OK
        assert abs(x.dual_obj - s0.stats().dual_obj) <= 1e-12 * abs(x.dual_obj)
    bt.close()
    for s in alone + together:
        s.close()
