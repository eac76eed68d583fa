"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances (derived from the FP32 arithmetic of the per-edge path):
  x      |dx| <= 2e-6 z + 4 u x_ref, except on users with an edge within FP32
         resolution of the simplex threshold (the active set is decided in
         FP32 there), where |dx| <= 16 u (|c| + |a lam|) / gamma; u = 2^-24.
  grad   |dG_j| <= 2e-6 (sum_i a_ij x_ij + b_j) + the same border allowance
         summed over the item's edges.
  g      relative 2e-6.
  lam    after T iterations: |dlam|_inf <= 1e-5 max(|lam_ref|_inf, 1e-6).
  g(y_t) along the iteration: at the solver's own point, relative 2e-6 as g;
         against the oracle's trajectory (whose points y_t differ from the
         solver's by the lam tolerance), relative 1e-5.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_cases import (EPS32, mixed_instance, oracle_problem, tiny_instance, to_device, with_empty_users,
                       x_error_report)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def solver_for(dlm, inst, kind=oracle.SIMPLEX_LE, z=1.0, bf16=False):
    rp, col, c, a, b = to_device(inst, torch, bf16)
    return dlm.Solver(rp, col, c, a, b, inst.J, kind=kind, z=z, bf16=bf16)


CASES = [
    ("tiny", "f32", oracle.SIMPLEX_LE, 1e-2),
    ("mixed", "f32", oracle.SIMPLEX_LE, 1e-1),
    ("mixed", "f32", oracle.SIMPLEX_LE, 1e-3),
    ("mixed", "bf16", oracle.SIMPLEX_LE, 1e-2),
    ("mixed", "f32", oracle.SIMPLEX_EQ, 1e-2),
    ("mixed", "f32", oracle.BOX, 1e-2),
]


@pytest.mark.parametrize("name,dtype,kind,gamma", CASES)
def test_calculate_matches_oracle(dlm_lib, name, dtype, kind, gamma):
    bf16 = dtype == "bf16"
    inst = tiny_instance() if name == "tiny" else mixed_instance(bf16=False)
    s = solver_for(dlm_lib, inst, kind, 1.0, bf16)
    p = oracle_problem(inst, kind, 1.0, bf16)
    rng = np.random.default_rng(17)
    for trial in range(3):
        scale = [0.3, 1.0, 2.5][trial]
        lam32 = (rng.uniform(0, 1, size=inst.J) * scale).astype(np.float32)
        lam32[rng.uniform(size=inst.J) < 0.2] = 0.0
        lam = lam32.astype(np.float64)
        g, grad, x = s.calculate(torch.from_numpy(lam32).cuda(), gamma)
        ref = oracle.sweep(p, lam, gamma)
        xg = x.cpu().numpy()
        dx, tol = x_error_report(xg, ref["x"], p, lam, gamma)
        bad = dx > tol
        assert not bad.any(), (f"x: {bad.sum()} edges over tolerance; max dx {dx.max():.3e}; "
                               f"bulk max {np.median(dx):.3e}")
        # gradient: exact fixed-point sums of FP32 products
        gref = ref["grad"]
        scale_j = np.bincount(p.col, weights=p.a * ref["x"], minlength=p.J) + np.abs(p.b)
        allow = np.bincount(p.col, weights=p.a * np.maximum(tol - 2e-6, 0), minlength=p.J)
        dg = np.abs(grad.cpu().numpy().astype(np.float64) - gref)
        assert (dg <= 2e-6 * scale_j + allow + 1e-6).all(), f"grad max err {dg.max():.3e}"
        assert abs(g - ref["g"]) <= 2e-6 * (abs(ref["g"]) + abs(ref["obj"]) + 1e-9), (g, ref["g"])
    s.close()


def test_trajectory_tiny_500_iterations(dlm_lib):
    # 10,000 users x 100 items, gamma = 1e-2 fixed, lam0 = 0, 500 accelerated
    # steps of size 1/L, L = max_j sum_i a_ij^2 / gamma.
    inst = tiny_instance()
    s = solver_for(dlm_lib, inst)
    s.set_schedule(1e-2)
    s.step(500)
    lam = s.lam().cpu().numpy().astype(np.float64)
    p = oracle_problem(inst)
    ref = oracle.fista(p, 500, 1e-2, trajectory=False)["lam"]
    err = np.abs(lam - ref).max()
    assert err <= 1e-5 * max(np.abs(ref).max(), 1e-6), f"lam_500 max err {err:.3e} (|lam| {np.abs(ref).max():.3f})"
    # x(lam_T) and g(lam_T) at the solver's own iterate
    g, _, x = s.calculate(torch.from_numpy(lam.astype(np.float32)).cuda(), 1e-2)
    sw = oracle.sweep(p, lam, 1e-2)
    dx, tol = x_error_report(x.cpu().numpy(), sw["x"], p, lam, 1e-2)
    assert (dx <= tol).all()
    assert abs(g - sw["g"]) <= 2e-6 * abs(sw["g"])
    s.close()


@pytest.mark.parametrize("precondition", [False, True])
def test_trajectory_with_continuation(dlm_lib, precondition):
    # gamma 1e-1 -> 1e-3 halved every 20 iterations (the production schedule
    # compressed), momentum restart at each stage change.
    inst = mixed_instance(seed=5, I=3000, J=300)
    s = solver_for(dlm_lib, inst)
    s.set_schedule(1e-1, 1e-3, 0.5, 20)
    s.set_options(precondition=precondition)
    T = 200
    s.step(T)
    lam = s.lam().cpu().numpy().astype(np.float64)
    _, _, st = s.get_state()
    p = oracle_problem(inst)
    ref = oracle.fista(p, T, 1e-1, 1e-3, 0.5, 20, precondition=precondition)
    err = np.abs(lam - ref["lam"]).max()
    print(f"continuation precondition={precondition}: max |dlam| / |lam| = "
          f"{err / max(np.abs(ref['lam']).max(), 1e-6):.3e}")
    assert err <= 1e-5 * max(np.abs(ref["lam"]).max(), 1e-6), f"max err {err:.3e}"
    assert st.iter == T and st.stage == T // 20
    g = s.trajectory(0, T)
    rel = np.abs(g - ref["g_traj"]) / np.abs(ref["g_traj"])
    print(f"continuation precondition={precondition}: max rel |dg(y_t)| = {rel.max():.3e}")
    assert rel.max() <= 1e-5, f"g trajectory: max rel err {rel.max():.3e} at t = {rel.argmax()}"
    s.close()


def test_long_schedule_past_64_stages(dlm_lib):
    # gamma 1e-1 -> 1e-3 by a factor 0.95 every 5 iterations: 90 stage
    # changes (each restarts the momentum) before gamma reaches gamma_end at
    # iteration 450, then 150 iterations there.
    inst = mixed_instance(seed=5, I=3000, J=300)
    s = solver_for(dlm_lib, inst)
    s.set_schedule(1e-1, 1e-3, 0.95, 5)
    T = 600
    s.step(T)
    lam = s.lam().cpu().numpy().astype(np.float64)
    p = oracle_problem(inst)
    ref = oracle.fista(p, T, 1e-1, 1e-3, 0.95, 5)
    assert oracle.stage_gamma(1e-1, 1e-3, 0.95, 89) > 1e-3 and oracle.stage_gamma(1e-1, 1e-3, 0.95, 90) == 1e-3
    err = np.abs(lam - ref["lam"]).max()
    print(f"95-stage schedule: max |dlam| / |lam| = {err / max(np.abs(ref['lam']).max(), 1e-6):.3e}")
    assert err <= 1e-5 * max(np.abs(ref["lam"]).max(), 1e-6), f"max err {err:.3e}"
    _, _, st = s.get_state()
    assert st.iter == T and st.stage == T // 5
    g = s.trajectory(0, T)
    assert np.abs(g - ref["g_traj"]).max() <= 1e-5 * np.abs(ref["g_traj"]).max()
    assert s.stats().gamma == 1e-3
    s.close()
    # the same schedule driven to a certified gap (row normalization and the
    # adaptive restart: the plain step 1/L is set by the largest item and is
    # far too short for this heavy-tailed instance at gamma = 1e-3)
    s = solver_for(dlm_lib, inst)
    s.set_schedule(1e-1, 1e-3, 0.95, 5)
    s.set_options(precondition=True, restart=True, gap_every=25)
    out = s.solve(1e-4, 20000)
    assert out.converged and out.status == dlm_lib.DLM_OK and out.rel_gap <= 1e-4 and out.gamma == 1e-3
    assert out.iter >= 450  # gamma reaches gamma_end at iteration 450
    s.close()


def test_schedules_that_never_reach_gamma_end_are_rejected(dlm_lib):
    inst = mixed_instance(seed=5, I=500, J=60)
    s = solver_for(dlm_lib, inst)
    with pytest.raises(dlm_lib.DlmError) as e:
        s.set_schedule(1e-1, 1e-3, 1.0, 5)
    assert e.value.status == dlm_lib.DLM_ERR_INVALID_ARG
    with pytest.raises(dlm_lib.DlmError) as e:  # about 4.6 million stages
        s.set_schedule(1e-1, 1e-3, 1.0 - 1e-6, 5)
    assert e.value.status == dlm_lib.DLM_ERR_UNSUPPORTED
    s.set_schedule(1e-2, 1e-2, 1.0, 5)  # a fixed ridge with factor 1 is fine
    s.step(3)
    assert s.stats().gamma == 1e-2
    s.close()


def test_dual_objective_along_the_iteration(dlm_lib):
    # Every iteration records g(y_t) from the sweep's fixed-point objective
    # and an FP64 dot product: at the solver's own points it is the oracle's
    # g at the FP32 copy of y_t the sweep read; along the run it follows the
    # oracle's trajectory.
    inst = tiny_instance()
    s = solver_for(dlm_lib, inst)
    s.set_schedule(1e-2)
    p = oracle_problem(inst)
    T = 500
    ys = {}
    for t in range(T):
        if t in (0, 1, 2, 7, 50, 200, T - 1):
            _, y, _ = s.get_state()
            ys[t] = y.cpu().numpy()
        s.step(1)
    g = s.trajectory(0, T)
    for t, y in ys.items():
        y32 = y.astype(np.float32).astype(np.float64)
        ref = oracle.sweep(p, y32, 1e-2, want_x=False)
        assert abs(g[t] - ref["g"]) <= 2e-6 * (abs(ref["g"]) + abs(ref["obj"])), (t, g[t], ref["g"])
    ref = oracle.fista(p, T, 1e-2)["g_traj"]
    rel = np.abs(g - ref) / np.abs(ref)
    print(f"tiny trajectory: max rel |dg(y_t)| = {rel.max():.3e}")
    assert rel.max() <= 1e-5
    # the same iterations replayed through CUDA graphs give the same bits
    s2 = solver_for(dlm_lib, inst)
    s2.set_schedule(1e-2)
    s2.step(T)
    assert np.array_equal(s2.trajectory(0, T), g)
    with pytest.raises(dlm_lib.DlmError):
        s2.trajectory(T - 5, 10)  # beyond the current iteration
    s2.set_schedule(1e-2)
    with pytest.raises(dlm_lib.DlmError):
        s2.trajectory(0, 1)  # a new schedule starts a new record
    s.close()
    s2.close()


def test_trajectory_with_adaptive_restart(dlm_lib):
    # Fixed gamma, row normalization and the adaptive momentum restart on the
    # 10,000 x 100 instance.  The restart test is a sign decision on an FP64
    # sum that both sides make on their own (FP32 and FP64) iterates; here no
    # decision sits within rounding of zero, so the trajectories agree to the
    # FP32 tolerance and the same restarts fire.
    inst = tiny_instance()
    s = solver_for(dlm_lib, inst)
    s.set_schedule(1e-2)
    s.set_options(precondition=True, restart=True)
    T = 300
    s.step(T)
    lam = s.lam().cpu().numpy().astype(np.float64)
    p = oracle_problem(inst)
    ref = oracle.fista(p, T, 1e-2, precondition=True, restart=True, trajectory=False)
    _, _, st = s.get_state()
    assert st.theta == pytest.approx(ref["theta"], rel=1e-12)
    err = np.abs(lam - ref["lam"]).max()
    assert err <= 1e-5 * max(np.abs(ref["lam"]).max(), 1e-6), f"max err {err:.3e}"
    s.close()


def test_adaptive_restart_converges_to_the_oracle_optimum(dlm_lib):
    # On a heavier instance a restart decision can fall within rounding of
    # zero and then fire one step apart on the two sides, after which the
    # trajectories differ by more than rounding.  What is fixed is the limit,
    # so both runs are driven to convergence and compared there: the dual
    # value, the FP64 certificate of the GPU's own iterate and lam (the
    # iterate is FP64 on both sides; the GPU's gradient carries the FP32
    # per-edge arithmetic, measured 7e-8 relative in lam at the limit).
    inst = mixed_instance(seed=6, I=1500, J=150)
    s = solver_for(dlm_lib, inst)
    s.set_schedule(1e-2)
    s.set_options(precondition=True, restart=True)
    T = 2500
    s.step(T)
    lam = s.lam().cpu().numpy().astype(np.float64)
    p = oracle_problem(inst)
    ref = oracle.fista(p, T, 1e-2, precondition=True, restart=True, trajectory=False)["lam"]
    cert_ref = oracle.certify(p, ref, 1e-2)
    assert cert_ref["rel_gap"] <= 1e-7  # the reference has converged
    assert oracle.certify(p, lam, 1e-2)["rel_gap"] <= 1e-6
    g, _, _ = s.calculate(torch.from_numpy(lam.astype(np.float32)).cuda(), 1e-2, want_grad=False, want_x=False)
    assert abs(g - cert_ref["g"]) <= 1e-5 * abs(cert_ref["g"])
    err = np.abs(lam - ref).max()
    print(f"restart at convergence: max |dlam| / |lam| = {err / max(np.abs(ref).max(), 1e-6):.3e}, "
          f"certified gap of the solver's iterate {oracle.certify(p, lam, 1e-2)['rel_gap']:.3e}")
    assert err <= 1e-5 * max(np.abs(ref).max(), 1e-6), f"max err {err:.3e}"
    s.close()


def test_certificate_matches_oracle(dlm_lib):
    inst = mixed_instance(seed=8, I=3000, J=400)
    s = solver_for(dlm_lib, inst)
    s.set_schedule(1e-2)
    s.set_options(precondition=True)
    s.step(60)
    st = s.stats()
    lam = s.lam().cpu().numpy().astype(np.float64)
    ref = oracle.certify(oracle_problem(inst), lam, 1e-2)
    assert abs(st.dual_obj - ref["g"]) <= 2e-6 * abs(ref["g"])
    assert abs(st.primal_obj - ref["primal"]) <= 2e-6 * abs(ref["primal"])
    assert abs(st.rel_gap - ref["rel_gap"]) <= 1e-5 * max(1.0, abs(ref["rel_gap"])) + 4e-6
    assert st.rel_gap >= -1e-9
    assert abs(st.max_viol - ref["max_viol"]) <= 1e-5 * (1 + abs(ref["max_viol"]))
    assert st.iter == 60
    s.close()


def test_repeated_runs_are_bit_identical(dlm_lib):
    inst = mixed_instance(seed=9, I=5000, J=500)
    lams = []
    for rep in range(5):
        s = solver_for(dlm_lib, inst)
        s.set_schedule(1e-1, 1e-2, 0.5, 15)
        s.set_options(graph_iters=[10, 7, 1, 10, 3][rep])
        s.step(80)
        lams.append(s.lam().cpu().numpy())
        s.close()
    for l in lams[1:]:
        assert np.array_equal(l.view(np.uint32), lams[0].view(np.uint32))


def test_host_and_device_inputs_agree_bitwise(dlm_lib):
    inst = mixed_instance(seed=10, I=2000, J=200)
    s1 = solver_for(dlm_lib, inst)
    s2 = dlm_lib.Solver(inst.row_ptr, inst.col, inst.c, inst.a, inst.b, inst.J)
    for s in (s1, s2):
        s.set_schedule(5e-2)
        s.step(40)
    assert np.array_equal(s1.lam().cpu().numpy().view(np.uint32), s2.lam().cpu().numpy().view(np.uint32))
    s1.close()
    s2.close()


def test_checkpoint_resume(dlm_lib):
    inst = mixed_instance(seed=11, I=2000, J=300)
    s = solver_for(dlm_lib, inst)
    s.set_schedule(1e-1, 1e-2, 0.5, 10)
    s.step(25)
    lam, y, st = s.get_state()
    s.step(30)
    want = s.lam().cpu().numpy()
    s.set_state(lam, y, st)
    s.step(30)
    assert np.array_equal(s.lam().cpu().numpy().view(np.uint32), want.view(np.uint32))
    s.close()


def test_warm_start_and_slack_instance(dlm_lib):
    # All capacities slack: lam stays exactly 0 and x = Proj(-c / gamma).
    inst = mixed_instance(seed=12, I=1500, J=150)
    inst.b = np.bincount(inst.col, weights=inst.a, minlength=inst.J) + 1.0
    s = solver_for(dlm_lib, inst)
    s.set_schedule(1e-2)
    s.step(20)
    assert (s.lam().cpu().numpy() == 0).all()
    st = s.solve(1e-9, 100)
    assert st.converged and st.rel_gap <= 1e-9
    s.set_lambda(torch.full((inst.J,), 0.5, device="cuda"))
    assert (s.lam().cpu().numpy() == 0.5).all()
    s.close()


def test_degree_classes_and_edge_cases(dlm_lib):
    # one item, users with 0 and 1 edges, a single user of degree J
    J = 1
    rp = np.array([0, 0, 1, 1, 2, 3], dtype=np.int64)
    col = np.zeros(3, np.int32)
    c = np.array([-1.0, -0.5, -0.2], np.float32)
    a = np.ones(3, np.float32)
    b = np.array([0.5])
    inst = synth.Instance(rp, col, c, a, b, J)
    s = solver_for(dlm_lib, inst)
    s.set_schedule(0.1)
    s.step(3000)
    p = oracle_problem(inst)
    ref = oracle.fista(p, 3000, 0.1, trajectory=False)["lam"]
    np.testing.assert_allclose(s.lam().cpu().numpy(), ref, rtol=1e-5, atol=1e-7)
    s.close()
    # one user with every item (degree 1500 > 512: the streamed-row mapping)
    Jb = 1500
    rng = np.random.default_rng(3)
    rp = np.array([0, Jb], np.int64)
    inst = synth.Instance(rp, np.arange(Jb, dtype=np.int32), (-rng.uniform(0, 1, Jb)).astype(np.float32),
                          np.ones(Jb, np.float32), np.full(Jb, 0.01), Jb)
    s = solver_for(dlm_lib, inst)
    p = oracle_problem(inst)
    lam32 = rng.uniform(0, 0.3, Jb).astype(np.float32)
    for gamma in (1.0, 1e-2, 1e-4):
        g, grad, x = s.calculate(torch.from_numpy(lam32).cuda(), gamma)
        ref = oracle.sweep(p, lam32.astype(np.float64), gamma)
        dx, tol = x_error_report(x.cpu().numpy(), ref["x"], p, lam32.astype(np.float64), gamma)
        assert (dx <= tol).all(), dx.max()
    s.close()


@pytest.mark.parametrize("what", ["item", "rowptr", "nan", "negb", "dup_short", "dup_long", "dup_last"])
def test_invalid_inputs_are_rejected(dlm_lib, what):
    inst = mixed_instance(seed=13, I=300, J=50)
    rp, col, c, a, b = [v.copy() if hasattr(v, "copy") else v for v in
                        (inst.row_ptr, inst.col, inst.c, inst.a, inst.b)]
    deg = np.diff(rp)
    if what == "item":
        col[7] = inst.J
    elif what == "rowptr":
        rp[5], rp[6] = rp[6], rp[5] - 1
    elif what == "nan":
        c[3] = np.nan
    elif what == "negb":
        b[2] = -1.0
    elif what == "dup_short":  # a row of 2..32 edges (compared across lanes)
        u = int(np.flatnonzero((deg >= 5) & (deg <= 32))[3])
        col[rp[u] + 4] = col[rp[u] + 1]
    elif what == "dup_long":  # a row of more than 32 edges (the bitmap path)
        u = int(np.flatnonzero(deg > 40)[0])
        col[rp[u + 1] - 1] = col[rp[u]]
    else:  # the last row of the instance
        u = int(np.flatnonzero(deg >= 2)[-1])
        col[rp[u + 1] - 1] = col[rp[u + 1] - 2]
    with pytest.raises(dlm_lib.DlmError) as e:
        dlm_lib.Solver(rp, col, c, a, b, inst.J)
    assert e.value.status == dlm_lib.DLM_ERR_INVALID_ARG
