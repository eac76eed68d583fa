"""Pins for the oracle's accelerated projected dual ascent (Sec. 4.4 update on
lam >= 0; Sec. 6 gamma continuation; App. B.2 step 1/L and row
normalization): exact solutions by enumeration of active sets, hand-solved
fixtures, the LP limit, closed-form special cases and the FISTA rate bound.
CPU only."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))
RNG = np.random.default_rng(11)


def dense_qp(p):
    """The primal as min c^T x + gamma/2 ||x||^2 s.t. G x <= h (all inequalities)."""
    n = p.nnz
    rows, rhs, tags = [], [], []
    for k in range(n):  # -x <= 0
        r = np.zeros(n)
        r[k] = -1
        rows.append(r), rhs.append(0.0), tags.append(("pos", k))
    for i in range(p.I):  # sum_k x_ik <= z
        r = np.zeros(n)
        r[p.row_ptr[i]:p.row_ptr[i + 1]] = 1
        rows.append(r), rhs.append(p.z), tags.append(("user", i))
    for j in range(p.J):  # sum_i a_ij x_ij <= b_j
        r = np.where(p.col == j, p.a, 0.0)
        rows.append(r), rhs.append(p.b[j]), tags.append(("cap", j))
    return np.array(rows), np.array(rhs), tags


def solve_by_active_sets(p, gamma):
    """Enumerate every active set W of G x <= h; solve the KKT system
    [gamma I, G_W^T; G_W, 0] [x; mu] = [-c; h_W]; keep the primal-feasible
    candidate with mu >= 0 (unique for a strictly convex QP)."""
    G, h, tags = dense_qp(p)
    m, n = G.shape
    sols = []
    for r in range(0, n + 1):
        for W in itertools.combinations(range(m), r):
            W = list(W)
            K = np.zeros((n + r, n + r))
            K[:n, :n] = gamma * np.eye(n)
            K[:n, n:] = G[W].T
            K[n:, :n] = G[W]
            rhs = np.concatenate([-p.c, h[W]])
            try:
                sol = np.linalg.solve(K, rhs)
            except np.linalg.LinAlgError:
                continue
            if np.linalg.cond(K) > 1e12:
                continue
            x, mu = sol[:n], sol[n:]
            if (G @ x <= h + 1e-11).all() and (mu >= -1e-11).all():
                lam = np.zeros(p.J)
                for w, mv in zip(W, mu):
                    if tags[w][0] == "cap":
                        lam[tags[w][1]] = mv
                sols.append((x, lam))
    assert sols, "no KKT point found"
    x0 = sols[0][0]
    for x, _ in sols:
        np.testing.assert_allclose(x, x0, atol=1e-9)  # x* is unique
    return sols[0]


def tiny_problem(seed, I=3, J=2, b_scale=0.6):
    rng = np.random.default_rng(seed)
    row_ptr = np.arange(0, I * J + 1, J)
    col = np.tile(np.arange(J), I)
    c = -rng.uniform(0.2, 1.0, size=I * J)
    a = rng.uniform(0.5, 1.5, size=I * J)
    b = b_scale * rng.uniform(0.3, 1.0, size=J)
    return oracle.Problem(row_ptr, col, c, a, b, J)


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
@pytest.mark.parametrize("precondition", [False, True])
@pytest.mark.parametrize("restart", [False, True])
def test_converged_fista_matches_active_set_enumeration(seed, precondition, restart):
    p = tiny_problem(seed, b_scale=[0.6, 0.3, 6.0, 0.9][seed - 1])
    gamma = 0.1
    x_ref, lam_ref = solve_by_active_sets(p, gamma)
    out = oracle.fista(p, 30000, gamma, precondition=precondition, trajectory=False, restart=restart)
    np.testing.assert_allclose(out["lam"], lam_ref, atol=1e-9)
    g, grad, x = oracle.dual(p, out["lam"], gamma)
    np.testing.assert_allclose(x, x_ref, atol=1e-9)
    primal = p.c @ x_ref + 0.5 * gamma * x_ref @ x_ref
    np.testing.assert_allclose(g, primal, rtol=1e-10)  # strong duality (Sec. 3.2)


def test_enumeration_cases_cover_binding_and_slack():
    kinds = set()
    for seed, bs in [(1, 0.6), (2, 0.3), (3, 6.0), (4, 0.9)]:
        _, lam = solve_by_active_sets(tiny_problem(seed, b_scale=bs), 0.1)
        kinds |= {"binding" if v > 1e-9 else "slack" for v in lam}
    assert kinds == {"binding", "slack"}


def test_hand_solved_fixtures():
    with open(os.path.join(HERE, "golden", "hand_solved.json")) as f:
        cases = json.load(f)["cases"]
    for cs in cases:
        p = oracle.Problem(cs["row_ptr"], cs["col"], cs["c"], cs["a"], cs["b"], len(cs["b"]), cs["kind"], cs["z"])
        out = oracle.fista(p, 20000, cs["gamma"], trajectory=False)
        np.testing.assert_allclose(out["lam"], cs["lam"], atol=1e-9, err_msg=cs["name"])
        g, _, x = oracle.dual(p, out["lam"], cs["gamma"])
        np.testing.assert_allclose(x, cs["x"], atol=1e-9, err_msg=cs["name"])
        np.testing.assert_allclose(g, cs["primal"], rtol=1e-9, err_msg=cs["name"])


def test_lp_limit():
    # 0 <= P*_gamma - P*_LP <= gamma/2 * I * z^2 (||x_i||^2 <= z^2 on the simplex).
    scipy_opt = pytest.importorskip("scipy.optimize")
    r = synth.recipe_production(I=40, J=5, seed=3)
    r.deg_mean, r.deg_max = 3.0, 5
    inst = synth.generate(r)
    p = oracle.Problem.from_instance(inst)
    G, h, _ = dense_qp(p)
    lp = scipy_opt.linprog(p.c, A_ub=G, b_ub=h, bounds=[(None, None)] * p.nnz, method="highs")
    assert lp.status == 0
    for gamma in [0.1, 0.02, 0.005]:
        out = oracle.fista(p, 40000, gamma, precondition=True, trajectory=False)
        st = oracle.certify(p, out["lam"], gamma)
        assert st["rel_gap"] < 1e-7
        assert st["g"] >= lp.fun - 1e-9 and st["g"] <= lp.fun + 0.5 * gamma * p.I + 1e-9
        assert st["primal"] >= lp.fun - 1e-9


def test_all_capacities_slack_gives_zero_duals():
    r = synth.recipe_production(I=200, J=10, seed=8)
    r.deg_mean, r.deg_max = 4.0, 10
    inst = synth.generate(r)
    b = np.bincount(inst.col, weights=inst.a, minlength=inst.J) + 1.0  # >= sum_i a_ij * z
    p = oracle.Problem(inst.row_ptr, inst.col, inst.c, inst.a, b, inst.J)
    out = oracle.fista(p, 50, 0.05, trajectory=False)
    assert (out["lam"] == 0).all()
    _, _, x = oracle.dual(p, out["lam"], 0.05)
    for i in range(p.I):
        s, e = p.row_ptr[i], p.row_ptr[i + 1]
        ref, _ = oracle.project(-p.c[s:e] / 0.05, oracle.SIMPLEX_LE, 1.0)
        np.testing.assert_array_equal(x[s:e], ref)


def test_single_item_reduces_to_scalar_root():
    # J = 1, a = 1, every user eligible only for item 0:
    # x_i(lam) = clip(-(c_i + lam)/gamma, 0, 1) and lam* solves sum_i x_i(lam) = b.
    scipy_opt = pytest.importorskip("scipy.optimize")
    I, gamma = 500, 0.05
    c = -RNG.uniform(0, 1, size=I)
    b = 40.0
    p = oracle.Problem(np.arange(I + 1), np.zeros(I, np.int32), c, np.ones(I), [b], 1)
    f = lambda lam: np.clip(-(c + lam) / gamma, 0, 1).sum() - b  # noqa: E731
    lam_ref = scipy_opt.brentq(f, 0.0, 2.0, xtol=1e-15, rtol=1e-15)
    out = oracle.fista(p, 20000, gamma, trajectory=False)
    np.testing.assert_allclose(out["lam"][0], lam_ref, atol=1e-10)


def test_fista_rate_bound():
    # Beck & Teboulle (2009), Thm 4.4: g* - g(lam_t) <= 2 L ||lam_0 - lam*||^2 / (t+1)^2.
    p = tiny_problem(2, I=6, J=3, b_scale=0.4)
    gamma = 0.1
    L = oracle.row_sq(p).max() / gamma
    star = oracle.fista(p, 60000, gamma, trajectory=False)["lam"]
    gs = oracle.dual(p, star, gamma)[0]
    for t in [1, 2, 4, 8, 16, 32, 64, 128, 256]:
        lam_t = oracle.fista(p, t, gamma, trajectory=False)["lam"]
        gt = oracle.dual(p, lam_t, gamma)[0]
        assert gs - gt <= 2 * L * (star @ star) / (t + 1) ** 2 + 1e-12


def test_continuation_schedule_values():
    want = [0.1 * 2.0 ** -s for s in range(7)] + [1e-3, 1e-3]
    got = [oracle.stage_gamma(0.1, 1e-3, 0.5, s) for s in range(9)]
    np.testing.assert_allclose(got, want, rtol=1e-15)
    assert got[7] == 1e-3 and got[6] > 1e-3


def test_long_schedule_stages_follow_the_closed_form():
    # gamma_s = max(gamma_end, gamma_0 factor^s) for every stage, far past 64
    # stages (Sec. 6, App. B.2: the decay reaches gamma_end at stage 90 here)
    for s_ in (0, 1, 63, 64, 65, 89, 90, 91, 500):
        want = max(1e-3, 1e-1 * 0.95 ** s_)
        assert abs(oracle.stage_gamma(1e-1, 1e-3, 0.95, s_) - want) <= 1e-15 * want, s_
    r = synth.recipe_production(I=200, J=10, seed=13)
    r.deg_mean, r.deg_max = 4.0, 10
    p = oracle.Problem.from_instance(synth.generate(r))
    run = oracle.fista(p, 500, 1e-1, 1e-3, 0.95, iters_per_stage=5)
    want = [max(1e-3, 1e-1 * 0.95 ** (t // 5)) for t in range(500)]
    np.testing.assert_allclose(run["gamma_traj"], want, rtol=1e-14)


def test_recorded_dual_value_is_g_at_the_swept_point():
    # g_traj[t] is the dual objective at the point the t-th sweep evaluates,
    # y_t (the momentum point that t iterations leave), at that iteration's gamma
    r = synth.recipe_production(I=300, J=12, seed=21)
    r.deg_mean, r.deg_max = 5.0, 12
    p = oracle.Problem.from_instance(synth.generate(r))
    full = oracle.fista(p, 60, 0.2, 0.05, 0.5, iters_per_stage=20)
    for t in (0, 1, 7, 19, 20, 21, 45, 59):
        y_t = oracle.fista(p, t, 0.2, 0.05, 0.5, iters_per_stage=20)["y"] if t > 0 else np.zeros(p.D)
        g = oracle.sweep(p, y_t, full["gamma_traj"][t], want_x=False)["g"]
        assert abs(full["g_traj"][t] - g) <= 1e-12 * max(1.0, abs(g)), t


def test_stage_change_warm_starts_and_resets_momentum():
    # Two stages run at once equal stage 1, then a fresh run of stage 2 from
    # stage 1's lam (theta reset to 1, y = lam): Sec. 6 warm start.
    r = synth.recipe_production(I=300, J=12, seed=9)
    r.deg_mean, r.deg_max = 5.0, 12
    p = oracle.Problem.from_instance(synth.generate(r))
    both = oracle.fista(p, 80, 0.2, 0.1, 0.5, iters_per_stage=40)
    s1 = oracle.fista(p, 40, 0.2)
    s2 = oracle.fista(p, 40, 0.1, lam0=s1["lam"])
    np.testing.assert_array_equal(both["lam"], s2["lam"])
    np.testing.assert_array_equal(both["g_traj"][:40], s1["g_traj"])
    np.testing.assert_array_equal(both["g_traj"][40:], s2["g_traj"])


def test_row_normalisation_equals_plain_method_on_scaled_rows():
    # App. B.2: A' = D A, b' = D b with D_jj = ||A_j||^-1 (so A'A'^T = I and
    # L' = 1/gamma).  The preconditioned iteration in lam equals the plain
    # iteration on the scaled problem, mapped back by lam = D lam'.
    r = synth.recipe_production(I=400, J=15, seed=10)
    r.deg_mean, r.deg_max = 5.0, 12
    inst = synth.generate(r)
    p = oracle.Problem.from_instance(inst)
    n2 = oracle.row_sq(p)
    d = 1.0 / np.sqrt(n2)
    ps = oracle.Problem(p.row_ptr, p.col, p.c, p.a * d[p.col], p.b * d, p.J)
    np.testing.assert_allclose(oracle.row_sq(ps), 1.0, rtol=1e-13)
    pre = oracle.fista(p, 200, 0.05, precondition=True)
    plain = oracle.fista(ps, 200, 0.05, precondition=False)
    np.testing.assert_allclose(pre["lam"], plain["lam"] * d, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(pre["g_traj"], plain["g_traj"], rtol=1e-11)


def test_adaptive_restart_fires_on_overshoot():
    """One item, one user, a = 1: the dual is a concave scalar function, so the
    accelerated iteration started far above the optimum overshoots it; the
    restart resets the momentum (theta back to 1) the first time a step opposes
    it, and without the restart theta keeps growing."""
    p = oracle.Problem(np.array([0, 1]), np.array([0], dtype=np.int32), np.array([-1.0]), np.array([1.0]),
                       np.array([0.3]), 1)
    gamma = 0.5
    # optimum: x = 0.3 binding, -(c + lam)/gamma = 0.3 -> lam* = 1 - 0.15 = 0.85
    plain = [oracle.fista(p, t, gamma, lam0=np.array([3.0]), trajectory=False) for t in range(1, 40)]
    rst = [oracle.fista(p, t, gamma, lam0=np.array([3.0]), trajectory=False, restart=True) for t in range(1, 40)]
    assert all(plain[k + 1]["theta"] > plain[k]["theta"] for k in range(len(plain) - 1))
    assert any(r["theta"] == 1.0 for r in rst[2:])
    assert abs(rst[-1]["lam"][0] - 0.85) < 1e-9 and abs(plain[-1]["lam"][0] - 0.85) < 1e-3


def test_threaded_timing_loop_is_the_same_iteration():
    """The threaded loop that times the CPU baseline runs the same fixed-gamma
    iteration; only the order of the per-item sums differs."""
    import synth

    inst = synth.generate(synth.recipe_tiny())
    p = oracle.Problem(inst.row_ptr, inst.col, inst.c.astype(np.float64), inst.a.astype(np.float64), inst.b,
                       inst.J)
    for pre in (False, True):
        ref = oracle.fista(p, 40, 1e-2, precondition=pre, trajectory=False)["lam"]
        for nt in (1, 3, 8):
            got = oracle.fista_threads(p, 40, 1e-2, precondition=pre, nthreads=nt)
            assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max()), (pre, nt)


@pytest.mark.parametrize("sched,precondition,restart", [((1e-1, 1e-2, 0.5, 30), True, False),
                                                         ((1e-2, 1e-2, 0.5, 0), False, True),
                                                         ((5e-2, 5e-3, 0.5, 20), True, True)])
def test_threaded_solve_is_the_fista_iteration(sched, precondition, restart):
    # one thread: orc_fista's arithmetic exactly; four threads: the same
    # iteration with the item sums added in another order
    inst = synth.generate(synth.recipe_production(I=1500, J=40, seed=23))
    p = oracle.Problem.from_instance(inst)
    T = 150
    ref = oracle.fista(p, T, sched[0], sched[1], sched[2], sched[3], precondition=precondition, restart=restart,
                       trajectory=False)["lam"]
    one = oracle.solve_threads(p, *sched, precondition=precondition, restart=restart, target=-1.0,
                               gap_every=10 ** 9, max_iters=T, nthreads=1)
    assert one["iters"] == T and np.array_equal(one["lam"], ref)
    four = oracle.solve_threads(p, *sched, precondition=precondition, restart=restart, target=-1.0,
                                gap_every=10 ** 9, max_iters=T, nthreads=4)
    assert np.abs(four["lam"] - ref).max() <= 1e-11 * max(np.abs(ref).max(), 1e-9)


def test_threaded_solve_stops_at_the_first_certified_check():
    inst = synth.generate(synth.recipe_production(I=1500, J=40, seed=24))
    p = oracle.Problem.from_instance(inst)
    sched = (1e-1, 1e-2, 0.5, 40)  # gamma_end from iteration 160
    out = oracle.solve_threads(p, *sched, precondition=True, target=1e-4, gap_every=25, max_iters=20000, nthreads=3)
    T = out["iters"]
    assert T % 25 == 0 and T >= 175 and out["rel_gap"] <= 1e-4
    lam = oracle.fista(p, T, *sched, precondition=True, trajectory=False)["lam"]
    cert = oracle.certify(p, lam, 1e-2)
    assert abs(cert["rel_gap"] - out["rel_gap"]) <= 1e-9 and abs(cert["g"] - out["g"]) <= 1e-9 * abs(cert["g"])
    prev = oracle.certify(p, oracle.fista(p, T - 25, *sched, precondition=True, trajectory=False)["lam"], 1e-2)
    assert prev["rel_gap"] > 1e-4
