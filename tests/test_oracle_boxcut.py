"""Pins for the oracle's box-cut simple set {0 <= x <= z, sum x <= cut}:
both projection methods against brute-force enumeration of which coordinates
sit at 0, in between or at z; the two reductions (a slack budget gives the
box, a slack box gives the inequality simplex with radius cut); a
general-purpose solver; central finite differences of the dual; exact KKT
points of a small dense QP by enumerating its active sets; feasibility of the
certificate's scaled point.  CPU only."""
import itertools

import numpy as np
import pytest

import oracle


def brute_force(v, z, cut):
    """Every assignment of the coordinates to {0, free, z}, with the budget
    slack (theta = 0) or tight; the consistent one is the projection."""
    n = len(v)
    x0 = np.clip(v, 0, z)
    if x0.sum() <= cut + 1e-15:
        return x0, 0.0
    for assign in itertools.product(range(3), repeat=n):
        a = np.array(assign)
        free = a == 1
        if not free.any():
            continue
        theta = (v[free].sum() + z * (a == 2).sum() - cut) / free.sum()
        if theta < -1e-12:
            continue
        y = v - theta
        if (y[a == 0] <= 1e-12).all() and ((y[free] > -1e-12) & (y[free] < z + 1e-12)).all() and \
                (y[a == 2] >= z - 1e-12).all():
            return np.clip(y, 0, z), theta
    raise AssertionError("no consistent assignment")


@pytest.mark.parametrize("seed", range(40))
def test_projection_matches_enumeration(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 8))
    v = rng.normal(0.3, 0.8, n)
    z = float(rng.uniform(0.2, 1.5))
    cut = float(rng.uniform(0.1, 1.2) * n * z)
    ref, th = brute_force(v, z, cut)
    for method in (0, 1):
        x, t = oracle.project(v, oracle.BOX_CUT, z, method, cut)
        np.testing.assert_allclose(x, ref, atol=1e-12)
        assert abs(t - th) <= 1e-10
    assert x.sum() <= cut + 1e-12 and (x >= 0).all() and (x <= z).all()


def test_ties_at_breakpoints():
    # values that put the root exactly on a breakpoint, and equal values
    v = np.array([1.0, 1.0, 0.5, 0.5, 0.0])
    for z, cut in ((0.5, 1.0), (0.5, 1.5), (1.0, 2.0), (0.25, 0.5)):
        ref, _ = brute_force(v, z, cut)
        for method in (0, 1):
            np.testing.assert_allclose(oracle.project(v, oracle.BOX_CUT, z, method, cut)[0], ref, atol=1e-12)


@pytest.mark.parametrize("seed", range(10))
def test_reductions_to_box_and_simplex(seed):
    rng = np.random.default_rng(100 + seed)
    n = 12
    v = rng.normal(0.2, 1.0, n)
    # slack budget: the box
    z = 0.7
    xb, _ = oracle.project(v, oracle.BOX, z)
    xc, _ = oracle.project(v, oracle.BOX_CUT, z, 0, n * z + 1.0)
    np.testing.assert_array_equal(xc, xb)
    # slack box (z >= cut): the inequality simplex with radius cut
    cut = 0.8
    xs, _ = oracle.project(v, oracle.SIMPLEX_LE, cut)
    xc, _ = oracle.project(v, oracle.BOX_CUT, 5.0, 0, cut)
    np.testing.assert_allclose(xc, xs, atol=1e-13)


@pytest.mark.parametrize("seed", range(5))
def test_projection_matches_a_general_solver(seed):
    opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(200 + seed)
    n = 20
    v = rng.normal(0.1, 1.0, n)
    z, cut = 0.6, 2.5
    x, _ = oracle.project(v, oracle.BOX_CUT, z, 0, cut)
    res = opt.minimize(lambda y: 0.5 * np.sum((y - v) ** 2), np.zeros(n), jac=lambda y: y - v,
                       bounds=[(0, z)] * n, constraints=[{"type": "ineq", "fun": lambda y: cut - y.sum(),
                                                          "jac": lambda y: -np.ones(n)}],
                       method="SLSQP", options={"ftol": 1e-15, "maxiter": 500})
    assert 0.5 * np.sum((x - v) ** 2) <= res.fun + 1e-10
    np.testing.assert_allclose(x, res.x, atol=1e-6)


def small_problem(seed, I=3, J=2, z=0.6, cut=0.8, b_scale=0.6):
    rng = np.random.default_rng(seed)
    row_ptr = np.arange(0, I * J + 1, J)
    col = np.tile(np.arange(J), I)
    c = -rng.uniform(0.2, 1.0, size=I * J)
    a = rng.uniform(0.5, 1.5, size=I * J)
    b = b_scale * rng.uniform(0.3, 1.0, size=J)
    return oracle.Problem(row_ptr, col, c, a, b, J, oracle.BOX_CUT, z, cut=cut)


def test_dual_gradient_matches_central_differences():
    p = small_problem(5, I=4, J=3)
    rng = np.random.default_rng(3)
    gamma = 0.2
    lam = rng.uniform(0, 0.8, size=p.J)
    g, grad, _ = oracle.dual(p, lam, gamma)
    h = 1e-6
    for k in range(p.J):
        e = np.zeros(p.J)
        e[k] = h
        fd = (oracle.dual(p, lam + e, gamma)[0] - oracle.dual(p, lam - e, gamma)[0]) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, grad[k])


def kkt_by_enumeration(p, gamma):
    n, J = p.nnz, p.J
    rows, rhs, tags = [], [], []
    for k in range(n):
        r = np.zeros(n)
        r[k] = -1
        rows.append(r), rhs.append(0.0), tags.append(None)
        r = np.zeros(n)
        r[k] = 1
        rows.append(r), rhs.append(p.z), tags.append(None)
    for i in range(p.I):
        r = np.zeros(n)
        r[p.row_ptr[i]:p.row_ptr[i + 1]] = 1
        rows.append(r), rhs.append(p.cut), tags.append(None)
    for j in range(J):
        rows.append(np.where(p.col == j, p.a, 0.0)), rhs.append(p.b[j]), tags.append(j)
    G, h = np.array(rows), np.array(rhs)
    for r in range(0, n + 1):
        for W in itertools.combinations(range(G.shape[0]), r):
            W = list(W)
            K = np.zeros((n + r, n + r))
            K[:n, :n] = gamma * np.eye(n)
            K[:n, n:] = G[W].T
            K[n:, :n] = G[W]
            try:
                sol = np.linalg.solve(K, np.concatenate([-p.c, h[W]]))
            except np.linalg.LinAlgError:
                continue
            if np.linalg.cond(K) > 1e12:
                continue
            x, mult = sol[:n], sol[n:]
            if (G @ x <= h + 1e-11).all() and (mult >= -1e-11).all():
                lam = np.zeros(J)
                for w, v in zip(W, mult):
                    if tags[w] is not None:
                        lam[tags[w]] = v
                return x, lam
    raise AssertionError("no KKT point")


@pytest.mark.parametrize("seed,z,cut,bs", [(1, 0.6, 0.8, 0.6), (2, 0.4, 0.7, 0.5), (3, 1.0, 0.5, 2.0),
                                           (4, 0.3, 2.0, 0.4), (9, 0.5, 0.6, 0.9)])
def test_converged_solution_matches_enumeration(seed, z, cut, bs):
    p = small_problem(seed, z=z, cut=cut, b_scale=bs)
    gamma = 0.1
    x_ref, lam_ref = kkt_by_enumeration(p, gamma)
    out = oracle.fista(p, 60000, gamma, precondition=True, trajectory=False, restart=True)
    g, _, x = oracle.dual(p, out["lam"], gamma)
    np.testing.assert_allclose(x, x_ref, atol=1e-8)
    np.testing.assert_allclose(out["lam"], lam_ref, atol=1e-7)
    np.testing.assert_allclose(g, p.c @ x_ref + 0.5 * gamma * x_ref @ x_ref, rtol=1e-9)


def test_enumeration_cases_bind_the_budget_the_box_and_the_capacities():
    # the cases above: budgets binding with slack capacities (seed 3), capped
    # coordinates under binding capacities (seeds 1, 2, 4), and all three at
    # once (seed 9)
    p = small_problem(3, z=1.0, cut=0.5, b_scale=2.0)
    x, lam = kkt_by_enumeration(p, 0.1)
    assert (np.abs(np.add.reduceat(x, p.row_ptr[:-1]) - p.cut) < 1e-9).all() and (lam == 0).all()
    p = small_problem(4, z=0.3, cut=2.0, b_scale=0.4)
    x, lam = kkt_by_enumeration(p, 0.1)
    assert (np.abs(x - p.z) < 1e-9).any() and (lam > 0).any()
    p = small_problem(9, z=0.5, cut=0.6, b_scale=0.9)
    x, lam = kkt_by_enumeration(p, 0.1)
    assert (np.abs(np.add.reduceat(x, p.row_ptr[:-1]) - p.cut) < 1e-9).any()
    assert (np.abs(x - p.z) < 1e-9).any() and (lam > 0).all()


def test_certificate_point_is_feasible():
    p = small_problem(7, I=5, J=3, z=0.5, cut=0.7, b_scale=0.4)
    rng = np.random.default_rng(1)
    lam = rng.uniform(0, 0.3, p.J)
    cert = oracle.certify(p, lam, 0.05)
    assert cert["rel_gap"] >= -1e-12
    _, _, x = oracle.dual(p, lam, 0.05)
    Ax = np.bincount(p.col, weights=p.a * x, minlength=p.J)
    s = np.minimum(1.0, p.b / np.maximum(Ax, 1e-300))
    xt = s[p.col] * x
    assert (xt >= 0).all() and (xt <= p.z + 1e-15).all()
    assert (np.add.reduceat(xt, p.row_ptr[:-1]) <= p.cut + 1e-12).all()
    assert (np.bincount(p.col, weights=p.a * xt, minlength=p.J) <= p.b + 1e-12).all()
