"""Pins for the oracle's global count constraint sum_ij x_ij <= M (the paper's
example of a new coupling constraint, Sec. 5: one more dual coordinate mu, one
more term in A^T lam, one more gradient entry).  Checked against central
finite differences, exact KKT points found by enumerating the active sets of
the dense QP with the count row, a one-user closed form, and the slack limit
in which the constraint changes nothing.  CPU only."""
import itertools

import numpy as np
import pytest

import oracle


def small(seed, I=3, J=2, b_scale=0.6, M=1.2):
    rng = np.random.default_rng(seed)
    row_ptr = np.arange(0, I * J + 1, J)
    col = np.tile(np.arange(J), I)
    c = -rng.uniform(0.2, 1.0, size=I * J)
    a = rng.uniform(0.5, 1.5, size=I * J)
    b = b_scale * rng.uniform(0.3, 1.0, size=J)
    return oracle.Problem(row_ptr, col, c, a, b, J, M=M)


def kkt_by_enumeration(p, gamma):
    """Every active set W of G x <= h (x >= 0, per-user simplex, capacities,
    count row); the KKT point with feasible x and nonnegative multipliers."""
    n = p.nnz
    rows, rhs, tags = [], [], []
    for k in range(n):
        r = np.zeros(n)
        r[k] = -1
        rows.append(r), rhs.append(0.0), tags.append(("pos", k))
    for i in range(p.I):
        r = np.zeros(n)
        r[p.row_ptr[i]:p.row_ptr[i + 1]] = 1
        rows.append(r), rhs.append(p.z), tags.append(("user", i))
    for j in range(p.J):
        rows.append(np.where(p.col == j, p.a, 0.0)), rhs.append(p.b[j]), tags.append(("cap", j))
    rows.append(np.ones(n)), rhs.append(p.M), tags.append(("count", 0))
    G, h = np.array(rows), np.array(rhs)
    m = G.shape[0]
    for r in range(0, n + 1):
        for W in itertools.combinations(range(m), r):
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
                lam = np.zeros(p.J + 1)
                for w, v in zip(W, mult):
                    if tags[w][0] == "cap":
                        lam[tags[w][1]] = v
                    elif tags[w][0] == "count":
                        lam[p.J] = v
                return x, lam
    raise AssertionError("no KKT point")


def test_gradient_matches_central_differences():
    p = small(5, M=1.0)
    rng = np.random.default_rng(2)
    gamma = 0.2
    for _ in range(3):
        lam = rng.uniform(0, 0.8, size=p.D)
        g, grad, _ = oracle.dual(p, lam, gamma)
        h = 1e-6
        for k in range(p.D):
            e = np.zeros(p.D)
            e[k] = h
            fd = (oracle.dual(p, lam + e, gamma)[0] - oracle.dual(p, lam - e, gamma)[0]) / (2 * h)
            assert abs(fd - grad[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, grad[k])


@pytest.mark.parametrize("seed,M,bs", [(1, 0.9, 6.0), (2, 1.4, 0.6), (3, 0.5, 0.3), (4, 2.0, 0.9)])
@pytest.mark.parametrize("precondition", [True, False])
def test_converged_solution_matches_enumeration(seed, M, bs, precondition):
    p = small(seed, b_scale=bs, M=M)
    gamma = 0.1
    x_ref, lam_ref = kkt_by_enumeration(p, gamma)
    out = oracle.fista(p, 60000, gamma, precondition=precondition, trajectory=False, restart=True)
    np.testing.assert_allclose(out["lam"], lam_ref, atol=1e-8)
    g, _, x = oracle.dual(p, out["lam"], gamma)
    np.testing.assert_allclose(x, x_ref, atol=1e-8)
    np.testing.assert_allclose(g, p.c @ x_ref + 0.5 * gamma * x_ref @ x_ref, rtol=1e-9)


def test_enumeration_cases_bind_the_count_row():
    binding = [kkt_by_enumeration(small(s, b_scale=bs, M=M), 0.1)[1][-1] > 1e-9
               for s, M, bs in [(1, 0.9, 6.0), (2, 1.4, 0.6), (3, 0.5, 0.3), (4, 2.0, 0.9)]]
    assert any(binding) and not all(binding)


def test_one_user_closed_form():
    # one user, two items with slack capacities, u/gamma = (1, 0.5), z = 1,
    # M = 0.3: the count row alone binds; projecting onto sum <= 0.3 keeps
    # the first item only, x = (0.3, 0), and its multiplier is the threshold
    # mu = 1 - 0.3 = 0.7 (lam = 0).
    p = oracle.Problem(np.array([0, 2]), np.array([0, 1], dtype=np.int32), np.array([-1.0, -0.5]),
                       np.array([1.0, 1.0]), np.array([10.0, 10.0]), 2, M=0.3)
    out = oracle.fista(p, 5000, 1.0, precondition=True, trajectory=False)
    np.testing.assert_allclose(out["lam"], [0.0, 0.0, 0.7], atol=1e-10)
    _, _, x = oracle.dual(p, out["lam"], 1.0)
    np.testing.assert_allclose(x, [0.3, 0.0], atol=1e-10)


def test_slack_count_changes_nothing():
    p = small(2, b_scale=0.6, M=np.inf)
    q = small(2, b_scale=0.6, M=100.0)
    a = oracle.fista(p, 3000, 0.1, precondition=True, trajectory=False)["lam"]
    b = oracle.fista(q, 3000, 0.1, precondition=True, trajectory=False)["lam"]
    assert b[-1] == 0.0
    # the same fixed point; the step sizes differ (the count row enters the
    # Gershgorin bounds), so compare at convergence
    np.testing.assert_allclose(b[:-1], a, atol=1e-9)


def test_certificate_is_feasible_and_bounds_the_dual():
    p = small(3, b_scale=0.3, M=0.5)
    lam = oracle.fista(p, 200, 0.1, precondition=True, trajectory=False)["lam"]
    cert = oracle.certify(p, lam, 0.1)
    assert cert["rel_gap"] >= -1e-12  # weak duality with the scaled point
    # rebuild the scaled point and check it against every constraint
    sw = oracle.sweep(p, lam, 0.1)
    s = np.minimum(1.0, np.where(sw["Ax"] > p.b, p.b / np.maximum(sw["Ax"], 1e-300), 1.0))
    t = min(1.0, p.M / sw["count"]) if sw["count"] > p.M else 1.0
    xs = t * s[p.col] * sw["x"]
    assert xs.sum() <= p.M + 1e-12
    assert (np.bincount(p.col, weights=p.a * xs, minlength=p.J) <= p.b + 1e-12).all()
    assert cert["primal"] == pytest.approx(p.c @ xs + 0.05 * xs @ xs, rel=1e-12)
