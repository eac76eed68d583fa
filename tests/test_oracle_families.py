"""Pins for the oracle with several capacity families (Def. 1: m families,
each with one diagonal block per user, so A A^T is block diagonal with one
m x m block per item).  Checked against central finite differences, exact KKT
points from enumerating the active sets of the dense QP with 2 rows per item,
and two reductions to one family (a slack second family; a duplicated
family, whose duals split but whose x and dual sum do not).  CPU only."""
import itertools

import numpy as np
import pytest

import oracle


def two_family(seed, I=3, J=2, b_scale=(0.6, 0.6), M=np.inf):
    rng = np.random.default_rng(seed)
    row_ptr = np.arange(0, I * J + 1, J)
    col = np.tile(np.arange(J), I)
    c = -rng.uniform(0.2, 1.0, size=I * J)
    a = np.stack([rng.uniform(0.5, 1.5, size=I * J), rng.uniform(0.1, 2.0, size=I * J)], axis=1)
    b = np.stack([b_scale[0] * rng.uniform(0.3, 1.0, size=J), b_scale[1] * rng.uniform(0.3, 1.0, size=J)])
    return oracle.Problem(row_ptr, col, c, a, b, J, M=M)


def kkt_by_enumeration(p, gamma):
    n, J, m = p.nnz, p.J, p.m
    a = p.a.reshape(n, m)
    b = p.b.reshape(m, J)
    rows, rhs, tags = [], [], []
    for k in range(n):
        r = np.zeros(n)
        r[k] = -1
        rows.append(r), rhs.append(0.0), tags.append(None)
    for i in range(p.I):
        r = np.zeros(n)
        r[p.row_ptr[i]:p.row_ptr[i + 1]] = 1
        rows.append(r), rhs.append(p.z), tags.append(None)
    for f in range(m):
        for j in range(J):
            rows.append(np.where(p.col == j, a[:, f], 0.0)), rhs.append(b[f, j]), tags.append(f * J + j)
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
                lam = np.zeros(m * J)
                for w, v in zip(W, mult):
                    if tags[w] is not None:
                        lam[tags[w]] = v
                return x, lam
    raise AssertionError("no KKT point")


@pytest.mark.parametrize("M", [np.inf, 0.9])
def test_gradient_matches_central_differences(M):
    p = two_family(5, M=M)
    rng = np.random.default_rng(3)
    gamma = 0.2
    lam = rng.uniform(0, 0.8, size=p.D)
    g, grad, _ = oracle.dual(p, lam, gamma)
    assert grad.shape == (p.D,)
    h = 1e-6
    for k in range(p.D):
        e = np.zeros(p.D)
        e[k] = h
        fd = (oracle.dual(p, lam + e, gamma)[0] - oracle.dual(p, lam - e, gamma)[0]) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, grad[k])


@pytest.mark.parametrize("seed,bs", [(1, (0.6, 6.0)), (2, (6.0, 0.4)), (3, (0.5, 0.5)), (4, (0.3, 0.9))])
@pytest.mark.parametrize("precondition", [True, False])
def test_converged_solution_matches_enumeration(seed, bs, precondition):
    p = two_family(seed, b_scale=bs)
    gamma = 0.1
    x_ref, lam_ref = kkt_by_enumeration(p, gamma)
    out = oracle.fista(p, 60000, gamma, precondition=precondition, trajectory=False, restart=True)
    g, _, x = oracle.dual(p, out["lam"], gamma)
    np.testing.assert_allclose(x, x_ref, atol=1e-8)
    np.testing.assert_allclose(out["lam"], lam_ref, atol=1e-7)
    np.testing.assert_allclose(g, p.c @ x_ref + 0.5 * gamma * x_ref @ x_ref, rtol=1e-9)


def test_enumeration_binds_both_families_somewhere():
    lams = [kkt_by_enumeration(two_family(s, b_scale=bs), 0.1)[1]
            for s, bs in [(1, (0.6, 6.0)), (2, (6.0, 0.4)), (3, (0.5, 0.5)), (4, (0.3, 0.9))]]
    assert any(l[:2].max() > 1e-9 for l in lams) and any(l[2:].max() > 1e-9 for l in lams)


def test_slack_second_family_reduces_to_one():
    p2 = two_family(2, b_scale=(0.6, 1e6))
    a = p2.a.reshape(-1, 2)[:, 0]
    b = p2.b.reshape(2, -1)[0]
    p1 = oracle.Problem(p2.row_ptr, p2.col, p2.c, a, b, p2.J)
    l2 = oracle.fista(p2, 20000, 0.1, precondition=True, trajectory=False)["lam"]
    l1 = oracle.fista(p1, 20000, 0.1, precondition=True, trajectory=False)["lam"]
    assert (l2[p2.J:] == 0).all()
    np.testing.assert_allclose(l2[:p2.J], l1, atol=1e-9)


def test_duplicated_family_splits_the_dual():
    p1 = two_family(3, b_scale=(0.5, 0.5))
    a = p1.a.reshape(-1, 2)[:, 0]
    b = p1.b.reshape(2, -1)[0]
    one = oracle.Problem(p1.row_ptr, p1.col, p1.c, a, b, p1.J)
    dup = oracle.Problem(p1.row_ptr, p1.col, p1.c, np.stack([a, a], 1), np.stack([b, b]), p1.J)
    l1 = oracle.fista(one, 20000, 0.1, precondition=True, trajectory=False)["lam"]
    l2 = oracle.fista(dup, 20000, 0.1, precondition=True, trajectory=False)["lam"]
    np.testing.assert_allclose(l2[:p1.J] + l2[p1.J:], l1, atol=1e-8)
    x1 = oracle.dual(one, l1, 0.1)[2]
    x2 = oracle.dual(dup, l2, 0.1)[2]
    np.testing.assert_allclose(x2, x1, atol=1e-8)
