"""Pins for the oracle's per-user projection (Sec. 3.3 simple sets; Sec. 4.3
simplex projection of Duchi et al.): brute-force enumeration of active sets,
closed forms, KKT conditions, two independent algorithms and a library QP
solver.  CPU only."""
import itertools

import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(20260601)


def brute_force_simplex(v, z, eq):
    """Textbook active-set enumeration for min ||x - v||^2 over
    {x >= 0, sum x <= z} (or == z): for every support S and every choice of
    active/inactive sum constraint, solve the equality-constrained subproblem
    in closed form, keep the feasible candidates, return the one nearest v."""
    n = len(v)
    best, best_d = None, np.inf
    for r in range(0, n + 1):
        for S in itertools.combinations(range(n), r):
            S = list(S)
            for active in ([True] if eq else [False, True]):
                x = np.zeros(n)
                if active:
                    if not S:
                        continue
                    # min sum_S (x_k - v_k)^2 s.t. sum_S x_k = z  ->  x_S = v_S - t
                    t = (v[S].sum() - z) / len(S)
                    x[S] = v[S] - t
                else:
                    x[S] = v[S]
                if (x < -1e-13).any():
                    continue
                if eq and abs(x.sum() - z) > 1e-12:
                    continue
                if (not eq) and x.sum() > z + 1e-12:
                    continue
                d = ((x - v) ** 2).sum()
                if d < best_d - 1e-15:
                    best, best_d = x, d
    return np.maximum(best, 0.0)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 10])
@pytest.mark.parametrize("eq", [False, True])
@pytest.mark.parametrize("method", [0, 1])
def test_projection_matches_enumeration(n, eq, method):
    kind = oracle.SIMPLEX_EQ if eq else oracle.SIMPLEX_LE
    for trial in range(25):
        scale = [0.1, 1.0, 10.0][trial % 3]
        v = RNG.normal(size=n) * scale + (0.2 if trial % 2 else -0.1)
        z = [1.0, 0.5, 2.0][trial % 3]
        x, _ = oracle.project(v, kind, z, method)
        ref = brute_force_simplex(v, z, eq)
        np.testing.assert_allclose(x, ref, atol=1e-11 * max(1.0, np.abs(v).max()))


def test_projection_closed_forms():
    # n = 1: the inequality simplex is the interval [0, z]; equality gives z.
    for v in [-3.0, -1e-9, 0.0, 0.3, 1.0, 7.5]:
        x, _ = oracle.project(np.array([v]), oracle.SIMPLEX_LE, 1.0)
        assert x[0] == min(max(v, 0.0), 1.0)
        x, _ = oracle.project(np.array([v]), oracle.SIMPLEX_EQ, 1.0)
        assert x[0] == 1.0
    # a point already inside the inequality simplex (after clipping) is kept: early exit
    v = np.array([0.2, -0.5, 0.3, 0.1])
    x, th = oracle.project(v, oracle.SIMPLEX_LE, 1.0)
    assert th == 0.0 and np.array_equal(x, np.maximum(v, 0))
    # uniform vector onto the equality simplex: z/n each
    x, _ = oracle.project(np.full(7, 3.3), oracle.SIMPLEX_EQ, 2.0)
    np.testing.assert_allclose(x, np.full(7, 2.0 / 7), rtol=1e-14)
    # one dominant coordinate: x = z e_k
    x, th = oracle.project(np.array([10.0, 1.0, 2.0]), oracle.SIMPLEX_LE, 1.0)
    assert np.array_equal(x, [1.0, 0.0, 0.0]) and th == 9.0
    # box: clipping
    x, _ = oracle.project(np.array([-1.0, 0.5, 2.0]), oracle.BOX, 1.0)
    assert np.array_equal(x, [0.0, 0.5, 1.0])


@pytest.mark.parametrize("eq", [False, True])
def test_projection_kkt(eq):
    kind = oracle.SIMPLEX_EQ if eq else oracle.SIMPLEX_LE
    for trial in range(200):
        n = int(RNG.integers(1, 60))
        v = RNG.normal(size=n) * RNG.choice([0.01, 1.0, 100.0])
        z = float(RNG.choice([1.0, 0.25, 3.0]))
        x, th = oracle.project(v, kind, z)
        assert (x >= 0).all()
        # stationarity: x = max(v - theta, 0)
        np.testing.assert_allclose(x, np.maximum(v - th, 0), atol=1e-12 * max(1, np.abs(v).max()))
        if eq:
            assert abs(x.sum() - z) <= 1e-12 * max(1, np.abs(v).sum())
        else:
            assert th >= 0
            assert x.sum() <= z + 1e-12 * max(1, np.abs(v).sum())
            # complementary slackness theta * (sum x - z) = 0
            assert th * abs(x.sum() - z) <= 1e-10 * max(1, th)


@pytest.mark.parametrize("eq", [False, True])
def test_sort_and_bisection_agree(eq):
    kind = oracle.SIMPLEX_EQ if eq else oracle.SIMPLEX_LE
    for trial in range(200):
        n = int(RNG.integers(1, 300))
        v = RNG.normal(size=n) * RNG.choice([0.1, 1.0, 1000.0])
        x0, t0 = oracle.project(v, kind, 1.0, method=0)
        x1, t1 = oracle.project(v, kind, 1.0, method=1)
        np.testing.assert_allclose(x0, x1, atol=1e-12 * max(1, np.abs(v).max()))


def test_projection_against_scipy_qp():
    scipy_opt = pytest.importorskip("scipy.optimize")
    for trial in range(20):
        n = int(RNG.integers(2, 12))
        v = RNG.normal(size=n)
        cons = [{"type": "ineq", "fun": lambda x: 1.0 - x.sum(), "jac": lambda x: -np.ones_like(x)}]
        res = scipy_opt.minimize(lambda x: ((x - v) ** 2).sum(), np.zeros(n), jac=lambda x: 2 * (x - v),
                                 bounds=[(0, None)] * n, constraints=cons, method="SLSQP",
                                 options=dict(ftol=1e-14, maxiter=500))
        x, _ = oracle.project(v, oracle.SIMPLEX_LE, 1.0)
        np.testing.assert_allclose(x, res.x, atol=1e-6)


def test_box_against_enumeration():
    for trial in range(50):
        v = RNG.normal(size=6) * 2
        u = 0.7
        x, _ = oracle.project(v, oracle.BOX, u)
        # per coordinate the candidates are 0, u and v_k; keep the feasible nearest one
        for k in range(6):
            cands = [c for c in (0.0, u, v[k]) if 0 <= c <= u]
            assert x[k] == min(cands, key=lambda c: abs(c - v[k]))
