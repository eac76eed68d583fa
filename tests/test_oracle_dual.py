"""Pins for the oracle's dual evaluation (Sec. 3.2: Eq. dual, Eq.
primal-recovery, Eq. dual-gradient by Danskin's theorem; App. B.2 Lipschitz
bound ||A||^2/gamma; Def. 1 diagonal-block structure).  CPU only."""
import numpy as np
import pytest

import oracle
import synth

RNG = np.random.default_rng(7)


def small_problem(I=300, J=20, seed=5, kind=oracle.SIMPLEX_LE, z=1.0):
    r = synth.recipe_production(I=I, J=J, seed=seed)
    r.deg_mean, r.deg_max = 6.0, 15
    inst = synth.generate(r)
    return oracle.Problem.from_instance(inst, kind=kind, z=z), inst


@pytest.mark.parametrize("kind", [oracle.SIMPLEX_LE, oracle.SIMPLEX_EQ, oracle.BOX])
def test_gradient_matches_central_differences(kind):
    p, _ = small_problem(kind=kind)
    gamma = 0.1
    for trial in range(3):
        lam = RNG.uniform(0, 2.0, size=p.J)
        g0, grad, _ = oracle.dual(p, lam, gamma)
        fd = np.empty(p.J)
        for j in range(p.J):
            h = 1e-5
            e = np.zeros(p.J)
            e[j] = h
            fd[j] = (oracle.dual(p, lam + e, gamma)[0] - oracle.dual(p, lam - e, gamma)[0]) / (2 * h)
        np.testing.assert_allclose(fd, grad, rtol=1e-6, atol=1e-6 * np.abs(grad).max())


def test_concave_and_smooth():
    p, _ = small_problem()
    gamma = 0.05
    n2 = oracle.row_sq(p)
    L = n2.max() / gamma
    for trial in range(50):
        lam = RNG.uniform(0, 3, size=p.J)
        mu = np.maximum(lam + RNG.normal(size=p.J) * RNG.choice([1e-3, 0.1, 1.0]), 0)
        gl, dl, _ = oracle.dual(p, lam, gamma)
        gm, _, _ = oracle.dual(p, mu, gamma)
        lin = gl + dl @ (mu - lam)
        tol = 1e-10 * (abs(gl) + abs(gm) + 1)
        assert gm <= lin + tol  # concavity
        assert gm >= lin - 0.5 * L * ((mu - lam) ** 2).sum() - tol  # L-smoothness


def test_norm_closed_form_matches_dense_spectrum():
    # Def. 1 with one family: every column of A (one edge) has one nonzero, so
    # A A^T is diagonal and ||A||_2^2 = max_j sum_i a_ij^2.
    p, inst = small_problem(I=60, J=7)
    A = np.zeros((p.J, p.nnz))
    A[p.col, np.arange(p.nnz)] = p.a
    AAt = A @ A.T
    assert np.abs(AAt - np.diag(np.diag(AAt))).max() == 0.0
    n2 = oracle.row_sq(p)
    np.testing.assert_allclose(n2, np.diag(AAt), rtol=1e-14)
    np.testing.assert_allclose(n2.max(), np.linalg.eigvalsh(AAt).max(), rtol=1e-12)


def test_primal_recovery_minimises_lagrangian():
    # x*(lam) must minimise c^T x + gamma/2 ||x||^2 + lam^T A x over C, user by user.
    scipy_opt = pytest.importorskip("scipy.optimize")
    p, _ = small_problem(I=30, J=6)
    gamma = 0.2
    lam = RNG.uniform(0, 1, size=p.J)
    _, _, x = oracle.dual(p, lam, gamma)
    for i in range(p.I):
        s, e = p.row_ptr[i], p.row_ptr[i + 1]
        w = p.c[s:e] + p.a[s:e] * lam[p.col[s:e]]
        f = lambda y: w @ y + 0.5 * gamma * y @ y  # noqa: E731
        res = scipy_opt.minimize(f, np.full(e - s, 1.0 / (e - s) * 0.5), jac=lambda y: w + gamma * y,
                                 bounds=[(0, None)] * (e - s), method="SLSQP",
                                 constraints=[{"type": "ineq", "fun": lambda y: 1 - y.sum()}],
                                 options=dict(ftol=1e-15, maxiter=1000))
        assert f(x[s:e]) <= res.fun + 1e-9


def test_weak_duality_and_scaled_point_feasible():
    p, inst = small_problem()
    for gamma in [1.0, 0.1, 0.01]:
        for trial in range(10):
            lam = RNG.uniform(0, 2, size=p.J) * (trial % 3 != 0)
            st = oracle.certify(p, lam, gamma)
            assert st["rel_gap"] >= -1e-12
            sw = oracle.sweep(p, lam, gamma)
            s = np.where(sw["Ax"] > p.b, p.b / np.where(sw["Ax"] > 0, sw["Ax"], 1), 1.0)
            xt = sw["x"] * s[p.col]
            Axt = np.bincount(p.col, weights=p.a * xt, minlength=p.J)
            assert (Axt <= p.b * (1 + 1e-12) + 1e-12).all()
            sums = np.add.reduceat(xt, p.row_ptr[:-1]) if p.nnz else np.zeros(0)
            assert (sums <= 1 + 1e-12).all() and (xt >= 0).all()
            primal = (p.c * xt).sum() + 0.5 * gamma * (xt ** 2).sum()
            np.testing.assert_allclose(st["primal"], primal, rtol=1e-12, atol=1e-12)
