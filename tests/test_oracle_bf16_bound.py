"""Pin for the error statement of the BF16 storage form: rounding c alone
(A and b fixed) moves the optimum by at most ||dc||_2 / gamma.

The primal (Sec. 3.1, Eq. primal) is min c^T x + gamma/2 ||x||^2 over the
fixed convex feasible set F, i.e. x*(c) = Proj_F(-c / gamma); a Euclidean
projection onto a convex set is nonexpansive, so
    ||x*(c + dc) - x*(c)||_2 <= ||dc||_2 / gamma,
with equality when no constraint binds (x* = -c / gamma).  The oracle's
converged solutions must satisfy both.  CPU only."""
import numpy as np

import oracle
import synth


def bf16(v):
    return synth.bf16_to_f32(synth.round_bf16(np.asarray(v, dtype=np.float32))).astype(np.float64)


def solved(p, gamma, T):
    r = oracle.fista(p, T, gamma, precondition=True, restart=True, trajectory=False)
    cert = oracle.certify(p, r["lam"], gamma)
    return oracle.sweep(p, r["lam"], gamma)["x"], cert, r["lam"]


def test_bound_is_attained_when_nothing_binds():
    # box [0, z] with -c / gamma strictly inside and every capacity slack:
    # x* = -c / gamma on both sides, so ||dx*|| = ||dc|| / gamma exactly
    rng = np.random.default_rng(3)
    I, J, gamma, z = 400, 30, 0.5, 1.0
    deg = rng.integers(1, 6, size=I)
    rp = np.zeros(I + 1, np.int64)
    np.cumsum(deg, out=rp[1:])
    col = np.concatenate([rng.choice(J, size=d, replace=False) for d in deg]).astype(np.int32)
    c = -rng.uniform(0.05, 0.45, size=rp[-1]).astype(np.float32).astype(np.float64)  # -c/gamma in (0.1, 0.9)
    a = np.ones(rp[-1])
    b = np.bincount(col, weights=a, minlength=J) * z + 1.0  # slack
    cr = bf16(c)
    p = oracle.Problem(rp, col, c, a, b, J, oracle.BOX, z)
    pr = oracle.Problem(rp, col, cr, a, b, J, oracle.BOX, z)
    x, _, _ = solved(p, gamma, 50)
    xr, _, _ = solved(pr, gamma, 50)
    np.testing.assert_allclose(x, -c / gamma, rtol=0, atol=1e-15)
    dx, bound = np.linalg.norm(xr - x), np.linalg.norm(cr - c) / gamma
    assert bound > 1e-3
    assert abs(dx - bound) <= 1e-12 * bound


def test_bound_holds_on_a_binding_instance():
    r = synth.recipe_production(I=600, J=25, seed=41)
    inst = synth.generate(r)
    gamma = 1e-2
    c = inst.c.astype(np.float64)
    a = inst.a.astype(np.float64)
    cr = bf16(inst.c)
    p = oracle.Problem(inst.row_ptr, inst.col, c, a, inst.b, inst.J)
    pr = oracle.Problem(inst.row_ptr, inst.col, cr, a, inst.b, inst.J)
    x, cert, lam = solved(p, gamma, 4000)
    xr, cert_r, _ = solved(pr, gamma, 4000)
    # both solves have converged, and capacities bind (the bound is not the
    # trivial unconstrained case)
    assert cert["rel_gap"] <= 1e-10 and cert_r["rel_gap"] <= 1e-10
    assert (lam > 1e-6).sum() >= 3
    dx, bound = np.linalg.norm(xr - x), np.linalg.norm(cr - c) / gamma
    assert 0 < dx <= bound
