"""Pins of the FP64 warm-start reference (oracle/mlp.py) against facts that do
not come from the reference itself: central finite differences, networks
evaluated by hand, Adam's closed-form first step, brute-force feature loops,
and hand-worked bfloat16 ties (checked also against torch's conversion)."""
import math

import numpy as np
import pytest

from oracle import mlp


def small_net(H=6, seed=3):
    rng = np.random.default_rng(seed)
    return {"W1": rng.normal(size=(mlp.F, H)), "b1": rng.normal(size=H) * 0.1,
            "W2": rng.normal(size=(H, H)) / np.sqrt(H), "b2": rng.normal(size=H) * 0.1,
            "w3": rng.normal(size=H), "b3": np.array([0.3])}


def data(n=9, seed=4):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, mlp.F)) * np.array([1, 2, 0.5, 0.5, 1, 0.1, 3]) + 1.0
    y = rng.uniform(0, 2, size=n)
    return X, y


def test_gradient_matches_central_differences():
    P = small_net()
    X, y = data()
    mu, sd = mlp.normalizer(X)
    loss, g = mlp.loss_and_grad(P, X, y, mu, sd)
    h = 1e-6
    for k, v in P.items():
        fd = np.zeros_like(v)
        for idx in np.ndindex(v.shape):
            Pp = {kk: vv.copy() for kk, vv in P.items()}
            Pm = {kk: vv.copy() for kk, vv in P.items()}
            Pp[k][idx] += h
            Pm[k][idx] -= h
            lp, _ = mlp.loss_and_grad(Pp, X, y, mu, sd)
            lm, _ = mlp.loss_and_grad(Pm, X, y, mu, sd)
            fd[idx] = (lp - lm) / (2 * h)
        err = np.abs(fd - g[k]).max()
        assert err <= 1e-6 * max(1.0, np.abs(fd).max()), (k, err)


def test_forward_of_hand_built_networks():
    L2 = math.log(2.0)  # softplus^-1(log 2) = 0: the residual path adds nothing
    X = np.array([[0.5, 1, 2, 3, L2, 5, 6], [-2.0, 0, 0, 0, L2, 0, 0]])
    mu, sd = np.zeros(mlp.F), np.ones(mlp.F)
    H = 3
    P = {k: np.zeros_like(v) for k, v in mlp.init_params(H, 0).items()}
    # all-zero network: softplus(b3)
    P["b3"] = np.array([0.7])
    assert np.allclose(mlp.predict(P, X, mu, sd), math.log(1 + math.exp(0.7)), rtol=0, atol=1e-15)
    # one path: h1_0 = relu(x0), h2_0 = relu(2 h1_0 - 0.25), out = softplus(3 h2_0 - 1)
    P["W1"][0, 0] = 1.0
    P["W2"][0, 0] = 2.0
    P["b2"][0] = -0.25
    P["w3"][0] = 3.0
    P["b3"] = np.array([-1.0])
    want = []
    for x0 in (0.5, -2.0):
        h = max(2 * max(x0, 0.0) - 0.25, 0.0)
        want.append(math.log1p(math.exp(3 * h - 1)))
    assert np.allclose(mlp.predict(P, X, mu, sd), want, rtol=1e-15, atol=0)
    # a zero network returns the previous dual (floored at 1e-6)
    Z = {k: np.zeros_like(v) for k, v in P.items()}
    Xl = X.copy()
    Xl[:, 4] = [0.37, 0.0]
    assert np.allclose(mlp.predict(Z, Xl, mu, sd), [0.37, 1e-6], rtol=1e-12, atol=0)
    # standardization enters as (x - mu) / sd
    mu2, sd2 = np.full(mlp.F, 0.5), np.full(mlp.F, 2.0)
    h0 = max(2 * max((0.5 - 0.5) / 2, 0) - 0.25, 0)
    assert math.isclose(mlp.predict(P, X[:1], mu2, sd2)[0], math.log1p(math.exp(3 * h0 - 1)), rel_tol=1e-15)


def test_adam_first_step_closed_form():
    P = {"w": np.array([1.0, -2.0, 0.5, 3.0])}
    g = {"w": np.array([0.2, -4.0, 0.0, 1e-9])}
    m, v = mlp.adam_init(P)
    P1, m1, v1 = mlp.adam_step(P, g, m, v, 1, 0.01)
    # m_hat = g, v_hat = g^2: step = lr * g / (|g| + eps)
    want = P["w"] - 0.01 * g["w"] / (np.abs(g["w"]) + 1e-8)
    assert np.allclose(P1["w"], want, rtol=1e-14, atol=1e-16)
    assert np.allclose(m1["w"], 0.1 * g["w"]) and np.allclose(v1["w"], 0.001 * g["w"] ** 2)
    # second step with the same gradient: m_hat = g, v_hat = g^2 again
    P2, _, _ = mlp.adam_step(P1, g, m1, v1, 2, 0.01)
    assert np.allclose(P2["w"], want - 0.01 * g["w"] / (np.abs(g["w"]) + 1e-8), rtol=1e-12, atol=1e-15)


def test_features_against_loops():
    rng = np.random.default_rng(9)
    I, J = 40, 7
    rows = [sorted(rng.choice(J - 1, size=rng.integers(0, 5), replace=False)) for _ in range(I)]  # item J-1 empty
    row_ptr = np.zeros(I + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([j for r in rows for j in r], dtype=np.int32)
    c = -rng.uniform(0.1, 3, size=len(col))
    b = rng.uniform(0, 5, size=J)
    lam = rng.uniform(0, 1, size=J)
    grad = rng.normal(size=J)
    X = mlp.item_features(row_ptr, col, c, J, b, lam, 1e-2, grad)
    for j in range(J):
        vals = [-c[k] for k in range(len(col)) if col[k] == j]
        assert X[j, 0] == pytest.approx(math.log(1 + b[j]), rel=1e-15)
        assert X[j, 1] == pytest.approx(math.log(1 + len(vals)), rel=1e-15)
        assert X[j, 2] == pytest.approx(sum(vals) / len(vals) if vals else 0.0, rel=1e-14)
        assert X[j, 3] == (max(vals) if vals else 0.0)
        assert X[j, 4] == lam[j] and X[j, 5] == pytest.approx(math.log(1e-2), rel=1e-15)
        assert X[j, 6] == pytest.approx(grad[j] / (1 + b[j]), rel=1e-15)
    mu, sd = mlp.normalizer(X)
    assert sd[5] == 1.0  # constant column
    assert np.allclose(mu, X.mean(axis=0)) and np.allclose(sd[:5], X[:, :5].std(axis=0))


def test_bf16_rounding():
    cases = {1.0: 1.0, 1 + 2 ** -8: 1.0, 1 + 3 * 2 ** -8: 1 + 2 ** -6, 1 + 2 ** -7: 1 + 2 ** -7,
             1 + 2 ** -8 + 2 ** -20: 1 + 2 ** -7, -3.0: -3.0, 0.0: 0.0, 2 ** -130: 2 ** -130}
    for x, want in cases.items():
        assert mlp.bf16(x) == want, (x, mlp.bf16(x), want)
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    v = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-6, 6, size=5000),
                        np.float32(1.0) + np.arange(-512, 512, dtype=np.float32) * np.float32(2 ** -16)])
    v32 = v.astype(np.float32)
    ref = torch.from_numpy(v32).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
    assert np.array_equal(mlp.bf16(v32), ref)


def test_bf16_mode_tracks_fp64_mode():
    P = mlp.init_params(16, 1)
    X, y = data(50)
    mu, sd = mlp.normalizer(X)
    a = mlp.forward(P, X, mu, sd)["out"]
    b = mlp.forward(P, X, mu, sd, bf16_round=True)["out"]
    assert np.abs(a - b).max() <= 0.05 * np.abs(a).max()
    _, g = mlp.loss_and_grad(P, X, y, mu, sd)
    _, gb = mlp.loss_and_grad(P, X, y, mu, sd, bf16_round=True)
    for k in g:
        assert np.linalg.norm(g[k] - gb[k]) <= 0.05 * np.linalg.norm(g[k]) + 1e-12, k
