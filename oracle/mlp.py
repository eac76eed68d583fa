"""FP64 reference of the learned warm start (numpy).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: the solver library
never uses it and shares no code with it.

The paper motivates warm starts for recurring solves (Sec. 1: the same
matching problem is re-solved on a fixed cadence with drifting data) but
specifies no predictor; the predictor here is the one this project defines:

  item features (one row per item j, F = 7 columns)
    0  log(1 + b_j)
    1  log(1 + deg_j)                    deg_j = number of eligible users
    2  mean over the item's edges of -c_ij     (0 for an item with no edge)
    3  max over the item's edges of -c_ij      (0 for an item with no edge)
    4  lam_prev_j                        the previous solve's dual
    5  log(gamma)
    6  G_j / (1 + b_j)                   G = A x(lam_prev) - b, the dual
                                         gradient of today's instance at
                                         lam_prev (one sweep)
  standardization  xn = (x - mu) / sd   (mu, sd over the training rows; a
                                         column with sd < 1e-6 uses sd = 1)
  network          z1 = xn W1 + b1, h1 = relu(z1)       W1: F x H
                   z2 = h1 W2 + b2, h2 = relu(z2)       W2: H x H
                   z3 = h2 w3 + b3                      w3: H
                   out = softplus(z3 + softplus^-1(max(lam_prev, 1e-6)))
                   (a residual form: the network predicts a correction
                   to the previous dual in softplus pre-activation space,
                   so a zero last layer returns lam_prev and out >= 0)
  loss             mean over rows of (out - lam*)^2
  optimizer        Adam (Kingma & Ba 2015, Algorithm 1), bias-corrected.

With ``bf16=True`` the forward and backward passes round to bfloat16 (round
to nearest even) exactly where the GPU kernels feed a tensor-core product:
xn, W1, h1, W2, h2, w3 in the forward pass and dz2, dz1 (and the weights
they meet) in the backward pass; everything else stays FP64.

Parity status (tests/test_oracle_mlp.py): gradients pinned by central
finite differences; forward pinned by hand-evaluated networks; Adam pinned
by its closed-form first step; features pinned by brute-force loops;
bfloat16 rounding pinned by hand-worked ties and torch's conversion.
"""
from __future__ import annotations

import numpy as np

F = 7
SD_FLOOR = 1e-6
LAM_FLOOR = 1e-6
LAM_COL = 4


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    x32 = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = x32.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(x32)
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(nan, np.nan, out)


def item_features(row_ptr, col, c, J, b, lam_prev, gamma, grad):
    """Feature rows [J, F] of one instance (definitions in the module docstring)."""
    col = np.asarray(col, dtype=np.int64)
    negc = -np.asarray(c, dtype=np.float64)
    deg = np.bincount(col, minlength=J).astype(np.float64)
    s = np.bincount(col, weights=negc, minlength=J)
    mx = np.full(J, -np.inf)
    np.maximum.at(mx, col, negc)
    has = deg > 0
    X = np.zeros((J, F))
    b = np.asarray(b, dtype=np.float64)
    X[:, 0] = np.log1p(b)
    X[:, 1] = np.log1p(deg)
    X[:, 2] = np.where(has, s / np.where(has, deg, 1.0), 0.0)
    X[:, 3] = np.where(has, mx, 0.0)
    X[:, 4] = np.asarray(lam_prev, dtype=np.float64)
    X[:, 5] = np.log(gamma)
    X[:, 6] = np.asarray(grad, dtype=np.float64) / (1.0 + b)
    return X


def normalizer(X):
    """Column means and standard deviations (population), sd floored to 1."""
    mu = X.mean(axis=0)
    sd = np.sqrt(((X - mu) ** 2).mean(axis=0))
    sd = np.where(sd < SD_FLOOR, 1.0, sd)
    return mu, sd


def init_params(H=128, seed=0):
    rng = np.random.default_rng(seed)
    return {"W1": rng.uniform(-1, 1, (F, H)) * np.sqrt(6.0 / F), "b1": np.zeros(H),
            "W2": rng.uniform(-1, 1, (H, H)) * np.sqrt(6.0 / H), "b2": np.zeros(H),
            "w3": rng.uniform(-1, 1, H) * np.sqrt(3.0 / H), "b3": np.zeros(1)}


def _softplus(z):
    return np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))


def _sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def softplus_inv(y):
    """log(exp(y) - 1) for y > 0."""
    y = np.asarray(y, dtype=np.float64)
    return y + np.log(-np.expm1(-y))


def forward(P, X, mu, sd, bf16_round=False):
    r = bf16 if bf16_round else (lambda v: np.asarray(v, dtype=np.float64))
    xn = r((X - mu) / sd)
    z1 = xn @ r(P["W1"]) + P["b1"]
    h1 = np.maximum(z1, 0.0)
    h1r = r(h1)
    z2 = h1r @ r(P["W2"]) + P["b2"]
    h2 = np.maximum(z2, 0.0)
    h2r = r(h2)
    z3 = h2r @ r(P["w3"]) + P["b3"][0]
    s = z3 + softplus_inv(np.maximum(X[:, LAM_COL], LAM_FLOOR))
    return {"xn": xn, "z1": z1, "h1": h1r, "z2": z2, "h2": h2r, "z3": z3, "s": s, "out": _softplus(s)}


def loss_and_grad(P, X, y, mu, sd, bf16_round=False):
    """Mean squared error of the prediction against y and its gradient."""
    r = bf16 if bf16_round else (lambda v: np.asarray(v, dtype=np.float64))
    f = forward(P, X, mu, sd, bf16_round)
    n = X.shape[0]
    e = f["out"] - y
    loss = float(np.mean(e * e))
    dz3 = (2.0 / n) * e * _sigmoid(f["s"])
    g = {"w3": f["h2"].T @ dz3, "b3": np.array([dz3.sum()])}
    dh2 = np.outer(dz3, r(P["w3"]))
    dz2 = r(dh2 * (f["z2"] > 0))
    g["W2"] = f["h1"].T @ dz2
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ r(P["W2"]).T
    dz1 = r(dh1 * (f["z1"] > 0))
    g["W1"] = f["xn"].T @ dz1
    g["b1"] = dz1.sum(axis=0)
    return loss, g


def adam_init(P):
    return {k: np.zeros_like(v) for k, v in P.items()}, {k: np.zeros_like(v) for k, v in P.items()}


def adam_step(P, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns new (P, m, v)."""
    P2, m2, v2 = {}, {}, {}
    for k in P:
        m2[k] = beta1 * m[k] + (1 - beta1) * g[k]
        v2[k] = beta2 * v[k] + (1 - beta2) * g[k] ** 2
        mh = m2[k] / (1 - beta1 ** t)
        vh = v2[k] / (1 - beta2 ** t)
        P2[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)
    return P2, m2, v2


def predict(P, X, mu, sd, bf16_round=False):
    return forward(P, X, mu, sd, bf16_round)["out"]
