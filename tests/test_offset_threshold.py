"""The per-row arithmetic of the short-row sweep (csrc/sweep_short.cu),
emulated in IEEE FP32 with numpy and checked against the oracle's FP64
projection (Sec. 3.2 Eq. primal-recovery, Sec. 4.3's sort-based simplex
threshold): each edge's value u = -(c + a y) as a float pair (the product's
rounding error exact by TwoProduct, the sum's by TwoSum), the values sorted,
the active count from the sort-based rule in FP32, the threshold recomputed
as v_0 plus an offset -- the FP32 sum of the active edges' differences
u - v_0, which lie within gamma z of 0 -- and x = (((u_h - tau) + u_l) -
taul) / gamma clipped.  The claims checked: on rows with no edge within FP32
resolution of the threshold, x is within 8u z + 4u x (u = 2^-24) whatever the
size of the values (rows whose values are large and cancel against gamma z
at gamma = 1e-3); on the others, within the tolerance of the GPU parity
tests, whose allowance covers the active set decided in FP32.
The kernel itself is held to the oracle by tests/test_gpu_short_rows.py;
this test pins the arithmetic it follows on adversarial rows no instance
generator produces."""
import numpy as np
import pytest

import oracle

F = np.float32
U = 2.0 ** -24


def f32(x):
    return np.float32(x)


def u_pair(c, a, y):
    """-(c + a y) as (h, l) with h + l exact up to the rounding of l."""
    p = f32(a * y)
    pe = f32(np.float64(a) * np.float64(y) - np.float64(p))  # exact: the product's error fits FP32
    s = f32(-c - p)
    bp = f32(s - (-c))
    err = f32(f32(-c - f32(s - bp)) + f32(-p - bp))
    return s, f32(err - pe)


def fma32(x, y, z):
    return f32(np.float64(x) * np.float64(y) + np.float64(z))


def row_x(c, a, y, kind, z, gamma):
    """x of one row by the short-row sweep's arithmetic (FP32 throughout)."""
    g = np.float64(gamma)
    gz = f32(g * z)
    gzl = f32(g * z - np.float64(gz))
    invg = f32(1.0 / g)
    n = c.shape[0]
    uh = np.empty(n, F)
    ul = np.empty(n, F)
    for k in range(n):
        uh[k], ul[k] = u_pair(c[k], a[k], y[k])
    v = np.sort(uh)[::-1]
    box, eq = kind == oracle.BOX, kind == oracle.SIMPLEX_EQ
    x = np.zeros(n, F)
    if not eq and not v[0] > 0:
        return x
    tau, taul, single = f32(0), f32(0), False
    if not box:
        sm, sr, r = f32(0), v[0], 1
        for q in range(n):
            sm = f32(sm + v[q])
            if q > 0 and fma32(q + 1, v[q], -sm) > -gz:
                r, sr = q + 1, sm
        tau = f32(v[0] - gz) if r == 1 else f32(f32(sr - gz) / f32(r))
        zero = not eq and tau <= 0
        single = not zero and r == 1
        if not zero and not single:
            v0, sd, cnt = v[0], f32(0), 0
            for k in range(n):
                if uh[k] > tau:
                    sd = f32(sd + f32(f32(uh[k] - v0) + ul[k]))
                    cnt += 1
            t = f32(f32(f32(sd - gz) - gzl) / f32(max(cnt, 1)))
            if not eq and f32(v0 + t) <= 0:
                zero = True
            else:
                tau, taul = v0, t
        if zero:
            tau, taul = f32(0), f32(0)
    tt = f32(tau + taul)
    zc = f32(z) if box else F(np.inf)
    for k in range(n):
        if uh[k] > tt:
            d = f32(f32(f32(uh[k] - tau) + ul[k]) - taul)
            x[k] = f32(z) if single else min(max(f32(d * invg), F(0)), zc)
    return x


def adversarial_row(rng, gamma, z):
    """Values clustered within a few gamma z of a base of any size (so the
    active edges' u cancel in FP32 against the threshold), from c, a, y of
    the sizes the instances have."""
    n = int(rng.integers(1, 33))
    base = rng.choice([-3.0, -1e-2, 0.0, 1e-3, 0.5, 5.0, 40.0])
    spread = gamma * z * rng.choice([0.3, 1.5, 6.0])
    target = base + spread * rng.uniform(-1.0, 0.2, n)
    a = rng.uniform(0.5, 1.5, n).astype(F)
    y = rng.uniform(0.0, 2.0, n).astype(F)
    c = (-(target + a.astype(np.float64) * y)).astype(F)
    if n > 2 and rng.random() < 0.3:  # exact ties
        c[1] = c[0]
        a[1] = a[0]
        y[1] = y[0]
    return c, a, y


@pytest.mark.parametrize("kind,z", [(oracle.SIMPLEX_LE, 1.0), (oracle.SIMPLEX_EQ, 0.7), (oracle.BOX, 0.6)])
@pytest.mark.parametrize("gamma", [1e-1, 1e-2, 1e-3])
def test_offset_threshold_matches_fp64_projection(kind, z, gamma):
    rng = np.random.default_rng(20 + int(-np.log10(gamma)) + 7 * kind)
    worst = 0.0
    for _ in range(400):
        c, a, y = adversarial_row(rng, gamma, z)
        x = row_x(c, a, y, kind, z, gamma).astype(np.float64)
        u = -(c.astype(np.float64) + a.astype(np.float64) * y.astype(np.float64))  # exact u of the stored values
        ref, theta = oracle.project(u / gamma, kind, z)
        tol = 2e-6 * z + 4 * U * ref
        # edges within FP32 resolution of the threshold (or of the box's cap):
        # the active set is decided in FP32 there
        mag = np.abs(c.astype(np.float64)) + np.abs(a.astype(np.float64) * y)
        res = 16 * U * mag.max() / gamma
        thr = gamma * theta if kind != oracle.BOX else 0.0
        near = np.abs(u - thr) <= 8 * U * mag.max()
        if kind == oracle.BOX:
            near |= np.abs(u - gamma * z) <= 8 * U * mag.max()
        err = np.abs(x - ref)
        if near.any():
            assert (err <= tol + res).all(), (kind, gamma, err.max(), u, ref, x)
        else:
            # no edge near the threshold: a few units in the last place of z
            far = 8 * U * z + 4 * U * ref
            assert (err <= far).all(), (kind, gamma, err.max(), far[err.argmax()], u, ref, x)
            worst = max(worst, (err / far).max())
    print(f"kind={kind} gamma={gamma}: rows off the threshold, worst error / (8u z + 4u x) = {worst:.3f}")


def test_plain_fp32_values_would_not_do():
    # The reason for the float pairs: rows whose u is large and whose values
    # cancel to within gamma z lose |u| eps / gamma of x without the low parts;
    # dropping them (u_l = 0) breaks the tolerance on such a row.
    rng = np.random.default_rng(5)
    gamma, z = 1e-3, 1.0
    failures = 0
    for _ in range(200):
        c, a, y = adversarial_row(rng, gamma, z)
        u = -(c.astype(np.float64) + a.astype(np.float64) * y.astype(np.float64))
        ref, _ = oracle.project(u / gamma, oracle.SIMPLEX_EQ, z)
        uh = np.array([u_pair(c[k], a[k], y[k])[0] for k in range(c.shape[0])], F)
        plain, _ = oracle.project(uh.astype(np.float64) / gamma, oracle.SIMPLEX_EQ, z)
        if (np.abs(plain - ref) > 2e-6 * z + 4 * U * ref).any():
            failures += 1
    assert failures > 0
