"""The per-row arithmetic of the general iteration sweep (csrc/sweep.cu:
the first pass's top-K record, the mode decision, the threshold over the
recorded edges, the Michelot iteration beyond them), emulated in IEEE FP32
with numpy and checked against the oracle's FP64 projection (Sec. 3.2 Eq.
primal-recovery; Sec. 4.3's simplex threshold).  u = -fma(a, y, c) ranks
the edges; the threshold is recomputed in float-pair arithmetic (TwoSum,
TwoProduct) over the final active set; x = ((u_h - tau) + (u_l - taul)) /
gamma.  The claims checked: on rows with no edge within FP32 resolution of
the threshold, x is within 8u z + 4u x (u = 2^-24) of the FP64 projection
however large the values; on the others, within the GPU parity tests'
tolerance; the four- and eight-wide records give the same x; and the
Michelot iteration, which can alternate between two active sets whose
FP32 thresholds round past each other (values of 40 clustered within
gamma z = 1e-3), reaches its pass cap only on such rows, whose x the cap's
fallback (the threshold over the current set) keeps within the tolerance.
The allocation-free entry point (csrc/noalloc.cu), whose warp-per-user
iteration stops once the threshold no longer rises, reaches that stop on
every row within d + 1 passes, with x within the same tolerances.  The
kernels are held to the oracle by the GPU tests; this test pins the
arithmetic they follow on adversarial rows."""
import numpy as np
import pytest

import oracle
from test_offset_threshold import F, U, adversarial_row, f32, u_pair


def two_sum(a, b):
    s = f32(a + b)
    bp = f32(s - a)
    return s, f32(f32(a - f32(s - bp)) + f32(b - bp))


def f2_add(p, q):
    s, e = two_sum(p[0], q[0])
    return s, f32(e + f32(p[1] + q[1]))


def f2_threshold(ps, gzh, gzl, n):
    """(sum - gamma z) / n for a pair sum, the quotient's remainder by FMA."""
    num = f2_add(ps, (f32(-gzh), f32(-gzl)))
    fn = f32(n)
    th = f32(num[0] / fn)
    r = f32(np.float64(-th) * np.float64(fn) + np.float64(num[0]))  # exact: fma remainder of a division
    return th, f32(f32(r + num[1]) / fn)


def fma_u(c, a, y):
    """-fma(a, y, c): the value the sweep ranks and tests edges by."""
    return f32(-(np.float64(a) * np.float64(y) + np.float64(c)))


CAPPED = []  # rows whose Michelot iteration ran to the pass cap


def row_x(c, a, y, kind, z, gamma, K):
    g = np.float64(gamma)
    gz = f32(g * z)
    gzl = f32(g * z - np.float64(gz))
    invg = f32(1.0 / g)
    n = c.shape[0]
    box, eq = kind == oracle.BOX, kind == oracle.SIMPLEX_EQ
    u = np.array([fma_u(c[k], a[k], y[k]) for k in range(n)], F)
    pairs = [u_pair(c[k], a[k], y[k]) for k in range(n)]
    # first pass: the K largest values, positions of the first K - 1 (strict
    # comparisons: among equal values the earlier edge ranks first)
    tv = [F(-np.inf)] * K
    tid = [0] * (K - 1)
    for k in range(n):
        x, xi = u[k], k
        for q in range(K - 1):
            if x > tv[q]:
                tv[q], x = x, tv[q]
                tid[q], xi = xi, tid[q]
        tv[K - 1] = max(tv[K - 1], x)
    v0 = tv[0]
    xs = np.zeros(n, F)
    if box:
        mode = 3 if v0 > 0 else 0
    elif v0 == -np.inf or (not eq and v0 <= 0):
        mode = 0
    else:
        sm, r, tau = v0, 1, f32(v0 - gz)
        for q in range(1, K):
            if r == q and tv[q] > tau:
                sm = f32(sm + tv[q])
                r = q + 1
                tau = f32(f32(sm - gz) / f32(q + 1))
        mode = 1 if (r == 1 and (eq or tau >= 0)) else (2 if r < K else 3)
    if mode == 0:
        return xs
    if mode == 1:
        xs[tid[0]] = f32(z)
        return xs
    taul = f32(0)
    if mode == 2:
        zero = not eq and tau <= 0
        if not zero:
            ps = (f32(0), f32(0))
            for i in range(r):
                ps = f2_add(ps, pairs[tid[i]])
            th, tl = f2_threshold(ps, gz, gzl, r)
            if not eq and f32(th + tl) <= 0:
                zero = True
            else:
                tau, taul = th, tl
        if zero:
            tau, taul = f32(0), f32(0)
        for i in range(r):
            k = tid[i]
            d = f32(f32(pairs[k][0] - tau) + f32(pairs[k][1] - taul))
            xs[k] = max(d, F(0)) * invg
        return xs
    # mode 3: Michelot from tau_K (the box: tau = 0 directly)
    zero = box
    if not box:
        prevn, settled, psum, cnt = -1, False, (f32(0), f32(0)), 0
        for _ in range(256):
            sm, cnt, ps = f32(0), 0, (f32(0), f32(0))
            for k in range(n):
                if u[k] > tau:
                    sm = f32(sm + u[k])
                    cnt += 1
                    ps = f2_add(ps, pairs[k])
            psum = ps
            if cnt == prevn or cnt == 0:
                settled = True
                break
            prevn = cnt
            tn = f32(f32(sm - gz) / f32(cnt))
            if tn == tau:
                settled = True
                break
            tau = tn
        if not settled:  # the pass cap: the threshold over the current set
            CAPPED.append(n)
            psum, cnt = (f32(0), f32(0)), 0
            for k in range(n):
                if u[k] > tau:
                    psum = f2_add(psum, pairs[k])
                    cnt += 1
        zero = not eq and tau <= 0
        if not zero:
            th, tl = f2_threshold(psum, gz, gzl, max(cnt, 1))
            if not eq and f32(th + tl) <= 0:
                zero = True
            else:
                tau, taul = th, tl
    if zero:
        tau, taul = f32(0), f32(0)
    for k in range(n):
        if u[k] > tau:
            d = f32(f32(pairs[k][0] - tau) + f32(pairs[k][1] - taul))
            xk = f32(d * invg)
            xs[k] = min(max(xk, F(0)), f32(z)) if box else max(d, F(0)) * invg
    return xs


@pytest.mark.parametrize("kind,z", [(oracle.SIMPLEX_LE, 1.0), (oracle.SIMPLEX_EQ, 0.7), (oracle.BOX, 0.6)])
@pytest.mark.parametrize("gamma", [1e-1, 1e-2, 1e-3])
def test_topk_threshold_matches_fp64_projection(kind, z, gamma):
    rng = np.random.default_rng(40 + int(-np.log10(gamma)) + 7 * kind)
    worst = 0.0
    capped = 0
    for _ in range(300):
        c, a, y = adversarial_row(rng, gamma, z)
        before = len(CAPPED)
        x4 = row_x(c, a, y, kind, z, gamma, 4)
        x8 = row_x(c, a, y, kind, z, gamma, 8)
        hit_cap = len(CAPPED) > before
        u = -(c.astype(np.float64) + a.astype(np.float64) * y.astype(np.float64))
        ref, theta = oracle.project(u / gamma, kind, z)
        mag = np.abs(c.astype(np.float64)) + np.abs(a.astype(np.float64) * y)
        thr = gamma * theta if kind != oracle.BOX else 0.0
        near = np.abs(u - thr) <= 8 * U * mag.max()
        if kind == oracle.BOX:
            near |= np.abs(u - gamma * z) <= 8 * U * mag.max()
        # the Michelot iteration runs to its pass cap only where FP32 cannot
        # separate the active set (two sets whose thresholds round past each
        # other): rows with an edge within that resolution of the threshold
        if hit_cap:
            capped += 1
            assert near.any(), (kind, gamma, u)
        for x in (x4, x8):
            err = np.abs(x.astype(np.float64) - ref)
            if near.any():
                tol = 2e-6 * z + 4 * U * ref + 16 * U * mag.max() / gamma
                assert (err <= tol).all(), (kind, gamma, err.max(), u, ref, x)
            else:
                far = 8 * U * z + 4 * U * ref
                assert (err <= far).all(), (kind, gamma, err.max(), far[err.argmax()], u, ref, x)
                worst = max(worst, (err / far).max())
        if not near.any():
            # off the threshold both records reach the same active set; the
            # sums then run over it in another order, so agree to rounding
            assert np.abs(x4.astype(np.float64) - x8).max() <= 8 * U * z + 4 * U * ref.max()
    print(f"kind={kind} gamma={gamma}: rows off the threshold, worst error / (8u z + 4u x) = {worst:.3f}; "
          f"rows at the pass cap: {capped}")


def static_row_x(c, a, y, kind, z, gamma, monotone=True):
    """x of one row by the allocation-free entry point's arithmetic
    (noalloc.cu: the Michelot iteration from max u - gamma z, at most d + 1
    passes), and whether the iteration stopped before that bound."""
    g = np.float64(gamma)
    gz = f32(g * z)
    gzl = f32(g * z - np.float64(gz))
    invg = f32(1.0 / g)
    d = c.shape[0]
    box, eq = kind == oracle.BOX, kind == oracle.SIMPLEX_EQ
    u = np.array([fma_u(c[k], a[k], y[k]) for k in range(d)], F)
    pairs = [u_pair(c[k], a[k], y[k]) for k in range(d)]
    tau, taul, zero, stopped = f32(0), f32(0), box, True
    if not box:
        m = u.max()
        if eq or m > 0:
            tau = f32(m - gz)
            prevn, stopped = -1, False
            for _ in range(d + 1):
                sel = u > tau
                cnt = int(sel.sum())
                sm = f32(0)
                for k in range(d):
                    if sel[k]:
                        sm = f32(sm + u[k])
                if cnt == prevn or cnt == 0:
                    stopped = True
                    break
                prevn = cnt
                tn = f32(f32(sm - gz) / f32(cnt))
                if (not tn > tau) if monotone else tn == tau:
                    stopped = True
                    break
                tau = tn
            zero = not eq and tau <= 0
            if not zero:
                ps, cnt = (f32(0), f32(0)), 0
                for k in range(d):
                    if u[k] > tau:
                        ps = f2_add(ps, pairs[k])
                        cnt += 1
                th, tl = f2_threshold(ps, gz, gzl, max(cnt, 1))
                if not eq and f32(th + tl) <= 0:
                    zero = True
                else:
                    tau, taul = th, tl
        else:
            zero = True
    if zero:
        tau, taul = f32(0), f32(0)
    x = np.zeros(d, F)
    for k in range(d):
        if u[k] > tau:
            h, l = pairs[k]
            if box:
                x[k] = min(max(f32(f32(h + l) * invg), F(0)), f32(z))
            elif zero:
                x[k] = max(f32(h + l), F(0)) * invg
            else:
                x[k] = max(f32(f32(h - tau) + f32(l - taul)), F(0)) * invg
    return x, stopped


@pytest.mark.parametrize("kind,z", [(oracle.SIMPLEX_LE, 1.0), (oracle.SIMPLEX_EQ, 0.7), (oracle.BOX, 0.6)])
@pytest.mark.parametrize("gamma", [1e-2, 1e-3])
def test_static_entry_point_iteration_stops_and_matches(kind, z, gamma):
    # the allocation-free entry point stops its iteration once the threshold
    # no longer rises: every row reaches that stop within d + 1 passes, with x
    # within the tolerances above; the stop on equality alone lets rows
    # alternate between two sets until the bound
    rng = np.random.default_rng(60 + int(-np.log10(gamma)) + 7 * kind)
    alternating = 0
    for _ in range(300):
        c, a, y = adversarial_row(rng, gamma, z)
        x, stopped = static_row_x(c, a, y, kind, z, gamma)
        assert stopped
        alternating += not static_row_x(c, a, y, kind, z, gamma, monotone=False)[1]
        u = -(c.astype(np.float64) + a.astype(np.float64) * y.astype(np.float64))
        ref, theta = oracle.project(u / gamma, kind, z)
        mag = np.abs(c.astype(np.float64)) + np.abs(a.astype(np.float64) * y)
        thr = gamma * theta if kind != oracle.BOX else 0.0
        near = np.abs(u - thr) <= 8 * U * mag.max()
        if kind == oracle.BOX:
            near |= np.abs(u - gamma * z) <= 8 * U * mag.max()
        err = np.abs(x.astype(np.float64) - ref)
        if near.any():
            assert (err <= 2e-6 * z + 4 * U * ref + 16 * U * mag.max() / gamma).all(), (kind, gamma, u, ref, x)
        else:
            assert (err <= 8 * U * z + 4 * U * ref).all(), (kind, gamma, u, ref, x)
    print(f"kind={kind} gamma={gamma}: rows the equality stop would leave alternating: {alternating}")
