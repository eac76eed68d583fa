"""The first pass over a row keeps its K largest u (K = 4 by default, 8 with
topk = 8) and fixes the active set from them when it has fewer than K edges.
On rows with at most three active edges both widths take the same decisions
and the same arithmetic (the threshold over the recorded edges in float-pair
arithmetic), so they must agree bit for bit: a check that neither width's
record is wrong on near ties.  The rows are built to hit them: equal and
ulp-apart top values, second and third values within a few ulps or 1e-5
relative of the threshold, values at powers of two, the count dual's floor,
exactly equal values below the active set, and short rows whose padding fills
the record.  With lambda = 0 every u is -c exactly."""
import numpy as np
import pytest

import oracle
import synth
from gpu_cases import oracle_problem, to_device, x_error_report

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GAMMA = 1e-3


def ulp_steps(v, k):
    """v moved k float32 ulps (k < 0: down)."""
    v = np.float32(v)
    for _ in range(abs(int(k))):
        v = np.nextafter(v, np.float32(np.inf if k > 0 else -np.inf))
    return np.float32(v)


def crafted_rows(seed, I, J, floor=0.0):
    """u of each row (float32), built so that at most three edges are active at
    gamma = GAMMA, z = 1, and near ties sit where the scan decides."""
    rng = np.random.default_rng(seed)
    gz = np.float32(GAMMA)
    rows = []
    for i in range(I):
        d = int(rng.integers(1, 41)) if rng.uniform() < 0.9 else int(rng.integers(41, 300))
        kind = i % 6
        base = np.float32(rng.choice([0.5, 1.0, 2.0, rng.uniform(0.4, 1.2)]))
        if kind == 1 and rng.uniform() < 0.5:
            base = ulp_steps(base, -1)  # just below a bucket / power-of-two edge
        u = rng.uniform(0.05, float(base) - 0.05, size=d).astype(np.float32)
        if kind == 0:  # generic
            u = rng.uniform(0.05, 1.2, size=d).astype(np.float32)
        elif kind == 1:  # a tie group of 1..3 at the top: equal or a few ulps apart
            m = min(d, int(rng.integers(1, 4)))
            for q in range(m):
                u[q] = ulp_steps(base, int(rng.choice([0, 0, -1, -2, 3])))
        elif kind in (2, 3):  # the next value within a few ulps (or 1e-5 relative) of the threshold
            u[0] = base
            if d > 1:
                tau1 = np.float32(base - gz)
                u[1] = ulp_steps(tau1, int(rng.integers(-3, 4))) if kind == 2 else \
                    np.float32(tau1 * (1 + rng.choice([-1e-5, 1e-5, 3e-6])))
            if d > 2 and kind == 3:
                u[2] = np.float32(u[1] - rng.choice([1e-7, 2e-3]))
        elif kind == 4:  # the largest u within a few ulps of the floor (count dual)
            u[0] = ulp_steps(np.float32(floor if floor > 0 else base), int(rng.integers(-2, 3)))
        else:  # exactly equal values below the active set (padding-free duplicates)
            u[:] = np.float32(rng.uniform(0.1, 0.3))
            u[0] = base
        rng.shuffle(u)
        # keep rows whose active set (FP64, sort rule) has at most three edges
        # with a margin: the fourth value lies clearly below the threshold
        srt = np.sort(u.astype(np.float64) - 0.0)[::-1]
        r = 1
        while r < len(srt) and srt[r] > (srt[:r].sum() - GAMMA) / r:
            r += 1
        if r >= 4 or (len(srt) > 3 and srt[3] > (srt[:3].sum() - GAMMA) / 3 - 1e-4):
            u = np.array([base], np.float32)
        rows.append(u)
    deg = np.array([len(u) for u in rows])
    rp = np.zeros(I + 1, np.int64)
    np.cumsum(deg, out=rp[1:])
    col = np.concatenate([rng.choice(J, size=len(u), replace=False) for u in rows]).astype(np.int32)
    c = -np.concatenate(rows).astype(np.float32)
    a = rng.uniform(0.5, 1.5, size=rp[-1]).astype(np.float32)
    b = np.bincount(col, weights=a, minlength=J) * 0.05 + 1.0
    return synth.Instance(rp, col, c, a, b, J)


@pytest.mark.parametrize("kind,M,mu", [(oracle.SIMPLEX_LE, None, 0.0), (oracle.SIMPLEX_EQ, None, 0.0),
                                       (oracle.BOX, None, 0.0), (oracle.SIMPLEX_LE, 500.0, 0.3)])
def test_four_and_eight_wide_records_agree_bit_for_bit(dlm_lib, kind, M, mu):
    inst = crafted_rows(11, 6000, 400, floor=mu)
    rp, col, c, a, b = to_device(inst, torch)
    out = {}
    for topk in (4, 8):
        s = dlm_lib.Solver(rp, col, c, a, b, inst.J, kind=kind)
        if M is not None:
            s.set_count_limit(M)
        s.set_options(topk=topk)
        lam = torch.zeros(s.dual_dim, dtype=torch.float32, device="cuda")
        if M is not None:
            lam[-1] = mu
        g, grad, x = s.calculate(lam, GAMMA)
        # one iteration of the solver from lambda = 0 (the iteration sweep)
        s.set_schedule(GAMMA)
        s.step(1)
        lam1, y1, _ = s.get_state()
        out[topk] = (g, grad.cpu().numpy(), x.cpu().numpy(), lam1.cpu().numpy(), y1.cpu().numpy())
        s.close()
    g4, grad4, x4, l4, y4 = out[4]
    g8, grad8, x8, l8, y8 = out[8]
    assert g4 == g8
    np.testing.assert_array_equal(grad4, grad8)
    np.testing.assert_array_equal(x4, x8)
    np.testing.assert_array_equal(l4, l8)
    np.testing.assert_array_equal(y4, y8)
    # and both are the oracle's sweep within the parity tolerance
    p = oracle_problem(inst, kind, 1.0)
    if M is not None:
        p = oracle.Problem(p.row_ptr, p.col, p.c, p.a, p.b, p.J, kind, 1.0, M=M)
    # the count dual as the kernel saw it (its float32 value)
    mu32 = float(np.float32(mu))
    lam64 = np.zeros(p.J + (1 if M is not None else 0))
    if M is not None:
        lam64[-1] = mu32
    ref = oracle.sweep(p, lam64, GAMMA)
    pc = oracle.Problem(p.row_ptr, p.col, p.c + mu32, p.a, p.b, p.J, kind, 1.0)
    dx, tol = x_error_report(x4, ref["x"], pc, np.zeros(p.J), GAMMA)
    assert (dx <= tol).all(), f"{int((dx > tol).sum())} edges over tolerance, max {dx.max():.3e}"


