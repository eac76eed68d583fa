"""The learned warm start on the GPU against the FP64 reference
(oracle/mlp.py) and against the method without it.

Tolerances.  The kernels round to bfloat16 at the points the reference's
``bf16_round`` mode rounds; what remains is FP32 accumulation against FP64
(relative ~1e-6) and the rare bfloat16 rounding decision that the two orders
take differently (one unit in the 8th bit of one activation), so outputs agree
to 2e-3 relative and gradients to 1e-2 relative in norm.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_cases import mixed_instance, oracle_problem, to_device
from oracle import mlp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def random_rows(n, seed=5):
    rng = np.random.default_rng(seed)
    X = np.empty((n, mlp.F), dtype=np.float32)
    X[:, 0] = rng.uniform(2, 9, n)
    X[:, 1] = rng.uniform(3, 11, n)
    X[:, 2] = rng.uniform(0.5, 2, n)
    X[:, 3] = X[:, 2] + rng.uniform(0, 3, n)
    X[:, 4] = np.where(rng.uniform(size=n) < 0.2, 0.0, rng.uniform(0, 1.5, n))
    X[:, 5] = np.log(1e-2)
    X[:, 6] = rng.normal(0, 0.05, n)
    y = np.maximum(X[:, 4] * (1 + 2 * X[:, 6]) + 0.05 * np.tanh(X[:, 0] - 5), 0).astype(np.float32)
    return X, y


def ws_with_random_params(dlm, H=128, seed=11, n=2000):
    ws = dlm.WarmStart(H, seed)
    rng = np.random.default_rng(seed)
    P = mlp.init_params(H, seed)
    P["w3"] = rng.normal(0, 0.3, H)
    P["b1"] = rng.normal(0, 0.1, H)
    P["b2"] = rng.normal(0, 0.1, H)
    P["b3"] = np.array([0.05])
    X, y = random_rows(n)
    mu, sd = mlp.normalizer(X.astype(np.float64))
    ws.set_params(ws.pack(P), mu, sd)
    th, mu32, sd32 = ws.params()
    return ws, {k: v.astype(np.float64) for k, v in ws.unpack(th).items()}, X, y, mu32.astype(np.float64), \
        sd32.astype(np.float64)


@pytest.mark.parametrize("bf16", [False, True])
def test_features_match_oracle(dlm_lib, bf16):
    inst = mixed_instance()
    rp, col, c, a, b = to_device(inst, torch, bf16)
    s = dlm_lib.Solver(rp, col, c, a, b, inst.J, bf16=bf16)
    rng = np.random.default_rng(3)
    lam = rng.uniform(0, 1, inst.J).astype(np.float32)
    gamma = 1e-2
    X = dlm_lib.WarmStart.features(s, torch.from_numpy(lam).cuda(), gamma).cpu().numpy().astype(np.float64)
    p = oracle_problem(inst, bf16=bf16)
    ref_grad = oracle.sweep(p, lam.astype(np.float64), gamma)["grad"]
    R = mlp.item_features(p.row_ptr, p.col, p.c, p.J, p.b, lam, gamma, ref_grad)
    deg = np.bincount(p.col, minlength=p.J)
    assert np.array_equal(np.expm1(X[:, 1]).round(), deg)
    assert np.array_equal(X[:, 3].astype(np.float32), R[:, 3].astype(np.float32))  # max is exact
    for f in (0, 1, 2, 5):
        assert np.allclose(X[:, f], R[:, f], rtol=2e-7, atol=1e-7), f
    assert np.array_equal(X[:, 4], lam.astype(np.float64))
    # the gradient feature carries the solver's FP32 gradient tolerance
    gtol = 1e-5 * (np.abs(p.b) + np.bincount(p.col, weights=np.abs(p.a), minlength=p.J)) / (1 + p.b) + 1e-6
    assert (np.abs(X[:, 6] - R[:, 6]) <= gtol).all()
    s.close()


def test_forward_matches_oracle(dlm_lib):
    ws, P, X, y, mu, sd = ws_with_random_params(dlm_lib)
    out = ws.predict(torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    ref = mlp.predict(P, X.astype(np.float64), mu, sd, bf16_round=True)
    # bulk: FP32 against FP64 accumulation; a few rows carry one bfloat16
    # rounding decision taken the other way (one unit in the 8th bit of an
    # activation of size <= 4, times weights of size <= 1)
    err = np.abs(out - ref)
    assert np.quantile(err / (np.abs(ref) + 0.1), 0.99) <= 1e-4, np.quantile(err, 0.99)
    assert (err <= 5e-3 * (np.abs(ref) + 0.1)).all(), err.max()
    # the FP64 network without rounding is close too (the BF16 error statement)
    ref64 = mlp.predict(P, X.astype(np.float64), mu, sd)
    assert np.abs(out - ref64).max() <= 0.05 * np.abs(ref64).max()
    ws.close()


def test_gradient_matches_oracle(dlm_lib):
    ws, P, X, y, mu, sd = ws_with_random_params(dlm_lib)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    loss, g = ws.loss_grad(Xd, yd)
    rl, rg = mlp.loss_and_grad(P, X.astype(np.float64), y.astype(np.float64), mu, sd, bf16_round=True)
    assert abs(loss - rl) <= 1e-4 * rl
    G = ws.unpack(g)
    for k in rg:
        d = np.linalg.norm(G[k].astype(np.float64) - rg[k])
        assert d <= 1e-2 * np.linalg.norm(rg[k]) + 1e-9, (k, d / np.linalg.norm(rg[k]))
    ws.close()


@pytest.mark.parametrize("H,n", [(8, 300), (40, 1000), (136, 700), (256, 2500)])
def test_widths_and_row_counts_match_oracle(dlm_lib, H, n):
    # The tensor-core products use 128 x 128 output tiles and 64-wide K
    # slices: widths below one tile (zero-padded columns), between one and two
    # (two column tiles), two full tiles; row counts leaving a partial row
    # tile, and split-K ranges of uneven length in the gradient products.
    ws, P, X, y, mu, sd = ws_with_random_params(dlm_lib, H=H, seed=13, n=n)
    out = ws.predict(torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    ref = mlp.predict(P, X.astype(np.float64), mu, sd, bf16_round=True)
    err = np.abs(out - ref)
    assert (err <= 5e-3 * (np.abs(ref) + 0.1)).all(), err.max()
    loss, g = ws.loss_grad(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda())
    rl, rg = mlp.loss_and_grad(P, X.astype(np.float64), y.astype(np.float64), mu, sd, bf16_round=True)
    assert abs(loss - rl) <= 1e-4 * rl
    G = ws.unpack(g)
    for k in rg:
        d = np.linalg.norm(G[k].astype(np.float64) - rg[k])
        assert d <= 1e-2 * np.linalg.norm(rg[k]) + 1e-9, (k, d / np.linalg.norm(rg[k]))
    ws.close()


def test_adam_step_matches_oracle(dlm_lib):
    ws, P, X, y, mu, sd = ws_with_random_params(dlm_lib)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    _, g = ws.loss_grad(Xd, yd)
    th0, _, _ = ws.params()
    lr = 1e-3
    ws.train(Xd, yd, 1, lr)
    th1, _, _ = ws.params()
    # Adam's first step from the GPU gradient, in FP64: theta - lr g / (|g| + eps)
    want = th0.astype(np.float64) - lr * g / (np.abs(g.astype(np.float64)) + 1e-8)
    assert np.abs(th1 - want).max() <= 1e-6
    ws.close()


def test_training_is_deterministic_and_learns(dlm_lib):
    X, y = random_rows(6000, seed=8)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    runs = []
    for _ in range(2):
        ws = dlm_lib.WarmStart(128, 7)
        losses = ws.train(Xd, yd, 400, 2e-3)
        runs.append((losses, ws.params()[0]))
        ws.close()
    assert np.array_equal(runs[0][1], runs[1][1]) and np.array_equal(runs[0][0], runs[1][0])
    losses = runs[0][0]
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])


def test_learned_start_gain(dlm_lib):
    """Recurring daily instances (60,000 users x 200 items, gamma 1e-3): the
    network trains on days 1-10 and is evaluated on days 13-18.  What it
    gains over the previous day's dual (the fallback it replaces): started
    at gamma_end (the solve the start feeds directly), it reaches the 1e-4
    certified gap in more than one gap-check interval fewer iterations
    (measured: 847 against 952).  Also reported, not asserted: the relative
    L1 distance of each start to the day's optimum, and the iterations when
    each warm start enters the gamma continuation it picks on days 11-12
    (held out from the network) -- both pick the cold start's continuation,
    and on this instance all three then need about the same iterations (610
    to 625).  Every solve: row normalization, a check every 10 iterations,
    warm starts with the adaptive restart."""
    g_end, gap_every = 1e-3, 10
    inst = synth.generate(synth.recipe_daily(I=60_000, J=200, seed=77))
    days = [inst]
    for d in range(1, 19):
        days.append(synth.next_day(days[-1], d, seed=77))

    def solver(i):
        rp, col, c, a, b = to_device(days[i], torch)
        return dlm_lib.Solver(rp, col, c, a, b, days[i].J)

    labels, feats = [], []
    for i in range(19):
        s = solver(i)
        s.set_options(precondition=True, gap_every=gap_every, restart=True)
        if i == 0:
            s.set_schedule(1e-1, g_end, 0.5, 50)
        else:
            s.set_schedule(g_end)
            s.set_lambda(labels[-1])
            feats.append(dlm_lib.WarmStart.features(s, labels[-1], g_end))
        st = s.solve(1e-6, 30_000)
        assert st.status in (dlm_lib.DLM_OK, dlm_lib.DLM_ERR_TIMEOUT) and st.rel_gap <= 1e-4
        labels.append(s.lam())
        s.close()
    ws = dlm_lib.WarmStart(128, 1)
    losses = ws.train(torch.cat(feats[:10]), torch.cat(labels[1:11]), 300, 1e-3)
    assert losses[-1] < 0.5 * losses[0]

    def start_of(i, mode):
        return labels[i - 1] if mode == "prev" else ws.predict(feats[i - 1])

    def iters(i, mode, sched):
        s = solver(i)
        s.set_options(precondition=True, gap_every=gap_every, restart=mode != "cold")
        s.set_schedule(sched[0], g_end, sched[1], sched[2])
        if mode != "cold":
            s.set_lambda(start_of(i, mode))
        st = s.solve(1e-4, 100_000)
        assert st.status == dlm_lib.DLM_OK
        s.close()
        return st.iter

    evald = range(13, 19)
    dist = {m: float(np.mean([((start_of(i, m) - labels[i]).abs().sum() / labels[i].abs().sum()).item()
                              for i in evald])) for m in ("prev", "learned")}
    fixed = (g_end, 1.0, 1 << 30)
    at_end = {m: float(np.mean([iters(i, m, fixed) for i in evald])) for m in ("prev", "learned")}
    cands = [(1e-1, 0.5, 50), (1e-1, 0.25, 25), (1e-2, 0.5, 25), fixed]
    chosen = {m: cands[int(np.argmin([np.mean([iters(i, m, c) for i in (11, 12)]) for c in cands]))]
              for m in ("prev", "learned")}
    cont = {m: float(np.mean([iters(i, m, chosen[m]) for i in evald])) for m in ("prev", "learned")}
    cont["cold"] = float(np.mean([iters(i, "cold", (1e-1, 0.5, 50)) for i in evald]))
    print(f"distance to the optimum {dist}; iterations at gamma_end {at_end}; "
          f"with continuations {chosen}: {cont}")
    assert at_end["learned"] <= at_end["prev"] - gap_every
    ws.close()
