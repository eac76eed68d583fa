"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (same layout, kernels, grid and block): after 20 iterations (400 on the
appendix instance), x(lam) of a seeded user sample against the FP64 oracle
evaluated one user at a time, and
properties that hold at any size over the whole instance (the gradient equals
A x - b of the solver's own x; weak duality of the certificate)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_cases import x_error_report

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

WORKLOADS = {
    # instance, storage, gamma schedule and row normalization as bench.py runs
    # them, and the iterations before the check (the appendix instance is
    # checked once half of its rows have four or more active edges)
    "production": (lambda: synth.generate(synth.recipe_production()), False, (1e-1, 1e-3, 0.5, 100), False, 20),
    "precision": (lambda: synth.generate(synth.recipe_precision()), True, (1e-3, 1e-3, 0.5, 1 << 30), False, 20),
    "appendix": (lambda: synth.generate_appendix(synth.recipe_appendix()), False, (1e-2, 1e-2, 0.5, 1 << 30), True,
                 400),
    # the box cut by a per-user budget {0 <= x <= 0.5, sum x <= 1} on the production shape
    "boxcut": (lambda: synth.generate(synth.recipe_production()), True, (1e-3, 1e-3, 0.5, 1 << 30), False, 20),
}
SETS = {"boxcut": dict(kind=oracle.BOX_CUT, z=0.5, cut=1.0)}


def rows_index(rp, rows):
    """Edge positions of the given rows (device tensors), in order."""
    starts, ends = rp[rows], rp[rows + 1]
    lens = ends - starts
    total = int(lens.sum().item())
    return torch.repeat_interleave(starts, lens) + (
        torch.arange(total, device=rp.device) - torch.repeat_interleave(torch.cumsum(lens, 0) - lens, lens))


@pytest.mark.parametrize("name", ["production", "precision", "appendix", "boxcut"])
def test_full_size_sampled_parity(dlm_lib, name):
    make, bf16, sched, precondition, iters = WORKLOADS[name]
    sset = SETS.get(name, dict(kind=oracle.SIMPLEX_LE, z=1.0, cut=None))
    inst = make()
    dev = torch.device("cuda")
    if bf16:
        c = torch.from_numpy(synth.round_bf16(inst.c).view(np.int16)).to(dev).view(torch.bfloat16)
        a = torch.from_numpy(synth.round_bf16(inst.a).view(np.int16)).to(dev).view(torch.bfloat16)
    else:
        c, a = torch.from_numpy(inst.c).to(dev), torch.from_numpy(inst.a).to(dev)
    rp = torch.from_numpy(inst.row_ptr).to(dev)
    col = torch.from_numpy(inst.col).to(dev)
    b = torch.from_numpy(inst.b).to(dev)
    s = dlm_lib.Solver(rp, col, c, a, b, inst.J, bf16=bf16, kind=sset["kind"], z=sset["z"], cut=sset["cut"])
    s.set_schedule(*sched)
    s.set_options(precondition=precondition)
    s.step(iters)
    lam32 = s.lam()
    st = s.stats()
    gamma = st.gamma
    assert st.status == dlm_lib.DLM_OK and st.rel_gap >= -1e-9  # weak duality
    g, grad, x = s.calculate(lam32, gamma)
    # gradient = A x - b of the same x, summed in FP64 over all 10^8-10^9 edges
    av = a.float() if bf16 else a
    ax = torch.zeros(inst.J, dtype=torch.float64, device=dev)
    ax.index_add_(0, col.long(), (av * x).double())
    dg = (grad.double() - (ax - b)).abs()
    assert float((dg - 2e-6 * (ax + b.abs()) - 1e-6).max().item()) <= 0.0
    # x of a seeded 0.1 % user sample against the FP64 oracle, one user at a time
    ids = synth.sample_users(inst.I, 0.001, 777)
    xs = x[rows_index(rp, torch.from_numpy(ids).to(dev))].cpu().numpy()
    sub = synth.subset(inst, ids)
    cs, as_ = sub.c, sub.a
    if bf16:
        cs, as_ = synth.bf16_to_f32(synth.round_bf16(cs)), synth.bf16_to_f32(synth.round_bf16(as_))
    p = oracle.Problem(sub.row_ptr, sub.col, cs.astype(np.float64), as_.astype(np.float64), sub.b, sub.J,
                       sset["kind"], sset["z"], cut=sset["cut"] if sset["cut"] is not None else np.inf)
    lam = lam32.cpu().numpy().astype(np.float64)
    ref = oracle.sweep(p, lam, gamma)
    dx, tol = x_error_report(xs, ref["x"], p, lam, gamma, cap=sset["z"] if sset["cut"] is not None else None)
    assert (dx <= tol).all(), f"{int((dx > tol).sum())} of {dx.size} sampled edges over tolerance, max {dx.max():.3e}"
    s.close()


def test_full_size_two_families_sampled_parity(dlm_lib):
    # the families workload: the production shape (20M x 2,000, BF16) with a
    # second coefficient a2 = U(0.1, 2) per edge and b2_j = 0.05 sum_i a2_ij,
    # gamma = 1e-3, the general multi-family sweep
    inst = synth.generate(synth.recipe_production())
    a2 = (0.1 + 1.9 * synth.uniforms(1005, 0, 7, inst.nnz)).astype(np.float32)
    c16, a16, a216 = synth.round_bf16(inst.c), synth.round_bf16(inst.a), synth.round_bf16(a2)
    b2 = 0.05 * np.bincount(inst.col, weights=synth.bf16_to_f32(a216).astype(np.float64), minlength=inst.J)
    dev = torch.device("cuda")
    pair = np.stack([a16, a216], axis=1)
    c = torch.from_numpy(c16.view(np.int16)).to(dev).view(torch.bfloat16)
    a = torch.from_numpy(pair.view(np.int16)).to(dev).view(torch.bfloat16)
    rp = torch.from_numpy(inst.row_ptr).to(dev)
    col = torch.from_numpy(inst.col).to(dev)
    b = torch.from_numpy(np.ascontiguousarray(np.stack([inst.b, b2]))).to(dev)
    s = dlm_lib.Solver(rp, col, c, a, b, inst.J, bf16=True)
    s.set_schedule(1e-3)
    s.step(20)
    lam32 = s.lam()
    st = s.stats()
    assert st.status == dlm_lib.DLM_OK and st.rel_gap >= -1e-9
    g, grad, x = s.calculate(lam32, 1e-3)
    J = inst.J
    af = a.float()
    for f in range(2):
        ax = torch.zeros(J, dtype=torch.float64, device=dev)
        ax.index_add_(0, col.long(), (af[:, f] * x).double())
        dg = (grad[f * J:(f + 1) * J].double() - (ax - b[f])).abs()
        assert float((dg - 2e-6 * (ax + b[f].abs()) - 1e-6).max().item()) <= 0.0, f
    ids = synth.sample_users(inst.I, 0.001, 778)
    eidx = rows_index(rp, torch.from_numpy(ids).to(dev))
    xs = x[eidx].cpu().numpy()
    sub = synth.subset(inst, ids)
    e_host = eidx.cpu().numpy()
    A = np.stack([synth.bf16_to_f32(a16[e_host]), synth.bf16_to_f32(a216[e_host])], axis=1).astype(np.float64)
    cs = synth.bf16_to_f32(c16[e_host]).astype(np.float64)
    p = oracle.Problem(sub.row_ptr, sub.col, cs, A, np.stack([inst.b, b2]), J)
    lam = lam32.cpu().numpy().astype(np.float64)
    ref = oracle.sweep(p, lam, 1e-3)
    # allowance at |c| + |a2 lam2|, as in the small two-family parity tests
    proxy = oracle.Problem(p.row_ptr, p.col, np.abs(cs) + np.abs(A[:, 1] * lam[J:][p.col]), A[:, 0], inst.b, J)
    dx, tol = x_error_report(xs, ref["x"], proxy, lam[:J], 1e-3)
    assert (dx <= tol).all(), f"{int((dx > tol).sum())} of {dx.size} sampled edges over tolerance, max {dx.max():.3e}"
    s.close()
