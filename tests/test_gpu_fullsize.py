"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (same layout, kernels, grid and block): after 20 iterations, x(lam) of a
seeded user sample against the FP64 oracle evaluated one user at a time, and
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
    # users x items, storage, gamma schedule as bench.py runs them
    "production": (synth.recipe_production(), False, (1e-1, 1e-3, 0.5, 100)),
    "precision": (synth.recipe_precision(), True, (1e-3, 1e-3, 0.5, 1 << 30)),
}


def rows_index(rp, rows):
    """Edge positions of the given rows (device tensors), in order."""
    starts, ends = rp[rows], rp[rows + 1]
    lens = ends - starts
    total = int(lens.sum().item())
    return torch.repeat_interleave(starts, lens) + (
        torch.arange(total, device=rp.device) - torch.repeat_interleave(torch.cumsum(lens, 0) - lens, lens))


@pytest.mark.parametrize("name", ["production", "precision"])
def test_full_size_sampled_parity(dlm_lib, name):
    recipe, bf16, sched = WORKLOADS[name]
    inst = synth.generate(recipe)
    dev = torch.device("cuda")
    if bf16:
        c = torch.from_numpy(synth.round_bf16(inst.c).view(np.int16)).to(dev).view(torch.bfloat16)
        a = torch.from_numpy(synth.round_bf16(inst.a).view(np.int16)).to(dev).view(torch.bfloat16)
    else:
        c, a = torch.from_numpy(inst.c).to(dev), torch.from_numpy(inst.a).to(dev)
    rp = torch.from_numpy(inst.row_ptr).to(dev)
    col = torch.from_numpy(inst.col).to(dev)
    b = torch.from_numpy(inst.b).to(dev)
    s = dlm_lib.Solver(rp, col, c, a, b, inst.J, bf16=bf16)
    s.set_schedule(*sched)
    s.step(20)
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
    p = oracle.Problem(sub.row_ptr, sub.col, cs.astype(np.float64), as_.astype(np.float64), sub.b, sub.J)
    lam = lam32.cpu().numpy().astype(np.float64)
    ref = oracle.sweep(p, lam, gamma)
    dx, tol = x_error_report(xs, ref["x"], p, lam, gamma)
    assert (dx <= tol).all(), f"{int((dx > tol).sum())} of {dx.size} sampled edges over tolerance, max {dx.max():.3e}"
    s.close()
