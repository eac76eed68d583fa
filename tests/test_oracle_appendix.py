"""The oracle on an instance of the appendix generator (App. A): resource
rows of A three orders of magnitude apart, greedy-load capacities.  With the
row normalization (per-item steps, App. B.2) the accelerated method reaches a
small certified gap; with the plain step 1/L, set by the largest row, it does
not move the small rows' duals (the comparison of the paper's
preconditioning figure).  CPU only."""
import numpy as np

import oracle
import synth


def test_row_normalization_on_the_appendix_instance():
    inst = synth.generate_appendix(synth.AppRecipe(I=20_000, J=300, seed=31))
    p = oracle.Problem(inst.row_ptr, inst.col, inst.c.astype(np.float64), inst.a.astype(np.float64), inst.b,
                       inst.J, oracle.SIMPLEX_LE, 1.0)
    rn = np.sqrt(oracle.row_sq(p))
    assert np.quantile(rn[rn > 0], 0.99) / np.quantile(rn[rn > 0], 0.01) > 100  # rows far apart in norm
    T = 1000
    pre = oracle.fista(p, T, 1e-2, precondition=True, trajectory=False, restart=True)
    plain = oracle.fista(p, T, 1e-2, precondition=False, trajectory=False, restart=True)
    g_pre = oracle.certify(p, pre["lam"], 1e-2)["rel_gap"]
    g_plain = oracle.certify(p, plain["lam"], 1e-2)["rel_gap"]
    assert g_pre <= 1e-4, g_pre
    assert g_plain >= 0.1, g_plain
