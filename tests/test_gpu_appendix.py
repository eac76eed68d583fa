"""Instances of the appendix generator (App. A: resource rows of A orders of
magnitude apart, greedy-load capacities) on the GPU against the FP64 oracle,
and instances with more items than the certificate sweep holds in shared
memory at once.  At 12,000 and 19,000 items the certificate sweep's three
item arrays (24 bytes per item) exceed the 227 KB a block can hold, so its
only path is one launch per item window."""
import numpy as np
import pytest

import oracle
import synth
from gpu_cases import x_error_report

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def app_instance(I, J, seed):
    return synth.generate_appendix(synth.AppRecipe(I=I, J=J, seed=seed))


def solver(dlm, inst, kind=oracle.SIMPLEX_LE):
    d = torch.device("cuda")
    return dlm.Solver(torch.from_numpy(inst.row_ptr).to(d), torch.from_numpy(inst.col).to(d),
                      torch.from_numpy(inst.c).to(d), torch.from_numpy(inst.a).to(d),
                      torch.from_numpy(inst.b).to(d), inst.J, kind=kind)


def oproblem(inst, kind=oracle.SIMPLEX_LE):
    return oracle.Problem(inst.row_ptr, inst.col, inst.c.astype(np.float64), inst.a.astype(np.float64), inst.b,
                          inst.J, kind, 1.0)


def priced_lambda(inst, rng, scale):
    """Duals that matter on every resource: lam_j a_ij of the order of c_ij
    (a uniform lam would price the small-s_j rows at nothing and close the
    large ones)."""
    med_a = np.ones(inst.J)
    for j, v in enumerate(np.split(inst.a[np.argsort(inst.col, kind="stable")],
                                   np.cumsum(np.bincount(inst.col, minlength=inst.J))[:-1])):
        if len(v):
            med_a[j] = np.median(v)
    lam = rng.uniform(0, 2, inst.J) * scale * np.median(-inst.c) / med_a
    lam[rng.uniform(size=inst.J) < 0.2] = 0.0
    return lam.astype(np.float32)


def check_calculate(s, inst, p, lam32, gamma):
    g, grad, x = s.calculate(torch.from_numpy(lam32).cuda(), gamma)
    lam = lam32.astype(np.float64)
    ref = oracle.sweep(p, lam, gamma)
    dx, tol = x_error_report(x.cpu().numpy(), ref["x"], p, lam, gamma)
    assert (dx <= tol).all(), f"{int((dx > tol).sum())} edges over tolerance, max {dx.max():.3e}"
    scale_j = np.bincount(p.col, weights=p.a * ref["x"], minlength=p.J) + np.abs(p.b)
    allow = np.bincount(p.col, weights=p.a * np.maximum(tol - 2e-6, 0), minlength=p.J)
    dg = np.abs(grad.cpu().numpy().astype(np.float64) - ref["grad"])
    assert (dg <= 2e-6 * scale_j + allow + 1e-6).all(), f"grad max err {dg.max():.3e}"
    assert abs(g - ref["g"]) <= 2e-6 * (abs(ref["g"]) + abs(ref["obj"]) + 1e-9) + float(np.abs(p.c) @ tol)


@pytest.mark.parametrize("kind,gamma,topk", [(oracle.SIMPLEX_LE, 1e-2, 4), (oracle.SIMPLEX_LE, 1e-3, 4),
                                             (oracle.BOX, 1e-2, 4), (oracle.SIMPLEX_EQ, 1e-1, 4),
                                             (oracle.SIMPLEX_LE, 1e-2, 8), (oracle.SIMPLEX_EQ, 1e-1, 8)])
def test_calculate_on_an_appendix_instance(dlm_lib, kind, gamma, topk):
    inst = app_instance(20_000, 300, 31)
    s = solver(dlm_lib, inst, kind)
    s.set_options(topk=topk)
    p = oproblem(inst, kind)
    rng = np.random.default_rng(5)
    for scale in (0.3, 1.0, 3.0):
        check_calculate(s, inst, p, priced_lambda(inst, rng, scale), gamma)
    s.close()


@pytest.mark.parametrize("topk", [4, 8])
def test_trajectory_with_row_normalization(dlm_lib, topk):
    inst = app_instance(20_000, 300, 31)
    s = solver(dlm_lib, inst)
    s.set_schedule(1e-2)
    s.set_options(precondition=True, topk=topk)
    # The momentum amplifies rounding geometrically on this instance (with
    # FP32 storage of the iterate, max |dlam| / max |lam| measured 2.2e-6
    # after 100 steps and 2.4e-5 after 200); here rows with four to seven
    # active edges are common, so topk = 8 takes most of them without the
    # threshold iteration.
    T = 200
    s.step(T)
    lam = s.lam().cpu().numpy().astype(np.float64)
    out = oracle.fista(oproblem(inst), T, 1e-2, precondition=True)
    ref = out["lam"]
    err = np.abs(lam - ref).max()
    print(f"appendix trajectory topk={topk}: max |dlam| / |lam| = {err / np.abs(ref).max():.3e}")
    assert err <= 1e-5 * np.abs(ref).max(), f"max err {err:.3e} (|lam| {np.abs(ref).max():.3f})"
    g = s.trajectory(0, T)
    assert np.abs(g - out["g_traj"]).max() <= 1e-5 * np.abs(out["g_traj"]).max()
    s.close()


def test_row_normalization_reaches_the_certified_gap(dlm_lib):
    # Rows of A several orders apart (App. A): with the per-item steps of the
    # row normalization the solve reaches 1e-4; the plain step 1/L, set by the
    # largest row, leaves the small rows' duals nearly still.
    inst = app_instance(20_000, 300, 31)
    p = oproblem(inst)
    s = solver(dlm_lib, inst)
    s.set_schedule(1e-2)
    s.set_options(precondition=True, gap_every=20, restart=True)
    st = s.solve(1e-4, 6000)
    assert st.status == dlm_lib.DLM_OK and st.rel_gap <= 1e-4
    lam = s.lam().cpu().numpy().astype(np.float64)
    cert = oracle.certify(p, lam, 1e-2)
    assert abs(st.dual_obj - cert["g"]) <= 2e-6 * abs(cert["g"])
    assert abs(st.primal_obj - cert["primal"]) <= 2e-6 * abs(cert["primal"])
    assert cert["rel_gap"] <= 1.5e-4
    s.close()
    plain = solver(dlm_lib, inst)
    plain.set_schedule(1e-2)
    plain.set_options(precondition=False, gap_every=20, restart=True)
    st0 = plain.solve(1e-4, int(st.iter))
    assert st0.rel_gap > 100 * max(st.rel_gap, 1e-6)
    plain.close()


@pytest.mark.parametrize("J", [12_000, 19_000])
def test_item_windows_of_the_certificate_sweep(dlm_lib, J):
    inst = app_instance(30_000, J, 41)
    s = solver(dlm_lib, inst)
    p = oproblem(inst)
    rng = np.random.default_rng(9)
    check_calculate(s, inst, p, priced_lambda(inst, rng, 1.0), 1e-2)
    s.set_schedule(1e-2)
    s.set_options(precondition=True)
    s.step(40)
    st = s.stats()
    lam = s.lam().cpu().numpy().astype(np.float64)
    ref = oracle.certify(p, lam, 1e-2)
    assert abs(st.dual_obj - ref["g"]) <= 2e-6 * abs(ref["g"])
    assert abs(st.primal_obj - ref["primal"]) <= 2e-6 * abs(ref["primal"])
    assert abs(st.max_viol - ref["max_viol"]) <= 1e-5 * (1 + abs(ref["max_viol"]))
    s.close()


def test_windowed_certificate_with_count_limit(dlm_lib):
    # the count sum is flushed by the first window only
    inst = app_instance(30_000, 12_000, 43)
    s = solver(dlm_lib, inst)
    M = 0.5 * inst.I
    s.set_count_limit(M)
    p = oproblem(inst)
    pc = oracle.Problem(p.row_ptr, p.col, p.c, p.a, p.b, p.J, p.kind, 1.0, M=M)
    rng = np.random.default_rng(2)
    lam32 = np.append(priced_lambda(inst, rng, 1.0), np.float32(0.05))
    g, grad, _ = s.calculate(torch.from_numpy(lam32).cuda(), 1e-2, want_x=False)
    ref = oracle.sweep(pc, lam32.astype(np.float64), 1e-2, want_x=False)
    # sum x over 30,000 users: FP32 x within 2e-6 z + 4 u x per edge, and up
    # to the threshold window on border users
    assert abs(grad.cpu().numpy()[-1] - ref["grad"][-1]) <= 2e-6 * inst.nnz * 1.0 + 1e-3
    assert abs(g - ref["g"]) <= 1e-5 * abs(ref["g"])
    s.close()


def test_item_limit(dlm_lib):
    # 12 bytes per item in every sweep block: 20,000 items exceed 227 KB
    J = 20_000
    rp = np.array([0, 2, 3], dtype=np.int64)
    col = np.array([0, J - 1, 5], dtype=np.int32)
    c = np.array([-1, -2, -1], dtype=np.float32)
    a = np.ones(3, dtype=np.float32)
    b = np.ones(J)
    with pytest.raises(dlm_lib.DlmError) as e:
        dlm_lib.Solver(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(), torch.from_numpy(c).cuda(),
                       torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), J)
    assert e.value.status == dlm_lib.DLM_ERR_UNSUPPORTED
    # just below the limit: created, and a step runs
    J = 19_000
    col = np.array([0, J - 1, 5], dtype=np.int32)
    s = dlm_lib.Solver(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(), torch.from_numpy(c).cuda(),
                       torch.from_numpy(a).cuda(), torch.from_numpy(np.ones(J)).cuda(), J)
    s.step(3)
    assert s.stats().status == dlm_lib.DLM_OK
    s.close()
