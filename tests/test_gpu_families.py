"""Several capacity families (Def. 1, m = 2) on the GPU against the FP64
oracle: one dual evaluation, the accelerated trajectory, the certificate, and
the combinations the general sweep does not take.  Tolerances are those of
the one-family parity tests (FP32 per-edge arithmetic, exact fixed-point
sums), with the active-set allowance taken at |c| + sum_k |a_k lam_k|."""
import numpy as np
import pytest

import oracle
import synth
from gpu_cases import EPS32, mixed_instance, tiny_instance, x_error_report

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def second_family(inst, seed=21, scale=0.05):
    rng = np.random.default_rng(seed)
    a2 = rng.uniform(0.1, 2.0, size=inst.col.shape[0]).astype(np.float32)
    b2 = scale * np.bincount(inst.col, weights=a2.astype(np.float64), minlength=inst.J)
    return a2, b2


def make(dlm, inst, a2, b2, kind=oracle.SIMPLEX_LE, bf16=False):
    d = torch.device("cuda")
    A = np.stack([inst.a, a2], axis=1)
    if bf16:
        c = torch.from_numpy(synth.round_bf16(inst.c).view(np.int16)).to(d).view(torch.bfloat16)
        a = torch.from_numpy(synth.round_bf16(A.reshape(-1)).view(np.int16).reshape(A.shape)).to(d).view(
            torch.bfloat16)
    else:
        c = torch.from_numpy(inst.c).to(d)
        a = torch.from_numpy(np.ascontiguousarray(A)).to(d)
    b = torch.from_numpy(np.stack([inst.b, b2])).to(d)
    rp = torch.from_numpy(inst.row_ptr).to(d)
    col = torch.from_numpy(inst.col).to(d)
    return dlm.Solver(rp, col, c, a, b, inst.J, kind=kind, bf16=bf16)


def oproblem(inst, a2, b2, kind=oracle.SIMPLEX_LE, bf16=False):
    c, A = inst.c, np.stack([inst.a, a2], axis=1)
    if bf16:
        c = synth.bf16_to_f32(synth.round_bf16(c))
        A = synth.bf16_to_f32(synth.round_bf16(A.reshape(-1))).reshape(A.shape)
    return oracle.Problem(inst.row_ptr, inst.col, c.astype(np.float64), A.astype(np.float64),
                          np.stack([inst.b, b2]), inst.J, kind, 1.0)


@pytest.mark.parametrize("kind,bf16,gamma", [(oracle.SIMPLEX_LE, False, 1e-2), (oracle.SIMPLEX_LE, True, 1e-1),
                                             (oracle.BOX, False, 1e-2), (oracle.SIMPLEX_EQ, False, 1e-1)])
def test_calculate_with_two_families(dlm_lib, kind, bf16, gamma):
    inst = mixed_instance()
    a2, b2 = second_family(inst)
    s = make(dlm_lib, inst, a2, b2, kind, bf16)
    p = oproblem(inst, a2, b2, kind, bf16)
    J = inst.J
    rng = np.random.default_rng(8)
    for scale in (0.2, 1.0):
        lam32 = (rng.uniform(0, 1, 2 * J) * scale).astype(np.float32)
        g, grad, x = s.calculate(torch.from_numpy(lam32).cuda(), gamma)
        lam = lam32.astype(np.float64)
        ref = oracle.sweep(p, lam, gamma)
        A = p.a.reshape(-1, 2)
        # allowance at |c| + sum_k |a_k lam_k|: a one-family stand-in with that
        # magnitude in its c
        proxy = oracle.Problem(p.row_ptr, p.col, np.abs(p.c) + np.abs(A[:, 1] * lam[J:][p.col]), A[:, 0], p.b[:J],
                               J, kind, 1.0)
        dx, tol = x_error_report(x.cpu().numpy(), ref["x"], proxy, lam[:J], gamma)
        assert (dx <= tol).all(), f"{int((dx > tol).sum())} edges over tolerance, max {dx.max():.3e}"
        gg = grad.cpu().numpy().astype(np.float64)
        assert gg.shape == (2 * J,)
        for f in range(2):
            Ax = np.bincount(p.col, weights=A[:, f] * ref["x"], minlength=J)
            slack = np.bincount(p.col, weights=A[:, f] * tol, minlength=J)
            gt = 2e-6 * (Ax + p.b[f * J:(f + 1) * J]) + slack + 1e-6
            assert (np.abs(gg[f * J:(f + 1) * J] - ref["grad"][f * J:(f + 1) * J]) <= gt).all(), f
        assert abs(g - ref["g"]) <= 2e-6 * abs(ref["g"]) + float(np.abs(p.c) @ tol)
    s.close()


@pytest.mark.parametrize("precondition", [True, False])
def test_trajectory_with_two_families(dlm_lib, precondition):
    inst = tiny_instance()
    a2, b2 = second_family(inst, seed=5, scale=0.04)
    s = make(dlm_lib, inst, a2, b2)
    s.set_schedule(1e-2)
    s.set_options(precondition=precondition)
    # On this instance the momentum oscillates and amplifies rounding
    # geometrically; with FP32 storage of the iterate that reached 6e-5 after
    # 300 steps, with the FP64 iterate the FP32 per-edge arithmetic alone
    # measured 4.7e-8 relative after 150 steps.
    T = 300
    s.step(T)
    lam = s.lam().cpu().numpy().astype(np.float64)
    p = oproblem(inst, a2, b2)
    out = oracle.fista(p, T, 1e-2, precondition=precondition)
    ref = out["lam"]
    assert lam.shape == (2 * inst.J,)
    err = np.abs(lam - ref).max()
    print(f"two families precondition={precondition}: max |dlam| / |lam| = "
          f"{err / max(np.abs(ref).max(), 1e-6):.3e}")
    assert err <= 1e-5 * max(np.abs(ref).max(), 1e-6), f"max err {err:.3e}"
    g = s.trajectory(0, T)
    assert np.abs(g - out["g_traj"]).max() <= 1e-5 * np.abs(out["g_traj"]).max()
    assert ref[:inst.J].max() > 1e-3 and ref[inst.J:].max() > 1e-3  # both families bind somewhere
    s.close()


def test_solve_and_certificate_with_two_families(dlm_lib):
    inst = mixed_instance(seed=12, I=3000, J=300)
    a2, b2 = second_family(inst, seed=6, scale=0.03)
    s = make(dlm_lib, inst, a2, b2)
    s.set_schedule(1e-1, 1e-2, 0.5, 50)
    s.set_options(precondition=True, gap_every=20, restart=True)
    st = s.solve(1e-4, 20000)
    assert st.status == dlm_lib.DLM_OK and st.rel_gap <= 1e-4
    lam = s.lam().cpu().numpy().astype(np.float64)
    p = oproblem(inst, a2, b2)
    cert = oracle.certify(p, lam, 1e-2)
    assert abs(st.dual_obj - cert["g"]) <= 2e-6 * abs(cert["g"])
    assert abs(st.primal_obj - cert["primal"]) <= 2e-6 * abs(cert["primal"])
    assert cert["rel_gap"] <= 1.5e-4
    s.close()


def test_unsupported_combinations(dlm_lib):
    inst = tiny_instance()
    a2, b2 = second_family(inst)
    s = make(dlm_lib, inst, a2, b2)
    with pytest.raises(dlm_lib.DlmError) as e:
        s.set_count_limit(100.0)
    assert e.value.status == dlm_lib.DLM_ERR_UNSUPPORTED
    rp, col = torch.from_numpy(inst.row_ptr).cuda(), torch.from_numpy(inst.col).cuda()
    one = dlm_lib.Solver(rp, col, torch.from_numpy(inst.c).cuda(), torch.from_numpy(inst.a).cuda(),
                         torch.from_numpy(inst.b).cuda(), inst.J)
    with pytest.raises(dlm_lib.DlmError) as e:  # members with different numbers of families
        dlm_lib.Batch([one, s])
    assert e.value.status == dlm_lib.DLM_ERR_UNSUPPORTED
    one.close()
    s.close()


def test_batch_of_two_family_members_is_bit_identical(dlm_lib):
    insts = [tiny_instance(), mixed_instance(seed=9, I=2500, J=200)]
    fams = [second_family(insts[0], seed=5, scale=0.04), second_family(insts[1], seed=6, scale=0.03)]

    def members():
        out = []
        for inst, (a2, b2), pre in zip(insts, fams, (True, False)):
            s = make(dlm_lib, inst, a2, b2)
            s.set_schedule(1e-2)
            s.set_options(precondition=pre)
            out.append(s)
        return out

    alone = members()
    for s in alone:
        s.step(80)
    together = members()
    bt = dlm_lib.Batch(together)
    bt.step(80)
    for s0, s1 in zip(alone, together):
        assert torch.equal(s0.lam(), s1.lam())
    st = bt.stats()
    assert all(x.status == dlm_lib.DLM_OK for x in st)
    bt.close()
    for s in alone + together:
        s.close()


def test_duplicated_family_matches_one_family_x(dlm_lib):
    inst = tiny_instance()
    s2 = make(dlm_lib, inst, inst.a.copy(), inst.b.copy())
    rp, col = torch.from_numpy(inst.row_ptr).cuda(), torch.from_numpy(inst.col).cuda()
    s1 = dlm_lib.Solver(rp, col, torch.from_numpy(inst.c).cuda(), torch.from_numpy(inst.a).cuda(),
                        torch.from_numpy(inst.b).cuda(), inst.J)
    rng = np.random.default_rng(3)
    lam = rng.uniform(0, 1, inst.J).astype(np.float32)
    split = np.concatenate([0.25 * lam, 0.75 * lam]).astype(np.float32)  # the same A^T lam, up to rounding
    _, _, x1 = s1.calculate(torch.from_numpy(lam).cuda(), 1e-2)
    _, _, x2 = s2.calculate(torch.from_numpy(split).cuda(), 1e-2)
    # u differs by the rounding of a lam against a (lam / 4) + a (3 lam / 4):
    # x by at most 16 u (|c| + |a lam|) / gamma on every edge
    bound = 16 * EPS32 * (np.abs(inst.c) + np.abs(inst.a * lam[inst.col])) / 1e-2
    assert (np.abs(x1.cpu().numpy() - x2.cpu().numpy()) <= bound + 1e-7).all()
    s1.close()
    s2.close()
