"""The short-row sweep (dlm_options.short_rows): iteration sweeps take a
kernel that holds each row of at most 32 edges in registers, sorts its values
and finds the threshold by the sort-based rule in one scan; wider rows take a
re-reading threshold iteration.  Iterates against the FP64 oracle (Sec. 3.2
primal recovery, the projected accelerated step) at the 1e-5 bound on lambda,
on instances with heavy degree tails (rows of 1 to 690 edges: every width
class and the wide path) and on App. A's requests (about ten edges, many
active), and bit-identity across runs and slice-to-CTA mappings."""
import numpy as np
import pytest

import oracle
import synth
from gpu_cases import mixed_instance, oracle_problem, tiny_instance, to_device

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def solver_for(dlm, inst, kind=oracle.SIMPLEX_LE, z=1.0, bf16=False):
    rp, col, c, a, b = to_device(inst, torch, bf16)
    return dlm.Solver(rp, col, c, a, b, inst.J, kind=kind, z=z, bf16=bf16)


def check_lam(s, ref, what):
    lam = s.lam().cpu().numpy().astype(np.float64)
    err = np.abs(lam - ref["lam"]).max()
    scale = max(np.abs(ref["lam"]).max(), 1e-6)
    print(f"{what}: max |dlam| / |lam| = {err / scale:.3e}")
    assert err <= 1e-5 * scale, f"{what}: max err {err:.3e} (|lam| {scale:.3f})"


def test_tiny_500_iterations(dlm_lib):
    # degrees 1 + Poisson(9): every width class up to 32
    inst = tiny_instance()
    s = solver_for(dlm_lib, inst)
    s.set_schedule(1e-2)
    s.set_options(short_rows=True)
    assert s.options().short_rows == 1
    s.step(500)
    check_lam(s, oracle.fista(oracle_problem(inst), 500, 1e-2, trajectory=False), "tiny, short rows")
    s.close()


@pytest.mark.parametrize("kind,z,bf16", [(oracle.SIMPLEX_LE, 1.0, False), (oracle.SIMPLEX_EQ, 0.7, False),
                                         (oracle.BOX, 0.6, False), (oracle.SIMPLEX_LE, 1.0, True)])
def test_continuation_trajectory(dlm_lib, kind, z, bf16):
    # heavy degree tail: rows of 1 .. 690 edges, every width class and the wide path
    inst = mixed_instance(seed=5, I=3000, J=300)
    s = solver_for(dlm_lib, inst, kind, z, bf16)
    s.set_schedule(1e-1, 1e-3, 0.5, 20)
    s.set_options(precondition=True, short_rows=True)
    T = 200
    s.step(T)
    ref = oracle.fista(oracle_problem(inst, kind, z, bf16), T, 1e-1, 1e-3, 0.5, 20, precondition=True)
    check_lam(s, ref, f"continuation kind={kind} bf16={bf16}")
    g = s.trajectory(0, T)
    rel = np.abs(g - ref["g_traj"]) / np.abs(ref["g_traj"])
    assert rel.max() <= 1e-5, f"g trajectory: max rel err {rel.max():.3e} at t = {rel.argmax()}"
    s.close()


def test_appendix_trajectory(dlm_lib):
    # App. A's requests: about ten edges each, most of them active near the
    # optimum, so nearly every row takes the short-row sweep's iteration
    inst = synth.generate_appendix(synth.AppRecipe(I=20_000, J=300, seed=31))
    s = solver_for(dlm_lib, inst)
    s.set_schedule(1e-2)
    s.set_options(precondition=True, short_rows=True)
    T = 200
    s.step(T)
    p = oracle.Problem(inst.row_ptr, inst.col, inst.c.astype(np.float64), inst.a.astype(np.float64), inst.b,
                       inst.J, oracle.SIMPLEX_LE, 1.0)
    ref = oracle.fista(p, T, 1e-2, precondition=True)
    check_lam(s, ref, "appendix, short rows")
    g = s.trajectory(0, T)
    assert np.abs(g - ref["g_traj"]).max() <= 1e-5 * np.abs(ref["g_traj"]).max()
    s.close()


def test_bit_identical_across_runs_and_mappings(dlm_lib):
    # each row's arithmetic involves no other row, and item sums are exact:
    # every mapping of the wider slices and every run give the same iterate
    inst = mixed_instance(seed=7, I=4000, J=500)
    out = []
    for mapping in (1, 2, 3, 3):
        s = solver_for(dlm_lib, inst)
        s.set_schedule(1e-1, 1e-3, 0.5, 25)
        s.set_options(mapping=mapping, short_rows=True, coop_max=1)
        s.step(120)
        lam, y, st = s.get_state()
        out.append((lam.cpu().numpy(), y.cpu().numpy(), s.trajectory(0, 120)))
        s.close()
    for lam, y, g in out[1:]:
        assert np.array_equal(lam.view(np.uint64), out[0][0].view(np.uint64))
        assert np.array_equal(y.view(np.uint64), out[0][1].view(np.uint64))
        assert np.array_equal(g.view(np.uint64), out[0][2].view(np.uint64))


def test_certified_solve_with_short_rows(dlm_lib):
    # the solve's certificate sweeps take the general kernel at the iterate
    # the short-row sweeps produced
    inst = synth.generate_appendix(synth.AppRecipe(I=20_000, J=300, seed=33))
    s = solver_for(dlm_lib, inst)
    s.set_schedule(1e-2)
    s.set_options(precondition=True, gap_every=20, restart=True, short_rows=True)
    st = s.solve(1e-4, 6000)
    assert st.status == dlm_lib.DLM_OK and st.rel_gap <= 1e-4
    p = oracle.Problem(inst.row_ptr, inst.col, inst.c.astype(np.float64), inst.a.astype(np.float64), inst.b,
                       inst.J, oracle.SIMPLEX_LE, 1.0)
    cert = oracle.certify(p, s.lam().cpu().numpy().astype(np.float64), 1e-2)
    assert abs(st.dual_obj - cert["g"]) <= 2e-6 * abs(cert["g"])
    assert cert["rel_gap"] <= 1.5e-4
    s.close()


def test_options_are_checked(dlm_lib):
    inst = tiny_instance()
    s = solver_for(dlm_lib, inst)
    o = s.options()
    o.short_rows = 2
    with pytest.raises(dlm_lib.DlmError) as e:
        dlm_lib.dlm_set_options(s.h, o)
    assert e.value.status == dlm_lib.DLM_ERR_INVALID_ARG
    s.close()
