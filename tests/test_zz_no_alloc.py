"""The allocation-free dual evaluation, dlm_calculate_static, for callers
that cannot allocate device memory (a process whose device memory belongs to
another framework's allocator, or a fixed memory budget): it must give the
same g, grad and x as the handle-based dlm_calculate, through the C-ABI, on
two calls in a row (the second call reuses the library's fixed scratch array
that the first one left behind)."""
import numpy as np
import pytest

import oracle
from gpu_cases import mixed_instance, oracle_problem, to_device, x_error_report

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("kind,z", [(oracle.SIMPLEX_LE, 1.0), (oracle.SIMPLEX_LE, 0.7), (oracle.SIMPLEX_EQ, 0.7),
                                    (oracle.BOX, 0.6)])
def test_static_entry_point_matches_handle_on_two_calls(dlm_lib, kind, z):
    inst = mixed_instance(seed=31, I=5000, J=600)
    rp, col, c, a, b = to_device(inst, torch)
    s = dlm_lib.Solver(rp, col, c, a, b, inst.J, kind=kind, z=z)
    p = oracle_problem(inst, kind, z)
    rng = np.random.default_rng(5)
    g_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    for gamma in (1e-2, 1e-3):
        lam32 = rng.uniform(0, 1.5, inst.J).astype(np.float32)
        lam32[rng.uniform(size=inst.J) < 0.2] = 0.0
        lam = torch.from_numpy(lam32).cuda()
        g_ref, grad_ref, x_ref = s.calculate(lam, gamma)
        grad = torch.empty(inst.J, dtype=torch.float32, device="cuda")
        x = torch.empty(inst.nnz, dtype=torch.float32, device="cuda")
        dlm_lib.dlm_calculate_static(inst.I, inst.J, inst.nnz, rp, col, c, a, b, kind, z, lam, gamma, g_dev, grad, x,
                                     None)
        torch.cuda.synchronize()
        lam64 = lam32.astype(np.float64)
        # x: the parity tolerance against the oracle; against the handle's x,
        # twice that (both sides carry their own rounding)
        ref = oracle.sweep(p, lam64, gamma)
        dx, tol = x_error_report(x.cpu().numpy(), ref["x"], p, lam64, gamma)
        assert (dx <= tol).all(), dx.max()
        dxh = np.abs(x.cpu().numpy().astype(np.float64) - x_ref.cpu().numpy())
        assert (dxh <= 2 * tol).all(), dxh.max()
        # grad and g: the tolerances of the single-sweep parity test
        scale_j = np.bincount(p.col, weights=p.a * ref["x"], minlength=p.J) + np.abs(p.b)
        allow = np.bincount(p.col, weights=p.a * np.maximum(tol - 2e-6, 0), minlength=p.J)
        dg = np.abs(grad.cpu().numpy().astype(np.float64) - grad_ref.cpu().numpy())
        assert (dg <= 2 * (2e-6 * scale_j + allow + 1e-6)).all(), dg.max()
        g = g_dev.item()
        assert abs(g - g_ref) <= 2 * 2e-6 * (abs(g_ref) + abs(ref["obj"])), (g, g_ref)
    s.close()


@pytest.mark.parametrize("bad", [-1, 600])
def test_static_entry_point_flags_an_out_of_range_item(dlm_lib, bad):
    # an item index outside [0, num_items) is not read through: the call
    # succeeds and reports g and grad as NaN; a following valid call is clean
    inst = mixed_instance(seed=32, I=800, J=600)
    rp, col, c, a, b = to_device(inst, torch)
    col_bad = col.clone()
    col_bad[17] = bad
    g_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    grad = torch.empty(inst.J, dtype=torch.float32, device="cuda")
    lam = torch.full((inst.J,), 0.2, dtype=torch.float32, device="cuda")
    dlm_lib.dlm_calculate_static(inst.I, inst.J, inst.nnz, rp, col_bad, c, a, b, oracle.SIMPLEX_LE, 1.0, lam, 1e-2,
                                 g_dev, grad, None, None)
    torch.cuda.synchronize()
    assert np.isnan(g_dev.item()) and torch.isnan(grad).all().item()
    dlm_lib.dlm_calculate_static(inst.I, inst.J, inst.nnz, rp, col, c, a, b, oracle.SIMPLEX_LE, 1.0, lam, 1e-2,
                                 g_dev, grad, None, None)
    torch.cuda.synchronize()
    ref = oracle.sweep(oracle_problem(inst), lam.cpu().numpy().astype(np.float64), 1e-2, want_x=False)
    assert abs(g_dev.item() - ref["g"]) <= 2e-6 * (abs(ref["g"]) + abs(ref["obj"]))


def test_static_entry_point_rejects_too_many_items(dlm_lib):
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(dlm_lib.DlmError) as e:
        dlm_lib.dlm_calculate_static(1, 70000, 0, torch.zeros(2, dtype=torch.int64, device="cuda"), None, None, None,
                                     torch.zeros(70000, dtype=torch.float64, device="cuda"), 0, 1.0,
                                     torch.zeros(70000, device="cuda"), 1e-2, z)
    assert e.value.status == dlm_lib.DLM_ERR_UNSUPPORTED and "65536" in str(e.value)
