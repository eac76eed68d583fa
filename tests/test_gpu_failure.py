"""Failure detection without a GPU fault: a corrupted checkpoint (a NaN in
the momentum point y, restored through dlm_set_state) is caught by the
update kernel's finiteness check, recorded in the handle's status word and
reported by the next status read as DLM_ERR_NUMERIC; dlm_solve stops with
that status.  The context stays usable."""
import numpy as np
import pytest

import oracle
from gpu_cases import mixed_instance, oracle_problem, to_device

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_corrupted_state_is_reported_and_context_survives(dlm_lib):
    inst = mixed_instance(seed=21, I=4000, J=300)
    arrs = to_device(inst, torch)
    s = dlm_lib.Solver(*arrs, inst.J)
    s.set_schedule(1e-2)
    s.step(5)
    lam, y, st = s.get_state()
    assert s.stats().status == dlm_lib.DLM_OK
    y[7] = float("nan")
    s.set_state(lam, y, st)
    s.step(1)
    assert s.stats().status == dlm_lib.DLM_ERR_NUMERIC
    out = dlm_lib.dlm_solve(s.h, 1e-9, 10)
    assert out.status == dlm_lib.DLM_ERR_NUMERIC and not out.converged
    s.close()
    # a fresh handle on the same device still computes correct results
    s2 = dlm_lib.Solver(*arrs, inst.J)
    s2.set_schedule(1e-2)
    s2.step(30)
    lam2 = s2.lam().cpu().numpy().astype(np.float64)
    ref = oracle.fista(oracle_problem(inst), 30, 1e-2, trajectory=False)["lam"]
    assert np.abs(lam2 - ref).max() <= 1e-5 * max(np.abs(ref).max(), 1e-6)
    assert s2.stats().status == dlm_lib.DLM_OK
    s2.close()
