"""Seeded instances and helpers shared by the GPU parity tests (no solver
arithmetic here: instances come from ``synth``, references from ``oracle``)."""
import numpy as np

import oracle
import synth

EPS32 = 2.0 ** -24


def with_empty_users(inst, k, seed=0):
    """Insert k users with no eligible items at seeded positions."""
    rng = np.random.default_rng(seed)
    deg = np.diff(inst.row_ptr)
    pos = np.sort(rng.integers(0, len(deg) + 1, size=k))
    deg2 = np.insert(deg, pos, 0)
    rp = np.zeros(len(deg2) + 1, dtype=np.int64)
    np.cumsum(deg2, out=rp[1:])
    return synth.Instance(rp, inst.col, inst.c, inst.a, inst.b, inst.J, None, inst.recipe)


def mixed_instance(seed=3, I=4000, J=700, bf16=False):
    """Production generators with a heavy degree tail so that every degree
    class (1 .. 513+) and every lane mapping is exercised, plus empty users."""
    r = synth.recipe_production(I=I, J=J, seed=seed)
    r.deg_sigma, r.deg_max = 1.4, 690
    inst = with_empty_users(synth.generate(r), 25, seed)
    if bf16:
        inst.c = synth.bf16_to_f32(synth.round_bf16(inst.c))
        inst.a = synth.bf16_to_f32(synth.round_bf16(inst.a))
    return inst


def tiny_instance():
    return synth.generate(synth.recipe_tiny())


def to_device(inst, torch, bf16=False):
    d = torch.device("cuda")
    rp = torch.from_numpy(inst.row_ptr).to(d)
    col = torch.from_numpy(inst.col).to(d)
    if bf16:
        c = torch.from_numpy(synth.round_bf16(inst.c).view(np.int16)).to(d).view(torch.bfloat16)
        a = torch.from_numpy(synth.round_bf16(inst.a).view(np.int16)).to(d).view(torch.bfloat16)
    else:
        c = torch.from_numpy(inst.c).to(d)
        a = torch.from_numpy(inst.a).to(d)
    b = torch.from_numpy(inst.b).to(d)
    return rp, col, c, a, b


def oracle_problem(inst, kind=oracle.SIMPLEX_LE, z=1.0, bf16=False):
    c, a = inst.c, inst.a
    if bf16:
        c = synth.bf16_to_f32(synth.round_bf16(c))
        a = synth.bf16_to_f32(synth.round_bf16(a))
    return oracle.Problem(inst.row_ptr, inst.col, c.astype(np.float64), a.astype(np.float64), inst.b, inst.J,
                          kind, z)


def x_error_report(x_gpu, x_ref, p, lam, gamma, cap=None):
    """Max |dx| over the bulk of edges and over users with an edge within
    FP32 resolution of the threshold (where the active set itself is only
    decided to FP32 precision).  With ``cap`` (the box bound of a budgeted
    box, whose threshold also depends on which edges sit at the cap) edges
    within that resolution of the cap count as border edges too.  Returns
    (bulk_max, bound_violations)."""
    dx = np.abs(x_gpu.astype(np.float64) - x_ref)
    M = np.abs(p.c) + np.abs(p.a * lam[p.col])
    window = 16 * EPS32 * M / gamma  # how far FP32 rounding of u moves x
    user = np.repeat(np.arange(p.I), np.diff(p.row_ptr))
    border_edge = (x_ref < window) & ((x_ref > 0) | (x_gpu > 0))
    if cap is not None:
        border_edge |= np.abs(x_ref - cap) < window
    border_user = np.zeros(p.I, dtype=bool)
    border_user[user[border_edge]] = True
    bw = np.zeros(p.I)
    np.maximum.at(bw, user, window)
    tol = 2e-6 * p.z + 4 * EPS32 * x_ref + np.where(border_user[user], bw[user], 0.0)
    return dx, tol
