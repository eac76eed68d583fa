"""FP64 CPU oracle for the ridge-regularized matching LP.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use it; the solver library never does.  It shares
no code with the CUDA path.  The arithmetic lives in ``oracle.c`` (plain C,
FP64, sequential); this module compiles it with gcc and marshals numpy arrays.

Parity status of each function (what pins it is in ``tests/test_oracle_*``):
  project    pinned: brute-force active-set enumeration, closed forms, KKT,
             two independent algorithms (sort and bisection), scipy QP.
  sweep/dual pinned: finite differences (Danskin), concavity, L-smoothness.
  families   (m capacity families, Def. 1) pinned: finite differences,
             KKT points by active-set enumeration with 2 rows per item, a
             slack second family and a duplicated family reducing to one.
  fista      pinned: exact KKT solutions by enumeration of active sets, the
             LP limit (scipy linprog), slack-capacity and one-item closed
             forms, the FISTA O(1/t^2) rate bound; with the adaptive
             restart, convergence to the same enumerated KKT solutions and a
             restart that fires on a hand-built overshoot.
  certify    pinned: weak duality, feasibility of the scaled point.
  The exact FP32-trajectory values on the large workloads are parity
  unpinned beyond oracle-vs-solver agreement (the paper prints no worked
  example).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

SIMPLEX_LE, SIMPLEX_EQ, BOX, BOX_CUT = 0, 1, 2, 3


class _Problem(ctypes.Structure):
    _fields_ = [
        ("I", ctypes.c_int64),
        ("J", ctypes.c_int64),
        ("nnz", ctypes.c_int64),
        ("row_ptr", ctypes.c_void_p),
        ("col", ctypes.c_void_p),
        ("c", ctypes.c_void_p),
        ("a", ctypes.c_void_p),
        ("b", ctypes.c_void_p),
        ("kind", ctypes.c_int32),
        ("_pad", ctypes.c_int32),
        ("z", ctypes.c_double),
        ("M", ctypes.c_double),
        ("m", ctypes.c_int32),
        ("_pad2", ctypes.c_int32),
        ("cut", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` (gcc -O2, no fast-math: IEEE FP64)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-shared", "-fPIC",
                                   "-pthread", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp, i64, i32, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        P = ctypes.POINTER(_Problem)
        lib.orc_project.argtypes = [vp, i64, i32, d, d, i32, vp]
        lib.orc_project.restype = d
        lib.orc_sweep.argtypes = [P, vp, d, vp, vp, vp, vp, vp, vp]
        lib.orc_sweep.restype = d
        lib.orc_dual.argtypes = [P, vp, d, vp, vp]
        lib.orc_dual.restype = d
        lib.orc_row_sq.argtypes = [P, vp]
        lib.orc_row_sum.argtypes = [P, vp]
        lib.orc_row_sum.restype = None
        lib.orc_certify.argtypes = [P, vp, d, vp]
        lib.orc_fista.argtypes = [P, d, d, d, i64, i32, i32, i64, vp, vp, vp, vp, vp, vp]
        lib.orc_stage_gamma.argtypes = [d, d, d, i64]
        lib.orc_fista_threads.argtypes = [P, d, i32, i64, i32, vp]
        lib.orc_fista_threads.restype = None
        lib.orc_solve_threads.argtypes = [P, d, d, d, i64, i32, i32, d, i64, i64, i32, vp, vp, vp]
        lib.orc_solve_threads.restype = None
        lib.orc_stage_gamma.restype = d
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class Problem:
    """An instance in FP64: user-major CSR (row_ptr int64, col int32), c, a
    (float64, e.g. float32 or bfloat16 values widened exactly), b (float64).
    With m capacity families (Def. 1) a has shape [nnz, m] and b [m, J]; the
    dual vector is then lam[k * J + j] (m J entries, plus mu with a count
    constraint M).  kind BOX_CUT: each user's x lies in [0, z] with
    sum_j x_ij <= cut."""

    def __init__(self, row_ptr, col, c, a, b, J=None, kind=SIMPLEX_LE, z=1.0, M=np.inf, cut=np.inf):
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.c = np.ascontiguousarray(c, dtype=np.float64)
        a = np.asarray(a, dtype=np.float64)
        b = np.asarray(b, dtype=np.float64)
        self.m = int(a.shape[1]) if a.ndim == 2 else 1
        self.a = np.ascontiguousarray(a.reshape(-1))
        self.b = np.ascontiguousarray(b.reshape(-1))
        self.I = int(self.row_ptr.shape[0] - 1)
        self.J = int(J if J is not None else self.b.shape[0] // self.m)
        if self.b.shape[0] != self.m * self.J or self.a.shape[0] != self.m * int(self.row_ptr[-1]):
            raise ValueError("a must be [nnz] or [nnz, m] and b [J] or [m, J]")
        self.nnz = int(self.row_ptr[-1])
        self.kind = int(kind)
        self.z = float(z)
        self.M = float(M)
        self.cut = float(cut)
        if self.kind == BOX_CUT and not (self.cut > 0 and np.isfinite(self.cut)):
            raise ValueError("BOX_CUT needs a finite cut > 0")
        self.D = self.m * self.J + (1 if np.isfinite(self.M) else 0)  # dual dimension
        s = _Problem()
        s.I, s.J, s.nnz = self.I, self.J, self.nnz
        s.row_ptr, s.col, s.c, s.a, s.b = (_p(self.row_ptr), _p(self.col), _p(self.c), _p(self.a), _p(self.b))
        s.kind, s.z, s.M, s.m = self.kind, self.z, self.M, self.m
        s.cut = self.cut if self.kind == BOX_CUT else 0.0
        self._s = s

    @classmethod
    def from_instance(cls, inst, kind=SIMPLEX_LE, z=1.0, c=None, a=None):
        return cls(inst.row_ptr, inst.col, inst.c if c is None else c, inst.a if a is None else a, inst.b,
                   inst.J, kind, z)


def project(v, kind=SIMPLEX_LE, z=1.0, method=0, cut=np.inf):
    """Projection of one segment onto the simplex / box / box cut by the
    budget sum x <= cut; returns (x, theta)."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    x = np.empty_like(v)
    th = _load().orc_project(_p(v), v.shape[0], kind, z, float(cut) if kind == BOX_CUT else 0.0, method, _p(x))
    return x, th


def _dual_vec(p: Problem, lam):
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    if lam.shape[0] != p.D:
        raise ValueError(f"dual vector needs {p.D} entries (num_items + 1 with a count constraint)")
    return lam


def sweep(p: Problem, lam, gamma, want_x=True):
    """One dual evaluation: dict(g, x, Ax, Cx, Qx, obj, count, grad); lam has
    p.D entries (the last is the count dual mu when p.M is finite), and so
    does grad."""
    lam = _dual_vec(p, lam)
    x = np.empty(p.nnz) if want_x else None
    Ax, Cx, Qx = np.empty(p.m * p.J), np.empty(p.J), np.empty(p.J)
    obj, count = ctypes.c_double(), ctypes.c_double()
    g = _load().orc_sweep(ctypes.byref(p._s), _p(lam), gamma, _p(x), _p(Ax), _p(Cx), _p(Qx), ctypes.byref(obj),
                          ctypes.byref(count))
    grad = Ax - p.b
    if p.D > p.m * p.J:
        grad = np.append(grad, count.value - p.M)
    return dict(g=g, x=x, Ax=Ax, Cx=Cx, Qx=Qx, obj=obj.value, count=count.value, grad=grad)


def dual(p: Problem, lam, gamma):
    """(g(lam), grad g(lam), x*(lam)); lam and grad have p.D entries."""
    lam = _dual_vec(p, lam)
    grad = np.empty(p.D)
    x = np.empty(p.nnz)
    g = _load().orc_dual(ctypes.byref(p._s), _p(lam), gamma, _p(grad), _p(x))
    return g, grad, x


def row_sq(p: Problem):
    out = np.empty(p.m * p.J)
    _load().orc_row_sq(ctypes.byref(p._s), _p(out))
    return out


def row_sum(p: Problem):
    out = np.empty(p.m * p.J)
    _load().orc_row_sum(ctypes.byref(p._s), _p(out))
    return out


def certify(p: Problem, lam, gamma):
    """dict(g, primal, rel_gap, max_viol, uncert_gap, primal_unscaled)."""
    lam = _dual_vec(p, lam)
    out = np.empty(6)
    _load().orc_certify(ctypes.byref(p._s), _p(lam), gamma, _p(out))
    return dict(g=out[0], primal=out[1], rel_gap=out[2], max_viol=out[3], uncert_gap=out[4],
                primal_unscaled=out[5])


def fista(p: Problem, T, gamma0, gamma_end=None, factor=0.5, iters_per_stage=0, precondition=False, lam0=None,
          trajectory=True, restart=False):
    """T iterations of accelerated projected dual ascent; dict(lam, y, theta,
    g_traj, gamma_traj).  restart=True adds the adaptive momentum restart."""
    gamma_end = gamma0 if gamma_end is None else gamma_end
    lam0 = np.zeros(p.D) if lam0 is None else _dual_vec(p, lam0)
    lam, y = np.empty(p.D), np.empty(p.D)
    th = ctypes.c_double()
    gt = np.empty(T) if trajectory else None
    gg = np.empty(T) if trajectory else None
    _load().orc_fista(ctypes.byref(p._s), gamma0, gamma_end, factor, iters_per_stage, int(bool(precondition)),
                      int(bool(restart)), T, _p(lam0), _p(lam), _p(y), ctypes.byref(th), _p(gt), _p(gg))
    return dict(lam=lam, y=y, theta=th.value, g_traj=gt, gamma_traj=gg)


def fista_threads(p: Problem, T, gamma, precondition=False, nthreads=1):
    """Timing only: T fixed-gamma iterations with the sweep split over
    nthreads threads (per-thread item sums added in thread order); returns lam."""
    if p.D != p.J:
        raise ValueError("the threaded timing loop covers the one-family capacity problem")
    lam = np.empty(p.J)
    _load().orc_fista_threads(ctypes.byref(p._s), gamma, int(bool(precondition)), T, int(nthreads), _p(lam))
    return lam


def solve_threads(p: Problem, gamma0, gamma_end=None, factor=0.5, iters_per_stage=0, precondition=False,
                  restart=False, target=1e-4, gap_every=25, max_iters=100_000, nthreads=1, lam0=None):
    """fista's iteration driven to a certified gap (checked every gap_every
    iterations once gamma is at gamma_end), with the sweep split over
    nthreads threads; dict(lam, iters, rel_gap, g, primal).  One capacity
    family, no count constraint."""
    if p.D != p.J or p.m != 1:
        raise ValueError("the threaded solve covers the one-family capacity problem")
    gamma_end = gamma0 if gamma_end is None else gamma_end
    lam0 = np.zeros(p.J) if lam0 is None else _dual_vec(p, lam0)
    lam, st = np.empty(p.J), np.empty(4)
    _load().orc_solve_threads(ctypes.byref(p._s), gamma0, gamma_end, factor, iters_per_stage,
                              int(bool(precondition)), int(bool(restart)), target, gap_every, max_iters,
                              int(nthreads), _p(lam0), _p(lam), _p(st))
    return dict(lam=lam, iters=int(st[0]), rel_gap=st[1], g=st[2], primal=st[3])


def stage_gamma(gamma0, gamma_end, factor, s):
    return _load().orc_stage_gamma(gamma0, gamma_end, factor, s)
