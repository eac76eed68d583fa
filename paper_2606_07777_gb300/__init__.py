"""GB300 dual-sweep solver for ridge-regularized matching LPs.

Thin Python binding of the C-ABI in ``include/dlm.h`` (library
``libdlm.so``, hand-written sm_103a CUDA kernels).  This module only marshals
arguments: every step of the iteration runs in the library's kernels.  There
is no CPU path; if the library cannot be built or loaded, ``load()`` raises.

PyTorch is used for device memory and streams: pass CUDA tensors (device
memspace) or CPU tensors / numpy arrays (host memspace).
"""
from __future__ import annotations

import ctypes
import os

from . import _build

__all__ = [
    "load", "build", "DlmError", "Solver", "dlm_create", "dlm_set_schedule", "dlm_set_options", "dlm_set_lambda",
    "dlm_calculate", "dlm_step", "dlm_solve", "dlm_get_stats", "dlm_get_lambda", "dlm_get_x", "dlm_get_state",
    "dlm_set_state", "dlm_get_info", "dlm_step_timed", "dlm_calculate_static", "dlm_destroy", "dlm_last_error",
    "dlm_get_options", "dlm_autotune", "dlm_get_trajectory", "dlm_release_cached_memory", "Batch", "dlm_batch_create", "dlm_batch_set_options", "dlm_batch_autotune",
    "dlm_batch_step", "dlm_batch_step_timed", "dlm_batch_get_stats", "dlm_batch_solve", "dlm_batch_destroy",
    "WarmStart", "WS_FEATURES",
]

WS_FEATURES = 7

DLM_OK, DLM_ERR_INVALID_ARG, DLM_ERR_OOM, DLM_ERR_CUDA, DLM_ERR_NUMERIC, DLM_ERR_TIMEOUT, DLM_ERR_UNSUPPORTED = range(7)
DLM_F32, DLM_BF16 = 0, 1
DLM_SIMPLEX_LE, DLM_SIMPLEX_EQ, DLM_BOX, DLM_BOX_CUT = 0, 1, 2, 3
DLM_MEM_DEVICE, DLM_MEM_HOST = 0, 1

_STATUS = {0: "DLM_OK", 1: "DLM_ERR_INVALID_ARG", 2: "DLM_ERR_OOM", 3: "DLM_ERR_CUDA", 4: "DLM_ERR_NUMERIC",
           5: "DLM_ERR_TIMEOUT", 6: "DLM_ERR_UNSUPPORTED"}


class DlmError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__(f"{where}: {_STATUS.get(status, status)}: {msg}")
        self.status = status


class ProblemDesc(ctypes.Structure):
    _fields_ = [("num_users", ctypes.c_int64), ("num_items", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("item_idx", ctypes.c_void_p), ("c", ctypes.c_void_p),
                ("a", ctypes.c_void_p), ("b", ctypes.c_void_p), ("val_dtype", ctypes.c_int32),
                ("kind", ctypes.c_int32), ("z", ctypes.c_double), ("memspace", ctypes.c_int32),
                ("num_families", ctypes.c_int32), ("cut", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("gap_every", ctypes.c_int32), ("precondition", ctypes.c_int32), ("mapping", ctypes.c_int32),
                ("graph_iters", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("coop_max", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("restart", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}

    def __repr__(self):
        return f"Options({self.as_dict()})"


class Stats(ctypes.Structure):
    _fields_ = [("iter", ctypes.c_int64), ("gamma", ctypes.c_double), ("dual_obj", ctypes.c_double),
                ("primal_obj", ctypes.c_double), ("rel_gap", ctypes.c_double), ("uncert_gap", ctypes.c_double),
                ("max_viol", ctypes.c_double), ("seconds", ctypes.c_double), ("status", ctypes.c_int32),
                ("converged", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class State(ctypes.Structure):
    _fields_ = [("iter", ctypes.c_int64), ("theta", ctypes.c_double), ("stage", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


_lib = None

# (name, argtypes) of every exported call, in header order.
_vp, _i64, _i32, _d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
_SIGS = {
    "dlm_create": [ctypes.POINTER(ProblemDesc), _vp, ctypes.POINTER(_vp)],
    "dlm_set_schedule": [_vp, _d, _d, _d, _i64],
    "dlm_set_options": [_vp, ctypes.POINTER(Options)],
    "dlm_set_lambda": [_vp, _vp, _i32],
    "dlm_calculate": [_vp, _vp, _d, ctypes.POINTER(_d), _vp, _vp],
    "dlm_step": [_vp, _i64],
    "dlm_solve": [_vp, _d, _i64, ctypes.POINTER(Stats)],
    "dlm_get_stats": [_vp, ctypes.POINTER(Stats)],
    "dlm_get_lambda": [_vp, _vp, _i32],
    "dlm_get_x": [_vp, _vp, _i32],
    "dlm_get_state": [_vp, _vp, _vp, ctypes.POINTER(State), _i32],
    "dlm_set_state": [_vp, _vp, _vp, ctypes.POINTER(State), _i32],
    "dlm_get_trajectory": [_vp, _i64, _i64, _vp],
    "dlm_release_cached_memory": [],
    "dlm_get_info": [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64)],
    "dlm_step_timed": [_vp, _i64, ctypes.POINTER(_d), ctypes.POINTER(_d), ctypes.POINTER(_d)],
    "dlm_calculate_static": [_i64, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _i32, _d, _vp, _d, _vp, _vp, _vp, _vp],
    "dlm_get_options": [_vp, ctypes.POINTER(Options)],
    "dlm_autotune": [_vp, _i32, ctypes.POINTER(Options), ctypes.POINTER(_d)],
    "dlm_batch_create": [ctypes.POINTER(_vp), _i32, _vp, ctypes.POINTER(_vp)],
    "dlm_batch_set_options": [_vp, ctypes.POINTER(Options)],
    "dlm_batch_autotune": [_vp, _i32, ctypes.POINTER(Options), ctypes.POINTER(_d)],
    "dlm_batch_step": [_vp, _i64],
    "dlm_batch_step_timed": [_vp, _i64, ctypes.POINTER(_d), ctypes.POINTER(_d), ctypes.POINTER(_d)],
    "dlm_batch_get_stats": [_vp, ctypes.POINTER(Stats)],
    "dlm_batch_solve": [_vp, _d, _i64, ctypes.POINTER(Stats)],
    "dlm_set_count_limit": [_vp, _d],
    "dlm_ws_create": [_i32, ctypes.c_uint64, _vp, ctypes.POINTER(_vp)],
    "dlm_ws_num_params": [_vp, ctypes.POINTER(_i64)],
    "dlm_ws_get_params": [_vp, _vp, _vp, _vp],
    "dlm_ws_set_params": [_vp, _vp, _vp, _vp],
    "dlm_ws_features": [_vp, _vp, _d, _vp],
    "dlm_ws_fit_normalizer": [_vp, _vp, _i64],
    "dlm_ws_loss_grad": [_vp, _vp, _vp, _i64, ctypes.POINTER(_d), _vp],
    "dlm_ws_train": [_vp, _vp, _vp, _i64, _i32, ctypes.c_float, _vp],
    "dlm_ws_predict": [_vp, _vp, _i64, _vp],
}
_VOID = {"dlm_destroy": [_vp], "dlm_batch_destroy": [_vp], "dlm_ws_destroy": [_vp]}
EXPORTS = list(_SIGS) + list(_VOID) + ["dlm_last_error"]


def build(force: bool = False) -> str:
    return _build.build(force=force)


def library_path() -> str:
    return _build.LIB


def load():
    """Load ``libdlm.so`` (building it first if it is missing or stale).
    Raises if it cannot be built or loaded: there is no fallback."""
    global _lib
    if _lib is None:
        if not _build.up_to_date():
            _build.build()
        lib = ctypes.CDLL(_build.LIB)
        for name, args in _SIGS.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        for name, args in _VOID.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = None
        lib.dlm_last_error.argtypes = []
        lib.dlm_last_error.restype = ctypes.c_char_p
        _lib = lib
    return _lib


def dlm_last_error() -> str:
    return load().dlm_last_error().decode()


def _call(name, *args):
    lib = load()
    st = getattr(lib, name)(*args)
    if st != DLM_OK:
        raise DlmError(st, name, lib.dlm_last_error().decode())
    return st


def _ptr(x):
    """Address of a torch tensor, numpy array or None."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    return int(x)


def dlm_create(desc: ProblemDesc, stream=None):
    h = ctypes.c_void_p()
    _call("dlm_create", ctypes.byref(desc), stream, ctypes.byref(h))
    return h


def dlm_set_schedule(h, gamma0, gamma_end, factor, iters_per_stage):
    _call("dlm_set_schedule", h, gamma0, gamma_end, factor, iters_per_stage)


def dlm_set_options(h, opt: Options):
    _call("dlm_set_options", h, ctypes.byref(opt))


def dlm_get_options(h) -> Options:
    o = Options()
    _call("dlm_get_options", h, ctypes.byref(o))
    return o


def dlm_autotune(h, iters=3):
    """(chosen Options, mean sweep ms of the winner)."""
    o, ms = Options(), ctypes.c_double()
    _call("dlm_autotune", h, iters, ctypes.byref(o), ctypes.byref(ms))
    return o, ms.value


def dlm_set_lambda(h, lam, memspace):
    _call("dlm_set_lambda", h, _ptr(lam), memspace)


def dlm_calculate(h, lam, gamma, grad=None, x=None) -> float:
    g = ctypes.c_double()
    _call("dlm_calculate", h, _ptr(lam), gamma, ctypes.byref(g), _ptr(grad), _ptr(x))
    return g.value


def dlm_step(h, n):
    _call("dlm_step", h, n)


def dlm_solve(h, target, max_iters) -> Stats:
    """Returns the final Stats; a run that stops on the iteration limit or on a
    device-reported status returns normally with that status in `.status`."""
    s = Stats()
    lib = load()
    st = lib.dlm_solve(h, target, max_iters, ctypes.byref(s))
    if st not in (DLM_OK, DLM_ERR_TIMEOUT, DLM_ERR_NUMERIC):
        raise DlmError(st, "dlm_solve", lib.dlm_last_error().decode())
    if st != DLM_OK and s.status == DLM_OK:
        s.status = st
    return s


def dlm_get_stats(h) -> Stats:
    s = Stats()
    _call("dlm_get_stats", h, ctypes.byref(s))
    return s


def dlm_get_lambda(h, out, memspace):
    _call("dlm_get_lambda", h, _ptr(out), memspace)


def dlm_get_x(h, out, memspace):
    _call("dlm_get_x", h, _ptr(out), memspace)


def dlm_get_state(h, lam, y, memspace) -> State:
    s = State()
    _call("dlm_get_state", h, _ptr(lam), _ptr(y), ctypes.byref(s), memspace)
    return s


def dlm_set_state(h, lam, y, state: State, memspace):
    _call("dlm_set_state", h, _ptr(lam), _ptr(y), ctypes.byref(state), memspace)


def dlm_get_trajectory(h, first_iter, n):
    """g(y_t) for t = first_iter .. first_iter + n - 1 (numpy float64)."""
    import numpy as np

    out = np.empty(max(int(n), 0), dtype=np.float64)
    _call("dlm_get_trajectory", h, int(first_iter), int(n), _ptr(out) if n > 0 else None)
    return out


def dlm_release_cached_memory():
    """Return the device memory the library's pools keep after handles are destroyed."""
    _call("dlm_release_cached_memory")


def dlm_get_info(h):
    v = [ctypes.c_int64() for _ in range(4)]
    _call("dlm_get_info", h, *[ctypes.byref(x) for x in v])
    return dict(num_users=v[0].value, num_items=v[1].value, nnz=v[2].value, bytes_per_iter=v[3].value)


def dlm_step_timed(h, n):
    """(sweep_ms, update_ms, total_ms) summed over n individually launched iterations."""
    v = [ctypes.c_double() for _ in range(3)]
    _call("dlm_step_timed", h, n, *[ctypes.byref(x) for x in v])
    return tuple(x.value for x in v)


def dlm_calculate_static(num_users, num_items, nnz, row_ptr, item_idx, c, a, b, kind, z, lam, gamma, g, grad=None,
                         x=None, stream=None):
    """Allocation-free dual evaluation (device arrays; g is a device double)."""
    _call("dlm_calculate_static", num_users, num_items, nnz, _ptr(row_ptr), _ptr(item_idx), _ptr(c), _ptr(a),
          _ptr(b), kind, z, _ptr(lam), gamma, _ptr(g), _ptr(grad), _ptr(x), stream)


def dlm_destroy(h):
    if h:
        load().dlm_destroy(h)


def dlm_batch_create(handles, stream=None):
    arr = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    bt = ctypes.c_void_p()
    _call("dlm_batch_create", arr, len(handles), stream, ctypes.byref(bt))
    return bt


def dlm_batch_set_options(bt, opt: Options):
    _call("dlm_batch_set_options", bt, ctypes.byref(opt))


def dlm_batch_autotune(bt, iters=3):
    o, ms = Options(), ctypes.c_double()
    _call("dlm_batch_autotune", bt, iters, ctypes.byref(o), ctypes.byref(ms))
    return o, ms.value


def dlm_batch_step(bt, n):
    _call("dlm_batch_step", bt, n)


def dlm_batch_step_timed(bt, n):
    v = [ctypes.c_double() for _ in range(3)]
    _call("dlm_batch_step_timed", bt, n, *[ctypes.byref(x) for x in v])
    return tuple(x.value for x in v)


def dlm_batch_get_stats(bt, n):
    out = (Stats * n)()
    _call("dlm_batch_get_stats", bt, out)
    return list(out)


def dlm_batch_solve(bt, n, target, max_iters):
    """(status, [Stats] per member); the iteration limit and device-reported
    statuses return normally."""
    out = (Stats * n)()
    lib = load()
    st = lib.dlm_batch_solve(bt, target, max_iters, out)
    if st not in (DLM_OK, DLM_ERR_TIMEOUT, DLM_ERR_NUMERIC):
        raise DlmError(st, "dlm_batch_solve", lib.dlm_last_error().decode())
    return st, list(out)


def dlm_batch_destroy(bt):
    if bt:
        load().dlm_batch_destroy(bt)


def _options(gap_every=0, precondition=False, mapping=0, graph_iters=0, ctas_per_sm=0, coop_max=0, block_threads=0,
             restart=False):
    o = Options()
    o.gap_every, o.precondition, o.mapping = gap_every, int(bool(precondition)), mapping
    o.graph_iters, o.ctas_per_sm, o.coop_max, o.block_threads = graph_iters, ctas_per_sm, coop_max, block_threads
    o.restart = int(bool(restart))
    return o


class Solver:
    """One matching-LP instance on the GPU.

    Arrays may be CUDA tensors (device memspace) or CPU tensors / numpy
    arrays (host memspace; copied in by ``dlm_create``).  ``c``/``a`` are
    float32, or bfloat16 (torch.bfloat16 tensors or uint16 bit patterns with
    ``bf16=True``)."""

    def __init__(self, row_ptr, col, c, a, b, num_items=None, kind=DLM_SIMPLEX_LE, z=1.0, bf16=None, stream=None,
                 cut=None):
        import torch

        self._torch = torch
        dev = getattr(row_ptr, "is_cuda", False)
        if bf16 is None:
            bf16 = getattr(c, "dtype", None) in (torch.bfloat16,) or str(getattr(c, "dtype", "")) == "uint16"
        # several capacity families: a is [nnz, m] (edge-major), b [m, num_items]
        self.num_families = int(a.shape[1]) if len(a.shape) == 2 else 1
        self.num_items = int(num_items if num_items is not None else b.shape[-1])
        self.num_users = int(row_ptr.shape[0] - 1)
        self.nnz = int(col.shape[0])
        self.bf16 = bool(bf16)
        desc = ProblemDesc()
        desc.num_families = self.num_families
        desc.num_users, desc.num_items, desc.nnz = self.num_users, self.num_items, self.nnz
        desc.row_ptr, desc.item_idx, desc.c, desc.a, desc.b = (_ptr(row_ptr), _ptr(col), _ptr(c), _ptr(a), _ptr(b))
        desc.val_dtype = DLM_BF16 if self.bf16 else DLM_F32
        desc.kind, desc.z = int(kind), float(z)
        desc.cut = float(cut) if cut is not None else 0.0  # DLM_BOX_CUT: per-user budget
        desc.memspace = DLM_MEM_DEVICE if dev else DLM_MEM_HOST
        self.device = torch.device("cuda", torch.cuda.current_device())
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        self._keep = (row_ptr, col, c, a, b)
        self.h = dlm_create(desc, ctypes.c_void_p(stream.cuda_stream))
        self._keep = None
        self.kind = int(kind)
        self.z = float(z)
        # m num_items (family-major), + 1 while a count constraint is set
        self.dual_dim = self.num_families * self.num_items

    def close(self):
        if getattr(self, "h", None):
            dlm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_schedule(self, gamma0, gamma_end=None, factor=0.5, iters_per_stage=1 << 30):
        dlm_set_schedule(self.h, gamma0, gamma0 if gamma_end is None else gamma_end, factor, iters_per_stage)

    def set_options(self, gap_every=0, precondition=False, mapping=0, graph_iters=0, ctas_per_sm=0, coop_max=0,
                    block_threads=0, restart=False):
        dlm_set_options(self.h, _options(gap_every, precondition, mapping, graph_iters, ctas_per_sm, coop_max,
                                         block_threads, restart))

    def options(self) -> Options:
        return dlm_get_options(self.h)

    def autotune(self, iters=3):
        """Tries the sweep mappings from the current state (which it keeps);
        returns (chosen Options, mean sweep ms)."""
        return dlm_autotune(self.h, iters)

    def set_count_limit(self, M):
        """Global count constraint sum x <= M (math.inf removes it); the dual
        vectors then carry its dual as one more entry."""
        import math

        _call("dlm_set_count_limit", self.h, float(M))
        self.dual_dim = self.num_families * self.num_items + (0 if math.isinf(M) else 1)

    def set_lambda(self, lam):
        dlm_set_lambda(self.h, lam, DLM_MEM_DEVICE if getattr(lam, "is_cuda", False) else DLM_MEM_HOST)

    def step(self, n):
        dlm_step(self.h, n)

    def step_timed(self, n):
        return dlm_step_timed(self.h, n)

    def solve(self, target_rel_gap, max_iters) -> Stats:
        return dlm_solve(self.h, target_rel_gap, max_iters)

    def stats(self) -> Stats:
        return dlm_get_stats(self.h)

    def calculate(self, lam, gamma, want_grad=True, want_x=True):
        t = self._torch
        grad = t.empty(self.dual_dim, dtype=t.float32, device=self.device) if want_grad else None
        x = t.empty(self.nnz, dtype=t.float32, device=self.device) if want_x else None
        g = dlm_calculate(self.h, lam, gamma, grad, x)
        return g, grad, x

    def lam(self):
        t = self._torch
        out = t.empty(self.dual_dim, dtype=t.float32, device=self.device)
        dlm_get_lambda(self.h, out, DLM_MEM_DEVICE)
        return out

    def x(self):
        t = self._torch
        out = t.empty(self.nnz, dtype=t.float32, device=self.device)
        dlm_get_x(self.h, out, DLM_MEM_DEVICE)
        return out

    def get_state(self):
        """(lam, y, State): the FP64 iterate and momentum point (CUDA float64)."""
        t = self._torch
        lam = t.empty(self.dual_dim, dtype=t.float64, device=self.device)
        y = t.empty_like(lam)
        s = dlm_get_state(self.h, lam, y, DLM_MEM_DEVICE)
        return lam, y, s

    def set_state(self, lam, y, s):
        dlm_set_state(self.h, lam, y, s, DLM_MEM_DEVICE)

    def info(self):
        return dlm_get_info(self.h)

    def trajectory(self, first_iter, n):
        """Dual objective g(y_t) of iterations first_iter .. first_iter + n - 1."""
        return dlm_get_trajectory(self.h, first_iter, n)


class Batch:
    """Several Solver instances iterated together: one sweep launch and one
    update launch per iteration for all of them.  Set each member's schedule,
    options and warm start first; close the batch before its members."""

    def __init__(self, solvers, stream=None):
        import torch

        self.members = list(solvers)
        if stream is None:
            stream = torch.cuda.current_stream(self.members[0].device)
        self.stream = stream
        self.bt = dlm_batch_create([m.h for m in self.members], ctypes.c_void_p(stream.cuda_stream))

    def close(self):
        if getattr(self, "bt", None):
            dlm_batch_destroy(self.bt)
            self.bt = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_options(self, gap_every=0, mapping=0, graph_iters=0, ctas_per_sm=0, coop_max=0, block_threads=0):
        dlm_batch_set_options(self.bt, _options(gap_every, False, mapping, graph_iters, ctas_per_sm, coop_max,
                                                block_threads))

    def autotune(self, iters=3):
        return dlm_batch_autotune(self.bt, iters)

    def step(self, n):
        dlm_batch_step(self.bt, n)

    def step_timed(self, n):
        return dlm_batch_step_timed(self.bt, n)

    def stats(self):
        return dlm_batch_get_stats(self.bt, len(self.members))

    def solve(self, target_rel_gap, max_iters):
        return dlm_batch_solve(self.bt, len(self.members), target_rel_gap, max_iters)


class WarmStart:
    """The learned warm start (a three-layer perceptron on per-item
    features, trained and evaluated by the library's tensor-core kernels).
    Arrays are CUDA tensors; parameters come back as numpy float32."""

    def __init__(self, width=128, seed=0, stream=None):
        import torch

        self._torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device())
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        self.width = int(width)
        h = ctypes.c_void_p()
        _call("dlm_ws_create", self.width, seed, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        self.h = h
        n = ctypes.c_int64()
        _call("dlm_ws_num_params", self.h, ctypes.byref(n))
        self.num_params = n.value

    def close(self):
        if getattr(self, "h", None):
            load().dlm_ws_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def features(solver, lam_prev, gamma):
        """Feature rows [num_items, 7] (CUDA float32) of a Solver's instance."""
        t = solver._torch
        X = t.empty((solver.num_items, WS_FEATURES), dtype=t.float32, device=solver.device)
        _call("dlm_ws_features", solver.h, _ptr(lam_prev), float(gamma), _ptr(X))
        return X

    def params(self):
        import numpy as np

        th = np.empty(self.num_params, dtype=np.float32)
        mu = np.empty(WS_FEATURES, dtype=np.float32)
        sd = np.empty(WS_FEATURES, dtype=np.float32)
        _call("dlm_ws_get_params", self.h, _ptr(th), _ptr(mu), _ptr(sd))
        return th, mu, sd

    def set_params(self, theta=None, mu=None, sd=None):
        import numpy as np

        f = lambda v: None if v is None else np.ascontiguousarray(v, dtype=np.float32)
        th, m, s = f(theta), f(mu), f(sd)
        _call("dlm_ws_set_params", self.h, _ptr(th), _ptr(m), _ptr(s))

    def fit_normalizer(self, X):
        _call("dlm_ws_fit_normalizer", self.h, _ptr(X), int(X.shape[0]))

    def loss_grad(self, X, y):
        import numpy as np

        loss = ctypes.c_double()
        g = np.empty(self.num_params, dtype=np.float32)
        _call("dlm_ws_loss_grad", self.h, _ptr(X), _ptr(y), int(X.shape[0]), ctypes.byref(loss), _ptr(g))
        return loss.value, g

    def train(self, X, y, steps, lr):
        import numpy as np

        losses = np.empty(max(int(steps), 1), dtype=np.float32)
        _call("dlm_ws_train", self.h, _ptr(X), _ptr(y), int(X.shape[0]), int(steps), float(lr), _ptr(losses))
        return losses[:steps]

    def predict(self, X):
        t = self._torch
        out = t.empty(X.shape[0], dtype=t.float32, device=X.device)
        _call("dlm_ws_predict", self.h, _ptr(X), int(X.shape[0]), _ptr(out))
        return out

    def unpack(self, theta):
        """Split a flat parameter vector into the named tensors (numpy)."""
        F, H = WS_FEATURES, self.width
        o = 0
        out = {}
        for name, shape in (("W1", (F, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", (1,))):
            n = 1
            for d in shape:
                n *= d
            out[name] = theta[o:o + n].reshape(shape)
            o += n
        return out

    def pack(self, P):
        import numpy as np

        return np.concatenate([np.asarray(P[k], dtype=np.float32).ravel() for k in ("W1", "b1", "W2", "b2", "w3",
                                                                                   "b3")])
