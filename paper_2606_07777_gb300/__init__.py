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
    "WarmStart", "WS_FEATURES", "ShardedSolver", "shard_local", "shard_combine", "shard_item_sums",
    "allreduce_shard_stats", "partition_users",
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
                ("num_families", ctypes.c_int32), ("cut", ctypes.c_double), ("shard", ctypes.c_void_p)]


class Shard(ctypes.Structure):
    """dlm_shard: statistics of a user-sharded instance and its exchange buffers."""
    _fields_ = [("nnz", ctypes.c_int64), ("active_users", ctypes.c_int64), ("max_item_degree", ctypes.c_int64),
                ("max_abs_a", ctypes.c_double), ("max_abs_c", ctypes.c_double), ("a_nonneg", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("item_sq", ctypes.c_void_p), ("item_sum", ctypes.c_void_p),
                ("exchange", ctypes.c_void_p), ("cert_exchange", ctypes.c_void_p), ("cert_obj", ctypes.c_void_p)]


class Options(ctypes.Structure):
    _fields_ = [("gap_every", ctypes.c_int32), ("precondition", ctypes.c_int32), ("mapping", ctypes.c_int32),
                ("graph_iters", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("coop_max", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("restart", ctypes.c_int32), ("topk", ctypes.c_int32),
                ("short_rows", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1)]

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
    "dlm_get_setup_seconds": [_vp, _vp, _i32],
    "dlm_shard_local": [ctypes.POINTER(ProblemDesc), _vp, ctypes.POINTER(Shard), _vp],
    "dlm_shard_item_sums": [ctypes.POINTER(ProblemDesc), ctypes.POINTER(Shard), _vp, _vp, _vp],
    "dlm_shard_sweep": [_vp],
    "dlm_shard_update": [_vp],
    "dlm_shard_cert_sweep": [_vp],
    "dlm_shard_cert_finish": [_vp, ctypes.POINTER(Stats)],
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
             restart=False, topk=0, short_rows=False):
    o = Options()
    o.gap_every, o.precondition, o.mapping = gap_every, int(bool(precondition)), mapping
    o.graph_iters, o.ctas_per_sm, o.coop_max, o.block_threads = graph_iters, ctas_per_sm, coop_max, block_threads
    o.restart = int(bool(restart))
    o.topk = int(topk)
    o.short_rows = int(bool(short_rows))
    return o


def _desc(row_ptr, col, c, a, b, num_items=None, kind=DLM_SIMPLEX_LE, z=1.0, bf16=None, cut=None):
    """A ProblemDesc for the arrays (CUDA tensors: device memspace; CPU
    tensors / numpy arrays: host memspace); returns (desc, bf16)."""
    import torch

    dev = getattr(row_ptr, "is_cuda", False)
    if bf16 is None:
        bf16 = getattr(c, "dtype", None) in (torch.bfloat16,) or str(getattr(c, "dtype", "")) == "uint16"
    desc = ProblemDesc()
    # several capacity families: a is [nnz, m] (edge-major), b [m, num_items]
    desc.num_families = int(a.shape[1]) if len(a.shape) == 2 else 1
    desc.num_items = int(num_items if num_items is not None else b.shape[-1])
    desc.num_users = int(row_ptr.shape[0] - 1)
    desc.nnz = int(col.shape[0])
    desc.row_ptr, desc.item_idx, desc.c, desc.a, desc.b = (_ptr(row_ptr), _ptr(col), _ptr(c), _ptr(a), _ptr(b))
    desc.val_dtype = DLM_BF16 if bf16 else DLM_F32
    desc.kind, desc.z = int(kind), float(z)
    desc.cut = float(cut) if cut is not None else 0.0  # DLM_BOX_CUT: per-user budget
    desc.memspace = DLM_MEM_DEVICE if dev else DLM_MEM_HOST
    desc.shard = None
    return desc, bool(bf16)


class Solver:
    """One matching-LP instance on the GPU.

    Arrays may be CUDA tensors (device memspace) or CPU tensors / numpy
    arrays (host memspace; copied in by ``dlm_create``).  ``c``/``a`` are
    float32, or bfloat16 (torch.bfloat16 tensors or uint16 bit patterns with
    ``bf16=True``)."""

    def __init__(self, row_ptr, col, c, a, b, num_items=None, kind=DLM_SIMPLEX_LE, z=1.0, bf16=None, stream=None,
                 cut=None, shard=None):
        import torch

        self._torch = torch
        desc, self.bf16 = _desc(row_ptr, col, c, a, b, num_items, kind, z, bf16, cut)
        self.num_families = desc.num_families
        self.num_items, self.num_users, self.nnz = desc.num_items, desc.num_users, desc.nnz
        if shard is not None:
            desc.shard = ctypes.addressof(shard)
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
                    block_threads=0, restart=False, topk=0, short_rows=False):
        dlm_set_options(self.h, _options(gap_every, precondition, mapping, graph_iters, ctas_per_sm, coop_max,
                                         block_threads, restart, topk, short_rows))

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

    def setup_seconds(self):
        """dlm_create's wall time by phase (dict)."""
        import numpy as np

        v = np.zeros(6)
        _call("dlm_get_setup_seconds", self.h, _ptr(v), 6)
        return dict(zip(("host_to_device", "validate", "degree_sort", "layout_and_item_sums", "handle_and_tables",
                         "total"), v.tolist()))

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

    def set_options(self, gap_every=0, mapping=0, graph_iters=0, ctas_per_sm=0, coop_max=0, block_threads=0, topk=0):
        dlm_batch_set_options(self.bt, _options(gap_every, False, mapping, graph_iters, ctas_per_sm, coop_max,
                                                block_threads, False, topk))

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


# ---------------------------------------------------------------------------
# User-sharded instances (include/dlm.h, "User-sharded instances")
# ---------------------------------------------------------------------------

def partition_users(row_ptr, nparts):
    """Contiguous user ranges [u0, u1) of about equal edge counts, one per part."""
    import numpy as np

    rp = np.asarray(row_ptr)
    nnz = int(rp[-1])
    cuts = [0]
    for k in range(1, nparts):
        cuts.append(int(np.searchsorted(rp, nnz * k // nparts, side="left")))
    cuts.append(len(rp) - 1)
    return [(cuts[k], max(cuts[k], cuts[k + 1])) for k in range(nparts)]


def shard_local(row_ptr, col, c, a, b, num_items=None, kind=DLM_SIMPLEX_LE, z=1.0, bf16=None, cut=None,
                stream=None):
    """This rank's statistics: (dict(nnz, active_users, max_abs_a, max_abs_c,
    a_nonneg), item degrees as int64 numpy [num_items])."""
    import numpy as np

    desc, _ = _desc(row_ptr, col, c, a, b, num_items, kind, z, bf16, cut)
    loc = Shard()
    deg = np.empty(desc.num_items, dtype=np.int64)
    _call("dlm_shard_local", ctypes.byref(desc), stream, ctypes.byref(loc), _ptr(deg))
    return dict(nnz=loc.nnz, active_users=loc.active_users, max_abs_a=loc.max_abs_a, max_abs_c=loc.max_abs_c,
                a_nonneg=loc.a_nonneg), deg


def shard_combine(locals_, degrees):
    """The whole instance's statistics from every rank's (the sums, maxima and
    minimum of the protocol)."""
    import numpy as np

    deg = np.sum(np.stack(degrees), axis=0)
    return dict(nnz=int(sum(x["nnz"] for x in locals_)), active_users=int(sum(x["active_users"] for x in locals_)),
                max_abs_a=float(max(x["max_abs_a"] for x in locals_)),
                max_abs_c=float(max(x["max_abs_c"] for x in locals_)),
                a_nonneg=int(min(x["a_nonneg"] for x in locals_)), max_item_degree=int(deg.max()) if deg.size else 0)


def allreduce_shard_stats(local, degree, group=None, device=None):
    """shard_combine over the ranks of a torch.distributed process group
    (int64 sums of the counts and degrees, maxima of the bounds, minimum of
    the sign flag): every rank gets the same combined statistics."""
    import numpy as np
    import torch
    import torch.distributed as dist

    dev = device if device is not None else torch.device("cpu")
    counts = torch.tensor([local["nnz"], local["active_users"]], dtype=torch.int64, device=dev)
    deg = torch.from_numpy(np.ascontiguousarray(degree, dtype=np.int64)).to(dev)
    bounds = torch.tensor([local["max_abs_a"], local["max_abs_c"], -float(local["a_nonneg"])], dtype=torch.float64,
                          device=dev)
    dist.all_reduce(counts, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(deg, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(bounds, op=dist.ReduceOp.MAX, group=group)
    c, d, bd = counts.cpu().numpy(), deg.cpu().numpy(), bounds.cpu().numpy()
    return dict(nnz=int(c[0]), active_users=int(c[1]), max_abs_a=float(bd[0]), max_abs_c=float(bd[1]),
                a_nonneg=int(-bd[2]), max_item_degree=int(d.max()) if d.size else 0)


def _shard_struct(g, item_sq=None, item_sum=None):
    sh = Shard()
    sh.nnz, sh.active_users, sh.max_item_degree = g["nnz"], g["active_users"], g["max_item_degree"]
    sh.max_abs_a, sh.max_abs_c, sh.a_nonneg = g["max_abs_a"], g["max_abs_c"], g["a_nonneg"]
    sh.item_sq, sh.item_sum = _ptr(item_sq), _ptr(item_sum)
    return sh


def shard_item_sums(row_ptr, col, c, a, b, global_stats, num_items=None, kind=DLM_SIMPLEX_LE, z=1.0, bf16=None,
                    cut=None, stream=None):
    """This rank's fixed-point item sums (sum a^2, sum a) at the exponents the
    combined statistics fix: two int64 numpy arrays [num_items]."""
    import numpy as np

    desc, _ = _desc(row_ptr, col, c, a, b, num_items, kind, z, bf16, cut)
    sq = np.empty(desc.num_items, dtype=np.int64)
    s1 = np.empty(desc.num_items, dtype=np.int64)
    g = _shard_struct(global_stats)
    _call("dlm_shard_item_sums", ctypes.byref(desc), ctypes.byref(g), stream, _ptr(sq), _ptr(s1))
    return sq, s1


class ShardedSolver(Solver):
    """One rank's shard (a contiguous range of users, with the full capacity
    vector b) of a user-sharded instance.  `global_stats`, `item_sq`,
    `item_sum` are the combined statistics and item sums (shard_combine /
    allreduce_shard_stats, then the summed shard_item_sums).  Each iteration
    is sweep(), the ranks' sum of `exchange`, update(); `reduce(tensor)` adds
    a tensor over the ranks in place (torch.distributed.all_reduce when a
    process group is given)."""

    def __init__(self, row_ptr, col, c, a, b, num_items, global_stats, item_sq, item_sum, kind=DLM_SIMPLEX_LE, z=1.0,
                 bf16=None, stream=None, cut=None, reduce=None):
        import numpy as np
        import torch

        J = int(num_items)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.exchange = torch.zeros(J + 2, dtype=torch.int64, device=dev)
        self.cert_exchange = torch.zeros(3 * J + 1, dtype=torch.int64, device=dev)
        self.cert_obj = torch.zeros(1, dtype=torch.float64, device=dev)
        self._sq = np.ascontiguousarray(item_sq, dtype=np.int64)
        self._s1 = np.ascontiguousarray(item_sum, dtype=np.int64)
        self._shard = _shard_struct(global_stats, self._sq, self._s1)
        self._shard.exchange = self.exchange.data_ptr()
        self._shard.cert_exchange = self.cert_exchange.data_ptr()
        self._shard.cert_obj = self.cert_obj.data_ptr()
        self.reduce = reduce
        self._gamma_end = 1e-2  # the handle's initial fixed ridge
        super().__init__(row_ptr, col, c, a, b, J, kind=kind, z=z, bf16=bf16, stream=stream, cut=cut,
                         shard=self._shard)
        # every row's threshold in its own lane: the result of a row then does
        # not depend on which users share its slice on this rank
        self.set_options(coop_max=1)

    @classmethod
    def distributed(cls, row_ptr, col, c, a, b, num_items, group=None, **kw):
        """The whole set-up over a torch.distributed process group (NCCL with
        CUDA tensors, or any backend for the host-side statistics)."""
        import numpy as np
        import torch
        import torch.distributed as dist

        backend = dist.get_backend(group)
        dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
        opts = {k: kw[k] for k in ("kind", "z", "bf16", "cut") if k in kw}
        loc, deg = shard_local(row_ptr, col, c, a, b, num_items, **opts)
        g = allreduce_shard_stats(loc, deg, group, dev)
        sq, s1 = shard_item_sums(row_ptr, col, c, a, b, g, num_items, **opts)
        t = torch.from_numpy(np.stack([sq, s1])).to(dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        sums = t.cpu().numpy()

        def reduce(x):
            dist.all_reduce(x, op=dist.ReduceOp.SUM, group=group)

        return cls(row_ptr, col, c, a, b, num_items, g, sums[0], sums[1], reduce=reduce, **kw)

    def sweep(self):
        _call("dlm_shard_sweep", self.h)

    def update(self):
        _call("dlm_shard_update", self.h)

    def step(self, n):
        for _ in range(int(n)):
            self.sweep()
            self.reduce(self.exchange)
            self.update()

    def cert_sweep(self):
        _call("dlm_shard_cert_sweep", self.h)

    def cert_finish(self) -> Stats:
        st = Stats()
        _call("dlm_shard_cert_finish", self.h, ctypes.byref(st))
        return st

    def stats(self) -> Stats:
        self.cert_sweep()
        self.reduce(self.cert_exchange)
        self.reduce(self.cert_obj)
        return self.cert_finish()

    def solve(self, target_rel_gap, max_iters, gap_every=50) -> Stats:
        """dlm_solve's loop over the ranks: the certified gap every gap_every
        iterations once gamma is at its final value."""
        import time

        t0 = time.perf_counter()
        done = 0
        while True:
            st = self.stats()
            if st.status != DLM_OK:
                break
            if st.gamma == self._gamma_end and st.rel_gap <= target_rel_gap:
                st.converged = 1
                break
            if done >= max_iters:
                break
            n = min(gap_every, max_iters - done)
            self.step(n)
            done += n
        st.seconds = time.perf_counter() - t0
        return st

    def set_schedule(self, gamma0, gamma_end=None, factor=0.5, iters_per_stage=1 << 30):
        self._gamma_end = gamma0 if gamma_end is None else gamma_end
        super().set_schedule(gamma0, gamma_end, factor, iters_per_stage)
