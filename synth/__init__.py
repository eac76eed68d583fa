"""Seeded synthetic matching-LP instances (shared by the solver's tests, the
benchmark and the oracle's tests; holds none of the solver's arithmetic).

The generator itself is plain C (``synth.c``), compiled here with gcc and
loaded through ctypes.  Every random value is a pure function of
``(seed, user id, purpose, draw)`` under Philox4x32-10, so rows can be
regenerated one user at a time and results do not depend on thread count.

Workload recipes (users x items, degree model, item popularity, values,
capacities) mirror the synthetic matching workloads the paper evaluates on
(Sec. 3.3; App. A): sparse user-major CSR with an int64 row pointer, int32
item index and float32 ``c`` (cost, <= 0) and ``a`` (capacity usage, > 0),
plus float64 capacities ``b``.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

DEG_POISSON, DEG_LOGNORMAL = 0, 1
ITEMS_UNIFORM, ITEMS_ZIPF = 0, 1
C_NEG_UNIFORM, C_NEG_LOGNORMAL = 0, 1
A_ONE, A_UNIFORM = 0, 1
B_ITEM_DEGREE, B_SUM_A = 0, 1


class _Params(ctypes.Structure):
    _fields_ = [
        ("I", ctypes.c_int64),
        ("J", ctypes.c_int32),
        ("_pad0", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("deg_model", ctypes.c_int32),
        ("deg_max", ctypes.c_int32),
        ("deg_mean", ctypes.c_double),
        ("deg_sigma", ctypes.c_double),
        ("item_model", ctypes.c_int32),
        ("c_model", ctypes.c_int32),
        ("zipf_s", ctypes.c_double),
        ("c_mu", ctypes.c_double),
        ("c_sigma", ctypes.c_double),
        ("a_model", ctypes.c_int32),
        ("b_model", ctypes.c_int32),
        ("a_lo", ctypes.c_double),
        ("a_hi", ctypes.c_double),
        ("b_frac", ctypes.c_double),
    ]


class _AppParams(ctypes.Structure):
    _fields_ = [
        ("I", ctypes.c_int64),
        ("J", ctypes.c_int32),
        ("_pad0", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("nu", ctypes.c_double),
        ("breadth_sigma", ctypes.c_double),
        ("v_sigma", ctypes.c_double),
        ("u_sigma", ctypes.c_double),
        ("eps_sigma", ctypes.c_double),
        ("c_max", ctypes.c_double),
        ("s_mu", ctypes.c_double),
        ("s_sigma", ctypes.c_double),
        ("rho_lo", ctypes.c_double),
        ("rho_hi", ctypes.c_double),
        ("b_eps", ctypes.c_double),
    ]


@dataclasses.dataclass
class Recipe:
    """One synthetic instance family (all fields are generator inputs)."""

    I: int
    J: int
    seed: int
    deg_model: int = DEG_LOGNORMAL
    deg_mean: float = 25.0
    deg_sigma: float = 1.0
    deg_max: int = 500
    item_model: int = ITEMS_ZIPF
    zipf_s: float = 0.8
    c_model: int = C_NEG_LOGNORMAL
    c_mu: float = 0.0
    c_sigma: float = 0.5
    a_model: int = A_UNIFORM
    a_lo: float = 0.5
    a_hi: float = 1.5
    b_model: int = B_SUM_A
    b_frac: float = 0.05

    def _c(self) -> _Params:
        p = _Params()
        for f in dataclasses.fields(self):
            setattr(p, f.name, getattr(self, f.name))
        return p


def build(force: bool = False) -> str:
    """Compile ``libsynth.so`` next to the source (gcc, OpenMP)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(
                ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
            )
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        vp = ctypes.c_void_p
        lib.synth_philox4x32_10.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
        lib.synth_degrees.argtypes = [P(_Params), vp, ctypes.c_int64, vp, ctypes.c_int]
        lib.synth_fill.argtypes = [P(_Params), vp, ctypes.c_int64, vp, vp, vp, vp, ctypes.c_int]
        lib.synth_capacity.argtypes = [P(_Params), ctypes.c_int64, vp, vp, vp, vp, ctypes.c_int]
        lib.synth_round_bf16.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_int]
        lib.synth_next_day_ids.argtypes = [ctypes.c_uint64, ctypes.c_int64, vp, ctypes.c_double,
                                           ctypes.c_int64, vp, ctypes.c_int]
        lib.synth_next_day_fill.argtypes = [P(_Params), ctypes.c_uint64, ctypes.c_int64, vp, vp, vp, vp, vp,
                                            vp, vp, vp, vp, vp, ctypes.c_double, ctypes.c_double, ctypes.c_int]
        lib.synth_scale_capacity.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_double, vp]
        lib.synth_uniforms.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, vp]
        lib.synth_poisson.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double,
                                      ctypes.c_int64, vp]
        AP = P(_AppParams)
        lib.synth_app_counts.argtypes = [AP, vp]
        lib.synth_app_pick.argtypes = [AP, vp, vp, ctypes.c_int]
        lib.synth_app_transpose.argtypes = [ctypes.c_int64, ctypes.c_int32, vp, vp, vp, vp, ctypes.c_int]
        lib.synth_app_values.argtypes = [AP, ctypes.c_int64, vp, vp, vp, vp, ctypes.c_int]
        lib.synth_app_capacity.argtypes = [AP, ctypes.c_int64, vp, vp, vp, vp, vp, ctypes.c_int]
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr, key):
    """Philox4x32-10 block function (for known-answer tests)."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib.synth_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def _np_empty(n, dtype):
    return np.empty(int(n), dtype=dtype)


@dataclasses.dataclass
class Instance:
    """User-major CSR matching instance (host arrays)."""

    row_ptr: np.ndarray  # int64 [I+1]
    col: np.ndarray  # int32 [nnz]
    c: np.ndarray  # float32 [nnz]
    a: np.ndarray  # float32 [nnz]
    b: np.ndarray  # float64 [J]
    J: int
    ids: np.ndarray | None = None  # user ids used to seed each row (None = 0..I-1)
    recipe: Recipe | None = None

    @property
    def I(self) -> int:  # noqa: E743
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


def generate(r: Recipe, ids: np.ndarray | None = None, nthreads: int = 0, alloc=_np_empty,
             capacity: bool = True) -> Instance:
    """Generate the rows of users ``ids`` (default 0..I-1) and, optionally,
    capacities ``b`` from those rows.  ``alloc(n, dtype)`` supplies output
    buffers (e.g. pinned host memory)."""
    lib = _load()
    p = r._c()
    n = r.I if ids is None else int(len(ids))
    if ids is not None:
        ids = np.ascontiguousarray(ids, dtype=np.int64)
    deg = np.empty(n, dtype=np.int32)
    lib.synth_degrees(ctypes.byref(p), _ptr(ids), n, _ptr(deg), nthreads)
    row_ptr = alloc(n + 1, np.int64)
    row_ptr[0] = 0
    np.cumsum(deg, dtype=np.int64, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    col = alloc(nnz, np.int32)
    c = alloc(nnz, np.float32)
    a = alloc(nnz, np.float32)
    lib.synth_fill(ctypes.byref(p), _ptr(ids), n, _ptr(row_ptr), _ptr(col), _ptr(c), _ptr(a), nthreads)
    b = np.zeros(r.J, dtype=np.float64)
    if capacity:
        lib.synth_capacity(ctypes.byref(p), n, _ptr(row_ptr), _ptr(col), _ptr(a), _ptr(b), nthreads)
    return Instance(row_ptr, col, c, a, b, r.J, ids, r)


def round_bf16(x: np.ndarray, nthreads: int = 0, out: np.ndarray | None = None) -> np.ndarray:
    """float32 -> bfloat16 bit patterns (uint16), round to nearest even."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    if out is None:
        out = np.empty(x.shape, dtype=np.uint16)
    _load().synth_round_bf16(_ptr(x), _ptr(out), x.size, nthreads)
    return out


def bf16_to_f32(bits: np.ndarray) -> np.ndarray:
    """bfloat16 bit patterns -> float32 (exact)."""
    return (bits.astype(np.uint32) << 16).view(np.float32)


def uniforms(seed: int, uid: int, purpose: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _load().synth_uniforms(seed, uid, purpose, n, _ptr(out))
    return out


def poisson(seed: int, uid: int, purpose: int, mu: float, n: int) -> np.ndarray:
    """n Poisson(mu) draws of the sampler the appendix generator uses."""
    out = np.empty(n, dtype=np.int64)
    _load().synth_poisson(seed, uid, purpose, mu, n, _ptr(out))
    return out


def sample_users(I: int, frac: float, seed: int) -> np.ndarray:
    """Seeded sorted sample of user ids (each kept with probability frac)."""
    u = np.empty(I, dtype=np.float64)
    # one counter-based uniform per user id, stream purpose 77
    lib = _load()
    lib.synth_uniforms(seed, 0, 77, I, _ptr(u))
    return np.nonzero(u < frac)[0].astype(np.int64)


def subset(inst: Instance, users: np.ndarray) -> Instance:
    """Rows ``users`` of ``inst`` as a new CSR (capacities copied)."""
    users = np.asarray(users, dtype=np.int64)
    lens = inst.row_ptr[users + 1] - inst.row_ptr[users]
    rp = np.zeros(len(users) + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    # edge positions of the selected rows, in order
    idx = np.repeat(inst.row_ptr[users], lens) + (np.arange(int(rp[-1]), dtype=np.int64) - np.repeat(rp[:-1], lens))
    return Instance(rp, inst.col[idx].copy(), inst.c[idx].copy(), inst.a[idx].copy(), inst.b.copy(), inst.J,
                    None if inst.ids is None else inst.ids[users], inst.recipe)


# --------------------------------------------------------------------------
# Workload recipes (the five instance families the solver is measured on)
# --------------------------------------------------------------------------

def recipe_tiny(seed: int = 1000) -> Recipe:
    """10,000 users x 100 items; degree 1+Poisson(9); distinct uniform items;
    c = -U(0,1); a = 1; b_j = 0.05 * (item degree)."""
    return Recipe(I=10_000, J=100, seed=seed, deg_model=DEG_POISSON, deg_mean=10.0, deg_max=100,
                  item_model=ITEMS_UNIFORM, c_model=C_NEG_UNIFORM, a_model=A_ONE, b_model=B_ITEM_DEGREE,
                  b_frac=0.05)


def recipe_production(I: int = 20_000_000, J: int = 2_000, seed: int = 1001) -> Recipe:
    """Truncated-lognormal degree (mean 25, sigma 1, max 500); item popularity
    proportional to rank^-0.8 without replacement; c = -LogNormal(0, 0.5);
    a = U(0.5, 1.5); b_j = 0.05 * sum_i a_ij."""
    return Recipe(I=I, J=J, seed=seed)


def recipe_precision(I: int = 80_000_000, J: int = 5_000, seed: int = 1002) -> Recipe:
    """The production generators at 80M users x 5,000 items (~2B nnz)."""
    return Recipe(I=I, J=J, seed=seed)


def recipe_batch(n: int = 64, seed: int = 1003, users_lo: float = 1e4, users_hi: float = 5e6,
                 items_lo: float = 50, items_hi: float = 2000):
    """n independent instances of the production generator: users and items
    log-uniform in the given ranges, gamma drawn from {1e-1, 1e-2, 1e-3}.
    Returns a list of (Recipe, gamma)."""
    u = uniforms(seed, 0, 91, 3 * n)
    out = []
    for k in range(n):
        I = int(round(math.exp(math.log(users_lo) + (math.log(users_hi) - math.log(users_lo)) * u[3 * k])))
        J = int(round(math.exp(math.log(items_lo) + (math.log(items_hi) - math.log(items_lo)) * u[3 * k + 1])))
        gamma = (1e-1, 1e-2, 1e-3)[min(2, int(u[3 * k + 2] * 3))]
        out.append((Recipe(I=I, J=J, seed=seed + 1 + k), gamma))
    return out


def recipe_daily(I: int = 5_000_000, J: int = 1_000, seed: int = 1004) -> Recipe:
    """Base instance of the recurring daily workload (production generators)."""
    return Recipe(I=I, J=J, seed=seed)


def next_day(prev: Instance, day: int, seed: int = 1004, churn_p: float = 0.02, noise_p: float = 0.10,
             noise_sd: float = 0.02, b_sd: float = 0.05, nthreads: int = 0) -> Instance:
    """Day ``day`` from day ``day-1``: 2% of user slots churn to new users
    (rows regenerated), c += N(0, noise_sd) on 10% of surviving edges,
    b_j *= 1 + N(0, b_sd)."""
    lib = _load()
    r = prev.recipe
    n = prev.I
    day_seed = (seed * 1_000_003 + day * 7919) & 0xFFFFFFFFFFFFFFFF
    prev_ids = prev.ids if prev.ids is not None else np.arange(n, dtype=np.int64)
    new_ids = np.empty(n, dtype=np.int64)
    lib.synth_next_day_ids(day_seed, n, _ptr(prev_ids), churn_p, (day + 1) * (1 << 40), _ptr(new_ids), nthreads)
    p = r._c()
    deg = (prev.row_ptr[1:] - prev.row_ptr[:-1]).astype(np.int32)
    churned = np.nonzero(new_ids != prev_ids)[0]
    if len(churned):
        d2 = np.empty(len(churned), dtype=np.int32)
        lib.synth_degrees(ctypes.byref(p), _ptr(np.ascontiguousarray(new_ids[churned])), len(churned), _ptr(d2),
                          nthreads)
        deg[churned] = d2
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=rp[1:])
    nnz = int(rp[-1])
    col = np.empty(nnz, np.int32)
    c = np.empty(nnz, np.float32)
    a = np.empty(nnz, np.float32)
    lib.synth_next_day_fill(ctypes.byref(p), day_seed, n, _ptr(prev_ids), _ptr(prev.row_ptr), _ptr(prev.col),
                            _ptr(prev.c), _ptr(prev.a), _ptr(new_ids), _ptr(rp), _ptr(col), _ptr(c), _ptr(a),
                            noise_p, noise_sd, nthreads)
    b = prev.b.copy()
    lib.synth_scale_capacity(day_seed, r.J, b_sd, _ptr(b))
    return Instance(rp, col, c, a, b, r.J, new_ids, r)


# --------------------------------------------------------------------------
# The appendix generator (App. A): item-major breadth, distinct requests per
# resource, capped lognormal values, greedy-load capacities
# --------------------------------------------------------------------------

@dataclasses.dataclass
class AppRecipe:
    """Inputs of the App. A construction.  The paper gives its form but not
    its parameters; the defaults are this project's choice:

    * nu = 10 edges per request on average (the 0.1 % density of the
      10,000-resource instance of the preconditioning experiment);
    * breadth w_j ~ LogNormal(0, 1), p_j = w_j / sum w, K_j ~ Poisson(p_j I nu)
      truncated at I;
    * value v_j u_i eps_ij with v_j ~ LogNormal(0, 0.5), u_i ~ LogNormal(0, 0.5),
      eps_ij ~ LogNormal(0, 0.25), capped at c_max = 5; cost c_ij = -value;
    * a_ij = s_j * value, s_j ~ LogNormal(0, 1.5), so resource rows of A
      differ by orders of magnitude;
    * b_j = rho_j (l_j + 1e-3) with rho_j ~ U[0.5, 1] and l_j the greedy load.
    """

    I: int
    J: int
    seed: int
    nu: float = 10.0
    breadth_sigma: float = 1.0
    v_sigma: float = 0.5
    u_sigma: float = 0.5
    eps_sigma: float = 0.25
    c_max: float = 5.0
    s_mu: float = 0.0
    s_sigma: float = 1.5
    rho_lo: float = 0.5
    rho_hi: float = 1.0
    b_eps: float = 1e-3

    def _c(self) -> _AppParams:
        p = _AppParams()
        for f in dataclasses.fields(self):
            setattr(p, f.name, getattr(self, f.name))
        return p


@dataclasses.dataclass
class ItemMajor:
    """The resource-major draw of the appendix generator: resource j's
    requests are users[col_ptr[j]:col_ptr[j+1]], ascending."""

    col_ptr: np.ndarray  # int64 [J+1]
    users: np.ndarray  # int64 [nnz]


def appendix_item_major(r: AppRecipe, nthreads: int = 0) -> ItemMajor:
    lib = _load()
    p = r._c()
    K = np.empty(r.J, dtype=np.int64)
    if lib.synth_app_counts(ctypes.byref(p), _ptr(K)) != 0:
        raise MemoryError("synth_app_counts")
    col_ptr = np.zeros(r.J + 1, dtype=np.int64)
    np.cumsum(K, out=col_ptr[1:])
    users = np.empty(int(col_ptr[-1]), dtype=np.int64)
    if lib.synth_app_pick(ctypes.byref(p), _ptr(col_ptr), _ptr(users), nthreads) != 0:
        raise MemoryError("synth_app_pick")
    return ItemMajor(col_ptr, users)


def generate_appendix(r: AppRecipe, nthreads: int = 0, alloc=_np_empty, want_load: bool = False):
    """The App. A instance in this package's user-major CSR (requests are the
    users, resources the items; requests without edges keep empty rows).
    With ``want_load`` also returns the greedy loads l_j."""
    lib = _load()
    p = r._c()
    im = appendix_item_major(r, nthreads)
    deg = np.bincount(im.users, minlength=r.I)
    row_ptr = alloc(r.I + 1, np.int64)
    row_ptr[0] = 0
    np.cumsum(deg, dtype=np.int64, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    col = alloc(nnz, np.int32)
    if lib.synth_app_transpose(r.I, r.J, _ptr(im.col_ptr), _ptr(im.users), _ptr(row_ptr), _ptr(col), nthreads) != 0:
        raise MemoryError("synth_app_transpose")
    del im
    c = alloc(nnz, np.float32)
    a = alloc(nnz, np.float32)
    if lib.synth_app_values(ctypes.byref(p), r.I, _ptr(row_ptr), _ptr(col), _ptr(c), _ptr(a), nthreads) != 0:
        raise MemoryError("synth_app_values")
    b = np.empty(r.J, dtype=np.float64)
    load = np.empty(r.J, dtype=np.float64)
    if lib.synth_app_capacity(ctypes.byref(p), r.I, _ptr(row_ptr), _ptr(col), _ptr(a), _ptr(load), _ptr(b),
                              nthreads) != 0:
        raise MemoryError("synth_app_capacity")
    inst = Instance(row_ptr, col, c, a, b, r.J, None, None)
    return (inst, load) if want_load else inst


def recipe_appendix(I: int = 25_000_000, J: int = 10_000, seed: int = 1006) -> AppRecipe:
    """The appendix generator at 25M requests x 10,000 resources, 0.1 %
    density (~250M nnz)."""
    return AppRecipe(I=I, J=J, seed=seed)
