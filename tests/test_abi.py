"""The C-ABI library loads and exports every entry point ``include/*.h``
declares, and rejects bad arguments on the host before touching a GPU.
CPU only (nvcc cross-compiles the library here)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

import paper_2606_07777_gb300 as dlm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(dlm_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    dlm.build()
    return dlm.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "dlm_create" in names and "dlm_solve" in names
    out = subprocess.run(["nm", "-D", "--defined-only", dlm.library_path()], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (dlm_[a-z0-9_]+)", out))
    missing = names - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    for n in names:
        assert hasattr(lib, n)
    assert set(dlm.EXPORTS) <= exported


def test_library_is_built_for_sm103a():
    out = subprocess.run(["strings", dlm.library_path()], capture_output=True, text=True).stdout
    assert "sm_103a" in out


def _desc(**kw):
    d = dlm.ProblemDesc()
    d.num_users, d.num_items, d.nnz = 2, 2, 3
    buf = (ctypes.c_int64 * 3)(0, 1, 3)
    d.row_ptr = ctypes.addressof(buf)
    d.item_idx = d.c = d.a = d.b = ctypes.addressof(buf)
    d.val_dtype, d.kind, d.z, d.memspace = 0, 0, 1.0, 1
    for k, v in kw.items():
        setattr(d, k, v)
    return d, buf


@pytest.mark.parametrize("field,value,needle", [
    ("num_items", 0, "num_items"),
    ("num_users", -1, "num_users"),
    ("nnz", -5, "nnz"),
    ("kind", 7, "kind"),
    ("val_dtype", 3, "val_dtype"),
    ("z", 0.0, "z must be"),
    ("z", float("nan"), "z must be"),
    ("memspace", 9, "memspace"),
    ("row_ptr", None, "null"),
])
def test_create_rejects_bad_arguments_on_host(lib, field, value, needle):
    d, keep = _desc(**{field: value})
    h = ctypes.c_void_p()
    st = lib.dlm_create(ctypes.byref(d), None, ctypes.byref(h))
    assert st == dlm.DLM_ERR_INVALID_ARG
    assert needle in lib.dlm_last_error().decode()
    assert not h.value


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.dlm_step(None, 1) == dlm.DLM_ERR_INVALID_ARG
    assert lib.dlm_set_schedule(None, 0.1, 0.01, 0.5, 10) == dlm.DLM_ERR_INVALID_ARG
    s = dlm.Stats()
    assert lib.dlm_get_stats(None, ctypes.byref(s)) == dlm.DLM_ERR_INVALID_ARG
    out = (ctypes.c_double * 4)()
    assert lib.dlm_get_trajectory(None, 0, 4, out) == dlm.DLM_ERR_INVALID_ARG
    lib.dlm_destroy(None)  # no-op
