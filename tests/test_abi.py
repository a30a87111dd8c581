"""Host-side checks of the C ABI: the library loads without a GPU and exports
every entry point include/lbm.h declares; defaults match the header."""
import ctypes
import os
import re

import pytest

from paper_1503_08718_gb300 import build, lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return lbm.load()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text))
    return names


def test_every_declared_entry_point_is_exported(lib):
    names = _declared()
    assert {"lbm_create", "lbm_set_geometry", "lbm_set_tensors", "lbm_solve",
            "lbm_k_eff", "lbm_destroy"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n
    # the Python binding wraps every declared entry point under the same name
    for n in names:
        assert callable(getattr(lbm, n)), n


def test_default_opts(lib):
    o = lbm.lbm_default_opts()
    assert (o.t_hot, o.t_cold, o.tau_max, o.tol) == (1.0, 0.0, 1.5, 1e-8)
    assert o.max_iters == 50_000_000 and o.check_every == 100
    assert o.storage == lbm.LBM_STORE_F32 and not o.t_init and not o.stream
    assert o.fuse == 1 and o.host_loop == 0
    assert ctypes.sizeof(lbm.lbm_solve_opts) == 88
    assert ctypes.sizeof(lbm.lbm_solve_info) == 56


def test_null_safety_without_a_device(lib):
    lbm.lbm_destroy(None)
    assert lbm.lbm_last_error(None) == "null context"
    st, k = lbm.lbm_k_eff(None)
    assert st == lbm.LBM_ERR_INVALID_ARG
    st, h = lbm.lbm_create(1, 8, 8, 0)
    assert st == lbm.LBM_ERR_INVALID_ARG and not h.value


def test_missing_library_fails_loudly(tmp_path):
    old = lbm._lib
    lbm._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            lbm.load(str(tmp_path / "nope.so"))
    finally:
        lbm._lib = old
