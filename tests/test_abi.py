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


def test_workspace_bytes_cover_the_buffers(lib):
    """lbm_workspace_bytes is at least the context's raw buffer bytes (two
    distribution buffers of 4 stored fields per node, phase map and its canonical copy, the
    T staging and snapshot fields, the check history) and only alignment and
    per-plane scratch above that; 16-bit storage needs less; bad input gives 0."""
    nx, ny, nz = 128, 128, 256
    N = nx * ny * nz
    raw = 2 * 4 * 4 * N + N + N + 4 * N + 4 * N + 8 * 4 * 65536
    got = lbm.lbm_workspace_bytes(nx, ny, nz, lbm.LBM_STORE_F32)
    assert raw <= got <= raw + (1 << 20)
    assert lbm.lbm_workspace_bytes(nx, ny, nz, lbm.LBM_STORE_BF16) < got
    # padding: rows of 5 nodes are padded to 8 (4-node vectors) along any axis
    assert lbm.lbm_workspace_bytes(5, 9, 7, lbm.LBM_STORE_F32) >= 2 * 4 * 4 * 8 * 9 * 7
    assert lbm.lbm_workspace_bytes(1, 8, 8, 0) == 0
    assert lbm.lbm_workspace_bytes(8, 8, 8, 9) == 0
    st, h = lbm.lbm_create_with_workspace(8, 8, 8, 0, 0, 1 << 20)
    assert st == lbm.LBM_ERR_INVALID_ARG and not h.value
