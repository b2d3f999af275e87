"""Host-side checks of the C ABI that need no GPU: the library builds, loads,
exports every entry point that include/mds.h declares, and rejects bad
arguments before touching a device."""
import ctypes
import os
import re

import pytest

from paper_1905_04582_gb300 import build as B
from paper_1905_04582_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return capi.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "mds.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mds_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mds_create", "mds_set_data", "mds_set_locations", "mds_set_sigma", "mds_log_likelihood",
                     "mds_gradient", "mds_leapfrog", "mds_destroy", "mds_hmc", "mds_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/mds.h but not exported"
    # and the binding covers exactly the header
    assert set(declared_functions()) == set(capi.SIGNATURES)


def test_create_rejects_bad_arguments_before_the_device(lib):
    h = ctypes.c_void_p()
    assert lib.mds_create(1, 2, 0, ctypes.byref(h)) == capi.MDS_ERR_INVALID_ARG
    assert b"N must be" in lib.mds_last_error(None)
    assert lib.mds_create(10, 0, 0, ctypes.byref(h)) == capi.MDS_ERR_INVALID_ARG
    assert lib.mds_create(10, capi.MDS_MAX_D + 1, 0, ctypes.byref(h)) == capi.MDS_ERR_INVALID_ARG
    assert lib.mds_create(10, 2, 7, ctypes.byref(h)) == capi.MDS_ERR_INVALID_ARG
    assert lib.mds_create(10, 2, 0, None) == capi.MDS_ERR_INVALID_ARG


def test_null_context_calls_fail_cleanly(lib):
    assert lib.mds_destroy(None) == capi.MDS_OK
    assert lib.mds_set_sigma(None, 1.0) == capi.MDS_ERR_INVALID_ARG
    assert lib.mds_problem_size(None, None, None) == capi.MDS_ERR_INVALID_ARG
    assert isinstance(lib.mds_last_error(None), bytes)


def test_create_without_gpu_reports_unsupported(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = lib.mds_create(100, 2, 0, ctypes.byref(h))
    assert st in (capi.MDS_ERR_UNSUPPORTED, capi.MDS_ERR_CUDA)
    assert h.value is None


def test_product_path_has_no_fallback(tmp_path, monkeypatch):
    # with the library absent, the binding raises instead of computing anything
    monkeypatch.setattr(capi, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(capi, "_lib", None)
    with pytest.raises(RuntimeError, match="no fallback"):
        capi.lib()


def test_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1905_04582_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, flags=re.M), f
                assert "mds_oracle" not in text, f


def test_locality_order_tiles_a_grid_into_squares(lib):
    """On a 64 x 64 grid the bisection order makes every run of 64 items an
    8 x 8 square (each cut halves the wider side at a multiple of 64 items)."""
    from paper_1905_04582_gb300.mds import locality_order
    import numpy as np
    g = np.stack(np.meshgrid(np.arange(64.0), np.arange(64.0), indexing="ij"), -1).reshape(-1, 2)
    g = g[np.random.default_rng(0).permutation(len(g))]  # any input order
    perm = locality_order(g)
    assert sorted(perm.tolist()) == list(range(len(g)))
    blocks = g[perm].reshape(64, 64, 2)
    span = blocks.max(axis=1) - blocks.min(axis=1)
    assert np.all(span == 7.0)
    assert np.array_equal(perm, locality_order(g))  # deterministic


def test_locality_order_ragged_and_rejects_bad_input(lib):
    from paper_1905_04582_gb300.mds import locality_order
    import numpy as np
    x = np.random.default_rng(1).standard_normal((333, 3))
    perm = locality_order(x)
    assert sorted(perm.tolist()) == list(range(333))
    assert len(locality_order(x[:1])) == 1
    bad = x.copy()
    bad[5, 1] = np.nan
    with pytest.raises(capi.MDSError) as e:
        locality_order(bad)
    assert e.value.status == capi.MDS_ERR_INVALID_ARG
