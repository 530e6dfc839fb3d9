"""CPU checks of the C ABI library: it loads without a GPU and exports every
function that include/lsgmres.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lsgmres.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\*?\s+\**([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared()
    for f in ("gmres_create", "gmres_set", "gmres_set_stream", "gmres_solve", "gmres_history",
              "gmres_destroy", "gmres_last_error"):
        assert f in names


def test_library_builds_and_exports_every_symbol():
    from paper_1809_05805_b300 import build, lsgmres

    build.build()
    lib = ctypes.CDLL(lsgmres.LIB_PATH)
    missing = [f for f in declared() if not hasattr(lib, f)]
    assert not missing, missing
    assert sorted(lsgmres.EXPORTS) == declared()


def test_create_error_paths_without_gpu():
    """gmres_create rejects a malformed CSR on the host before touching the device."""
    import numpy as np

    from paper_1809_05805_b300 import lsgmres

    lib = lsgmres.load()
    rowptr = np.array([0, 3, 2], dtype=np.int32)  # rowptr[n] = nnz but decreasing
    col = np.array([0, 1], dtype=np.int32)
    val = np.ones(2)
    csr = lsgmres._Csr(2, 2, rowptr.ctypes.data, col.ctypes.data, val.ctypes.data, 0)
    h = ctypes.c_void_p()
    assert lib.gmres_create(ctypes.byref(csr), 5, 1e-8, ctypes.byref(h)) == lsgmres.ERR_ARG
    assert b"nondecreasing" in lib.gmres_last_error(None)
    csr = lsgmres._Csr(2, 2, rowptr.ctypes.data, col.ctypes.data, val.ctypes.data, 0)
    assert lib.gmres_create(ctypes.byref(csr), 0, 1e-8, ctypes.byref(h)) == lsgmres.ERR_ARG
