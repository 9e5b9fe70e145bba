"""The C-ABI library builds, loads and exports every declared entry point
(CPU only: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mpchol.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mp_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_paper_operations():
    names = _declared()
    for op in ["mp_tmat_create", "mp_generate_matern", "mp_chol", "mp_trsm", "mp_gemm",
               "mp_logdet", "mp_loglik", "mp_loglik_batch", "mp_morton_order"]:
        assert op in names


def test_library_builds_loads_and_exports_every_symbol():
    from paper_2406_02701_gb300 import build, mpchol
    build.build()
    lib = ctypes.CDLL(build.LIB)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    b = mpchol.load()
    assert b.mp_status_string(2) == b"matrix is not positive definite"
    assert b"sm_103a" in b.mp_version()


def test_context_without_device_is_an_error_not_a_crash():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2406_02701_gb300 import mpchol
    lib = mpchol.load()
    h = ctypes.c_void_p()
    st = lib.mp_ctx_create(0, ctypes.byref(h))
    assert st == mpchol.MP_ERR_ARG
