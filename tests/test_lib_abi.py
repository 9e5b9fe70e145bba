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


def test_handles_skip_destroy_once_their_context_is_closed():
    """A matrix, batch or server handle whose context is already closed (at
    interpreter shutdown, objects in reference cycles are finalised in any
    order) is dropped without calling its destroy function, which would
    reach through the freed context; with the context open it is destroyed
    once."""
    from paper_2406_02701_gb300 import mpchol

    class Lib:
        def __init__(self):
            self.calls = []

        def __getattr__(self, name):
            return lambda *a: self.calls.append(name)

    class Ctx:
        h = object()

    for cls, fn in ((mpchol.TiledMatrix, "mp_tmat_destroy"), (mpchol.Batch, "mp_batch_destroy"),
                    (mpchol.Server, "mp_server_destroy")):
        for open_ctx in (True, False):
            obj = cls.__new__(cls)
            obj.lib, obj.ctx, obj.h = Lib(), Ctx(), object()
            if not open_ctx:
                obj.ctx.h = None
            obj.close()
            obj.close()
            assert obj.h is None
            assert obj.lib.calls == ([fn] if open_ctx else []), (cls.__name__, open_ctx)
