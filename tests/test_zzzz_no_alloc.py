"""The allocation-free Morton ordering, called through the C ABI.

mp_morton_order_noalloc exists for callers that may not allocate device
memory (work enqueued during graph capture, loops that must not block on
the allocator, programs whose device memory another allocator owns).  Its
result must equal that of mp_morton_order, which sorts in a cudaMalloc'd
workspace; it is checked on two calls in a row, because every call reuses
the one fixed buffer that the previous call left behind.  This file is
named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

import mpinputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_02701_gb300 import mpchol
    L = mpchol.load()
    f = L.mp_morton_order_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    return L


def _with_workspace(L, locs):
    """Reference: mp_morton_order through a context (allocating workspace)."""
    ctx = C.c_void_p()
    assert L.mp_ctx_create(torch.cuda.current_device(), C.byref(ctx)) == 0
    n = locs.shape[0]
    out = torch.empty_like(locs)
    perm = torch.empty(n, dtype=torch.int64, device=locs.device)
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.mp_morton_order(ctx, n, C.c_void_p(locs.data_ptr()), C.c_void_p(out.data_ptr()),
                             C.c_void_p(perm.data_ptr()), s) == 0
    torch.cuda.synchronize()
    L.mp_ctx_destroy(ctx)
    return out, perm


def _no_alloc(L, locs):
    n = locs.shape[0]
    out = torch.empty_like(locs)
    perm = torch.empty(n, dtype=torch.int64, device=locs.device)
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = L.mp_morton_order_noalloc(n, C.c_void_p(locs.data_ptr()), C.c_void_p(out.data_ptr()),
                                   C.c_void_p(perm.data_ptr()), s)
    assert st == 0
    torch.cuda.synchronize()
    return out, perm


def test_no_alloc_morton_matches_workspace_version_twice(lib):
    # two calls in a row: the second one sorts a different, smaller set in
    # the buffer that still holds the first call's keys
    for n, seed in [(70000, 5), (3001, 6)]:
        locs = torch.from_numpy(I.points(n, seed)).to("cuda")
        ref_out, ref_perm = _with_workspace(lib, locs)
        got_out, got_perm = _no_alloc(lib, locs)
        assert torch.equal(got_perm, ref_perm)
        assert torch.equal(got_out, ref_out)
        p = got_perm.cpu().numpy()
        assert np.array_equal(np.sort(p), np.arange(n))


def test_no_alloc_rejects_sizes_beyond_its_buffer(lib):
    n = 131072 + 1
    locs = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    out = torch.empty_like(locs)
    perm = torch.empty(n, dtype=torch.int64, device="cuda")
    st = lib.mp_morton_order_noalloc(n, C.c_void_p(locs.data_ptr()), C.c_void_p(out.data_ptr()),
                                     C.c_void_p(perm.data_ptr()), None)
    assert st == 1   # MP_ERR_ARG
    buf = C.create_string_buffer(256)
    lib.mp_last_error(None, buf, 256)
    assert b"131072" in buf.value
