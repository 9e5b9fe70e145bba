"""ctypes binding of libmpchol.so (include/mpchol.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  `load()` fails loudly when the library is missing -- there is no
CPU fallback.  PyTorch provides device memory (tensors) and streams.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmpchol.so")

MP_OK, MP_ERR_ARG, MP_ERR_NOT_SPD, MP_ERR_OOM, MP_ERR_CUDA, MP_ERR_TIMEOUT, MP_ERR_STATE = range(7)
MP_F64, MP_F32, MP_BF16, MP_F16, MP_E4M3 = range(5)
MP_TMAT_KEEP_SIGMA = 1
MP_TMAT_SIMT_UPDATES = 2
MP_TMAT_STREAM_ALLOC = 4
MP_TMAT_FP64_PANEL = 8
MP_TMAT_DAG16 = 32
MP_TMAT_DAG32 = 64
MP_TMAT_LOWP_RING4 = 128
MP_TMAT_DIRECT = 256
MP_TMAT_TRACE = 512
TRACE_POINTS = ("taken", "inputs_final", "inverse_ready", "solved", "updated", "factored",
                "published", "done")
ELEM_BYTES = {MP_F64: 8, MP_F32: 4, MP_BF16: 2, MP_F16: 2, MP_E4M3: 1}


class mp_matern(C.Structure):
    _fields_ = [("sigma2", C.c_double), ("range", C.c_double), ("nu", C.c_double),
                ("nugget", C.c_double)]


class mp_serve_result(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int32), ("nrhs", C.c_int32), ("n", C.c_int64),
                ("b", C.c_int32), ("low_tiles", C.c_int32), ("offdiag_tiles", C.c_int32),
                ("pad_", C.c_int32), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double), ("logdet", C.c_double), ("loglik0", C.c_double)]


class mp_request(C.Structure):
    _fields_ = [("n", C.c_int64), ("h_map", C.c_void_p), ("d_locs", C.c_void_p),
                ("d_z", C.c_void_p), ("nrhs", C.c_int32), ("refine_iters", C.c_int32),
                ("cov", mp_matern), ("rule_band", C.c_int32), ("rule_near", C.c_uint8),
                ("rule_far", C.c_uint8), ("rule_pad_", C.c_uint8 * 2), ("rule_eps", C.c_double)]


class mp_tuned(C.Structure):
    _fields_ = [("b", C.c_int32), ("flags", C.c_uint32), ("ms", C.c_double), ("from_cache", C.c_int32),
                ("tried", C.c_int32)]


P = C.c_void_p
_SIGS = {
    "mp_ctx_create": (C.c_int, [C.c_int, C.POINTER(P)]),
    "mp_ctx_destroy": (None, [P]),
    "mp_status_string": (C.c_char_p, [C.c_int]),
    "mp_last_error": (C.c_int, [P, C.c_char_p, C.c_size_t]),
    "mp_version": (C.c_char_p, []),
    "mp_tmat_create": (C.c_int, [P, C.c_int64, C.c_int32, P, C.c_uint32, P, C.POINTER(P)]),
    "mp_tmat_destroy": (None, [P]),
    "mp_tmat_info": (C.c_int, [P, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                               C.POINTER(C.c_int32), C.POINTER(C.c_int64)]),
    "mp_tile_get": (C.c_int, [P, C.c_int32, C.c_int32, P, C.POINTER(C.c_double)]),
    "mp_tile_set": (C.c_int, [P, C.c_int32, C.c_int32, P, C.c_double]),
    "mp_morton_order": (C.c_int, [P, C.c_int64, P, P, P, P]),
    "mp_generate_matern": (C.c_int, [P, P, mp_matern]),
    "mp_chol": (C.c_int, [P, P, P]),
    "mp_chol_steps": (C.c_int, [P, C.c_int32, C.c_int32]),
    "mp_logdet": (C.c_int, [P, P]),
    "mp_tmat_set_wait_budget": (C.c_int, [P, C.c_int32]),
    "mp_tmat_chain_trace": (C.c_int, [P, P, C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
    "mp_potrf_dag_schedule": (C.c_int, [C.c_int32, P, C.c_int64, C.POINTER(C.c_int64)]),
    "mp_solve_dag_schedule": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, P, C.c_int64, C.POINTER(C.c_int64)]),
    "mp_trsm": (C.c_int, [P, C.c_int, P, C.c_int64, C.c_int32]),
    "mp_solve": (C.c_int, [P, P, C.c_int64, C.c_int32]),
    "mp_chol2inv": (C.c_int, [P, P, C.c_int64]),
    "mp_loglik": (C.c_int, [P, P, C.c_int64, C.c_int32, C.c_int32, P, P, P]),
    "mp_tile_norms": (C.c_int, [P, C.c_int64, C.c_int32, P, mp_matern, P, P]),
    "mp_map_guarded": (C.c_int, [C.c_int32, P, C.c_int32, C.c_uint8, C.c_uint8, C.c_double, P]),
    "mp_matern_host": (C.c_int, [mp_matern, C.c_int64, P, P]),
    "mp_tmat_stats": (C.c_int, [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                C.POINTER(C.c_int64)]),
    "mp_chol_profile": (C.c_int, [P, C.c_int32, P, P, P]),
    "mp_probe_fp64_peak": (C.c_int, [C.c_int, C.POINTER(C.c_double)]),
    "mp_gemm": (C.c_int, [P, C.c_int, C.c_char, C.c_char, C.c_int64, C.c_int64, C.c_int64,
                          C.c_double, P, C.c_int64, P, C.c_int64, C.c_double, P, C.c_int64, P]),
    "mp_server_create": (C.c_int, [P, C.c_int64, C.c_int32, C.c_double, C.c_uint8, C.POINTER(P)]),
    "mp_server_destroy": (None, [P]),
    "mp_server_submit": (C.c_int, [P, C.c_int64, P, P, C.c_int32, C.c_int32, mp_matern,
                                   C.POINTER(C.c_int64)]),
    "mp_server_poll": (C.c_int, [P, P, C.c_int32, C.POINTER(C.c_int32)]),
    "mp_server_result": (C.c_int, [P, C.c_int64, P, P]),
    "mp_server_factor": (C.c_int, [P, C.c_int64, C.POINTER(P)]),
    "mp_server_release": (C.c_int, [P, C.c_int64]),
    "mp_server_inject_alloc_failures": (C.c_int, [P, C.c_int32]),
    "mp_server_tune": (C.c_int, [P, P, C.c_int32, C.c_int32, C.c_char_p]),
    "mp_batch_create_ex": (C.c_int, [P, C.c_int32, P, C.c_int32, C.c_uint32, P, C.POINTER(P)]),
    "mp_batch_flags": (C.c_int, [P, C.POINTER(C.c_uint32)]),
    "mp_tune_batch": (C.c_int, [P, C.c_int32, P, C.c_char_p, P, P]),
    "mp_tune_tmat": (C.c_int, [P, C.c_int64, C.c_uint8, C.c_double, C.c_int32, C.c_char_p, P, P]),
    "mp_server_stats": (C.c_int, [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                  C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "mp_map_bound": (C.c_int, [C.c_int64, C.c_int32, P, mp_matern, C.c_int32, C.c_uint8, C.c_uint8,
                               C.c_double, P]),
    "mp_batch_create": (C.c_int, [P, C.c_int32, C.POINTER(mp_request), C.c_int32, P,
                                  C.POINTER(P)]),
    "mp_batch_destroy": (None, [P]),
    "mp_batch_info": (C.c_int, [P, C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
    "mp_batch_run": (C.c_int, [P, P, P]),
    "mp_loglik_batch": (C.c_int, [P, C.c_int32, C.POINTER(mp_request), P, P, P]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Loads the library (building it first when the CUDA toolkit is here and
    the library is missing or stale) and declares every entry point."""
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _build
    if not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libmpchol.so not found at {path}; run build()")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class MPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(s):
    if s is None:
        import torch
        s = torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Context:
    def __init__(self, device: int = 0):
        self.lib = load()
        h = P()
        self._check(self.lib.mp_ctx_create(device, C.byref(h)), None)
        self.h = h
        self.device = device

    def _check(self, st, ctx=None):
        if st != MP_OK:
            buf = C.create_string_buffer(512)
            self.lib.mp_last_error(ctx if ctx is not None else getattr(self, "h", None), buf, 512)
            raise MPError(st, f"{self.lib.mp_status_string(st).decode()}: {buf.value.decode()}")

    def check(self, st):
        self._check(st, self.h)

    def close(self):
        if getattr(self, "h", None):
            self.lib.mp_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def morton_order(self, locs, stream=None):
        import torch
        n = locs.shape[0]
        out = torch.empty_like(locs)
        perm = torch.empty(n, dtype=torch.int64, device=locs.device)
        self.check(self.lib.mp_morton_order(self.h, n, _ptr(locs), _ptr(out), _ptr(perm),
                                            _stream(stream)))
        return out, perm

    def tile_norms(self, n, b, locs, sigma2, range_, nu, nugget, stream=None):
        import torch
        nt = -(-n // b)
        out = torch.empty(nt * nt, dtype=torch.float64, device=locs.device)
        self.check(self.lib.mp_tile_norms(self.h, n, b, _ptr(locs),
                                          mp_matern(sigma2, range_, nu, nugget), _ptr(out),
                                          _stream(stream)))
        return out.view(nt, nt)

    def map_guarded(self, norms, band, near, far, eps):
        nrm = np.ascontiguousarray(np.asarray(norms, dtype=np.float64))
        nt = nrm.shape[0]
        m = np.empty((nt, nt), dtype=np.uint8)
        self.check(self.lib.mp_map_guarded(nt, nrm.ctypes.data_as(C.c_void_p), band, near, far,
                                           eps, m.ctypes.data_as(C.c_void_p)))
        return m

    def fp64_peak(self):
        v = C.c_double()
        self.check(self.lib.mp_probe_fp64_peak(self.device, C.byref(v)))
        return v.value

    def gemm(self, dtype, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, Cm, ldc, stream=None):
        self.check(self.lib.mp_gemm(self.h, dtype, ta.encode(), tb.encode(), m, n, k, alpha,
                                    _ptr(A), lda, _ptr(B), ldb, beta, _ptr(Cm), ldc,
                                    _stream(stream)))


class TiledMatrix:
    """mp_tmat: an n x n tiled matrix with a per-tile precision map."""

    def __init__(self, ctx: Context, n: int, b: int, pmap=None, keep_sigma=False, stream=None,
                 simt_updates=False, ozaki=True, flags=0):
        self.ctx, self.lib = ctx, ctx.lib
        self.n, self.b = n, b
        self.nt = -(-n // b)
        self.stream = stream
        self._map = None
        if pmap is not None:
            self._map = np.ascontiguousarray(np.asarray(pmap, dtype=np.uint8))
            assert self._map.shape == (self.nt, self.nt)
        h = P()
        flags = ((MP_TMAT_KEEP_SIGMA if keep_sigma else 0) | (MP_TMAT_SIMT_UPDATES if simt_updates else 0)
                 | (0 if ozaki else MP_TMAT_FP64_PANEL) | flags)
        mp = None if self._map is None else self._map.ctypes.data_as(C.c_void_p)
        ctx.check(self.lib.mp_tmat_create(ctx.h, n, b, mp, flags, _stream(stream), C.byref(h)))
        self.h = h

    def close(self):
        # a handle outlives its context only at interpreter shutdown (objects
        # held in reference cycles are finalised in any order): its memory
        # went with the context's process state, and destroying it would
        # reach through the freed context
        if getattr(self, "h", None):
            if getattr(getattr(self, "ctx", None), "h", None):
                self.lib.mp_tmat_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        n, b, nt, by = C.c_int64(), C.c_int32(), C.c_int32(), C.c_int64()
        self.ctx.check(self.lib.mp_tmat_info(self.h, C.byref(n), C.byref(b), C.byref(nt), C.byref(by)))
        return dict(n=n.value, b=b.value, nt=nt.value, bytes=by.value)

    def dtype(self, i, j):
        return MP_F64 if self._map is None else int(self._map[i, j])

    def generate(self, locs, sigma2, range_, nu, nugget):
        self.locs = locs            # keep the borrowed buffer alive
        self.ctx.check(self.lib.mp_generate_matern(self.h, _ptr(locs),
                                                   mp_matern(sigma2, range_, nu, nugget)))

    def chol(self):
        import torch
        dev = torch.device("cuda", self.ctx.device)
        info = torch.zeros(1, dtype=torch.int64, device=dev)
        logdet = torch.zeros(1, dtype=torch.float64, device=dev)
        self.ctx.check(self.lib.mp_chol(self.h, _ptr(info), _ptr(logdet)))
        return info, logdet

    def chol_steps(self, k0, k1):
        self.ctx.check(self.lib.mp_chol_steps(self.h, k0, k1))

    def set_wait_budget(self, polls: int):
        """Polls a task-graph wait makes before it gives up (0: default)."""
        self.ctx.check(self.lib.mp_tmat_set_wait_budget(self.h, polls))

    def chain_trace(self):
        """Stamps of the last factorisation's critical chain (the matrix
        was created with flags=MP_TMAT_TRACE): returns (ns, cycles, DB) with
        ns and cycles of shape (nt, b / DB, 8), the points of TRACE_POINTS
        for each diagonal block of each diagonal tile."""
        cnt, blk = C.c_int64(), C.c_int32()
        self.ctx.check(self.lib.mp_tmat_chain_trace(self.h, None, 0, C.byref(cnt), C.byref(blk)))
        buf = np.zeros(cnt.value, dtype=np.uint64)
        self.ctx.check(self.lib.mp_tmat_chain_trace(self.h, buf.ctypes.data_as(C.c_void_p), cnt.value,
                                                    C.byref(cnt), C.byref(blk)))
        w = buf.reshape(self.nt, -1, 16).astype(np.int64)
        return w[:, :, :8], w[:, :, 8:], blk.value

    def logdet(self, out):
        self.ctx.check(self.lib.mp_logdet(self.h, _ptr(out)))

    def solve(self, Bt):
        """Sigma X = B in place; Bt is (nrhs, n) float64 on the device (the
        transpose of the column-major n x nrhs B)."""
        self.ctx.check(self.lib.mp_solve(self.h, _ptr(Bt), Bt.shape[1], Bt.shape[0]))
        return Bt

    def chol2inv(self, out=None):
        """(L L^T)^-1 as an (n, n) float64 device tensor (symmetric)."""
        import torch
        if out is None:
            out = torch.empty((self.n, self.n), dtype=torch.float64, device=torch.device("cuda", self.ctx.device))
        self.ctx.check(self.lib.mp_chol2inv(self.h, _ptr(out), self.n))
        return out

    def trsm(self, B, trans=0):
        """B: (nrhs, ld) float64 CUDA tensor = column-major n x nrhs."""
        self.ctx.check(self.lib.mp_trsm(self.h, trans, _ptr(B), B.shape[1], B.shape[0]))

    def loglik(self, zt, refine_iters=0, ll=None, quad=None, iters=None):
        """zt: (nrhs, ld) float64 CUDA tensor (column-major z).  Returns device
        tensors (ll, quad, iters)."""
        import torch
        nrhs = zt.shape[0]
        dev = zt.device
        ll = torch.empty(nrhs, dtype=torch.float64, device=dev) if ll is None else ll
        quad = torch.empty(nrhs, dtype=torch.float64, device=dev) if quad is None else quad
        iters = torch.empty(nrhs, dtype=torch.int32, device=dev) if iters is None else iters
        self.ctx.check(self.lib.mp_loglik(self.h, _ptr(zt), zt.shape[1], nrhs, refine_iters,
                                          _ptr(ll), _ptr(quad), _ptr(iters)))
        return ll, quad, iters

    def stats(self):
        a, g, l = C.c_int64(), C.c_int64(), C.c_int64()
        self.ctx.check(self.lib.mp_tmat_stats(self.h, C.byref(a), C.byref(g), C.byref(l)))
        return dict(chol=a.value, generate=g.value, loglik=l.value)

    PROFILE_CLASSES = ["potrf_tile", "panel_trsm", "panel_round", "update_f64", "update_simt",
                       "update_tc_3xtf32", "fp8_round", "other", "panel_trsm_first", "panel_ozaki_gemm",
                       "ozaki_split", "update_tc_lowp"]

    def profile(self):
        k = len(self.PROFILE_CLASSES)
        ms = np.zeros(k, dtype=np.float32)
        nl = np.zeros(k, dtype=np.int64)
        fl = np.zeros(k, dtype=np.float64)
        self.ctx.check(self.lib.mp_chol_profile(self.h, k, ms.ctypes.data_as(C.c_void_p),
                                                nl.ctypes.data_as(C.c_void_p),
                                                fl.ctypes.data_as(C.c_void_p)))
        return {c: dict(ms=float(ms[i]), launches=int(nl[i]), flops=float(fl[i]))
                for i, c in enumerate(self.PROFILE_CLASSES)}

    def get_tile(self, i, j):
        """Returns (values as float64 numpy b x b, raw codes array, scale)."""
        dt = self.dtype(i, j)
        raw = np.empty(self.b * self.b * ELEM_BYTES[dt], dtype=np.uint8)
        s = C.c_double()
        self.ctx.check(self.lib.mp_tile_get(self.h, i, j, raw.ctypes.data_as(C.c_void_p), C.byref(s)))
        codes = decode(raw, dt).reshape(self.b, self.b)
        return codes * s.value, codes, s.value

    def set_tile(self, i, j, codes, scale=1.0):
        dt = self.dtype(i, j)
        raw = encode(np.asarray(codes, dtype=np.float64).reshape(-1), dt)
        self.ctx.check(self.lib.mp_tile_set(self.h, i, j, raw.ctypes.data_as(C.c_void_p), scale))


def _requests(reqs, keep):
    arr = (mp_request * len(reqs))()
    for k, r in enumerate(reqs):
        m = r.get("map")
        mp = None
        if m is not None:
            m = np.ascontiguousarray(np.asarray(m, dtype=np.uint8))
            keep.append(m)
            mp = m.ctypes.data
        keep += [r["locs"], r["zt"]]
        band, near, far, eps = r.get("rule", (0, 0, 0, 0.0))
        arr[k] = mp_request(r["n"], mp, r["locs"].data_ptr(), r["zt"].data_ptr(), r["zt"].shape[0], 0,
                            mp_matern(r["sigma2"], r["range"], r["nu"], r["nugget"]), band, near, far,
                            (C.c_uint8 * 2)(), eps)
    return arr


def tune_batch(ctx: "Context", reqs, cache_path=None, stream=None):
    """The autotuner's choice for these requests: dict(b, flags, ms, from_cache, tried)."""
    keep = []
    arr = _requests(reqs, keep)
    t = mp_tuned()
    ctx.check(ctx.lib.mp_tune_batch(ctx.h, len(reqs), arr, cache_path.encode() if cache_path else None,
                                    _stream(stream), C.byref(t)))
    return {k: getattr(t, k) for k, _ in mp_tuned._fields_}


def tune_tmat(ctx: "Context", n, far=MP_BF16, eps=1e-6, refine_iters=0, cache_path=None, stream=None):
    t = mp_tuned()
    ctx.check(ctx.lib.mp_tune_tmat(ctx.h, n, far, eps, refine_iters,
                                   cache_path.encode() if cache_path else None, _stream(stream), C.byref(t)))
    return {k: getattr(t, k) for k, _ in mp_tuned._fields_}


class Batch:
    """mp_batch: many log-likelihood requests in one CUDA graph."""

    def __init__(self, ctx: Context, reqs, b=0, stream=None, flags=None):
        """reqs: dicts with n, locs (device, n x 2), zt (device, nrhs x n),
        sigma2, range, nu, nugget, and either map (explicit, at this b) or
        rule = (band, near, far, eps) (the bound map at the plan's b).
        b = 0: the library's autotuner picks b and the schedule flags."""
        self.ctx, self.lib = ctx, ctx.lib
        self._keep = []
        self.arr = _requests(reqs, self._keep)
        h = P()
        if flags is None:
            ctx.check(self.lib.mp_batch_create(ctx.h, len(reqs), self.arr, b, _stream(stream), C.byref(h)))
        else:
            ctx.check(self.lib.mp_batch_create_ex(ctx.h, len(reqs), self.arr, b, flags, _stream(stream),
                                                  C.byref(h)))
        self.h = h
        self.count = len(reqs)
        self.total_rhs = sum(r["zt"].shape[0] for r in reqs)

    def info(self):
        by, b, f = C.c_int64(), C.c_int32(), C.c_uint32()
        self.ctx.check(self.lib.mp_batch_info(self.h, C.byref(by), C.byref(b)))
        self.ctx.check(self.lib.mp_batch_flags(self.h, C.byref(f)))
        return dict(bytes=by.value, b=b.value, flags=f.value)

    def run(self, ll=None, status=None):
        import torch
        dev = torch.device("cuda", self.ctx.device)
        ll = torch.empty(self.total_rhs, dtype=torch.float64, device=dev) if ll is None else ll
        status = torch.empty(self.count, dtype=torch.int32, device=dev) if status is None else status
        self.ctx.check(self.lib.mp_batch_run(self.h, _ptr(ll), _ptr(status)))
        return ll, status

    def close(self):
        # a handle outlives its context only at interpreter shutdown (objects
        # held in reference cycles are finalised in any order): its memory
        # went with the context's process state, and destroying it would
        # reach through the freed context
        if getattr(self, "h", None):
            if getattr(getattr(self, "ctx", None), "h", None):
                self.lib.mp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """mp_server: continuous batching of log-likelihood requests."""

    def __init__(self, ctx: Context, hbm_budget: int, max_slots: int = 8, eps: float = 1e-6,
                 far=MP_BF16):
        self.ctx, self.lib = ctx, ctx.lib
        h = P()
        ctx.check(self.lib.mp_server_create(ctx.h, int(hbm_budget), max_slots, eps, far, C.byref(h)))
        self.h = h
        self._buf = (mp_serve_result * 64)()

    def submit(self, locs: np.ndarray, z: np.ndarray, cov, refine_iters=0) -> int:
        """locs (n, 2) float64; z (n, nrhs) float64 (copied); cov = (sigma2, range, nu, nugget)."""
        locs = np.ascontiguousarray(locs, dtype=np.float64)
        zt = np.ascontiguousarray(np.asarray(z, dtype=np.float64).reshape(locs.shape[0], -1).T)
        rid = C.c_int64()
        self.ctx.check(self.lib.mp_server_submit(self.h, locs.shape[0], locs.ctypes.data_as(C.c_void_p),
                                                 zt.ctypes.data_as(C.c_void_p), zt.shape[0],
                                                 refine_iters, mp_matern(*cov), C.byref(rid)))
        return rid.value

    def poll(self):
        n = C.c_int32()
        self.ctx.check(self.lib.mp_server_poll(self.h, self._buf, len(self._buf), C.byref(n)))
        out = []
        for i in range(n.value):
            r = self._buf[i]
            out.append({k: getattr(r, k) for k, _ in mp_serve_result._fields_ if k != "pad_"})
        return out

    def result(self, rid: int, nrhs: int):
        ll = np.empty(nrhs)
        quad = np.empty(nrhs)
        st = self.lib.mp_server_result(self.h, rid, ll.ctypes.data_as(C.c_void_p),
                                       quad.ctypes.data_as(C.c_void_p))
        return st, ll, quad

    def release(self, rid: int):
        self.ctx.check(self.lib.mp_server_release(self.h, rid))

    def tune(self, sizes, refine_iters=0, cache_path=None):
        """Autotunes b and the schedule flags for requests of these sizes."""
        arr = np.ascontiguousarray(np.asarray(sizes, dtype=np.int64))
        self.ctx.check(self.lib.mp_server_tune(self.h, arr.ctypes.data_as(C.c_void_p), arr.size, refine_iters,
                                               cache_path.encode() if cache_path else None))

    def inject_alloc_failures(self, count: int):
        """The next `count` admissions fail their allocation (host-made)."""
        self.ctx.check(self.lib.mp_server_inject_alloc_failures(self.h, count))

    def stats(self):
        q, r, k, b = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        self.ctx.check(self.lib.mp_server_stats(self.h, C.byref(q), C.byref(r), C.byref(k), C.byref(b)))
        return dict(queued=q.value, running=r.value, kept=k.value, bytes=b.value)

    def close(self):
        # a handle outlives its context only at interpreter shutdown (objects
        # held in reference cycles are finalised in any order): its memory
        # went with the context's process state, and destroying it would
        # reach through the freed context
        if getattr(self, "h", None):
            if getattr(getattr(self, "ctx", None), "h", None):
                self.lib.mp_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def matern_host(r, sigma2, range_, nu):
    """C(r) by the library's host evaluation (closed forms or the per-nu
    Chebyshev table of the generation kernels)."""
    lib = load()
    r = np.ascontiguousarray(np.asarray(r, dtype=np.float64).reshape(-1))
    out = np.empty_like(r)
    st = lib.mp_matern_host(mp_matern(sigma2, range_, nu, 0.0), r.size, r.ctypes.data_as(C.c_void_p),
                            out.ctypes.data_as(C.c_void_p))
    if st != MP_OK:
        raise MPError(st, "mp_matern_host")
    return out


def potrf_dag_schedule(nb):
    """The diagonal tile's task order for nb blocks: int array (tasks, 4)
    of op, r, c, k (host only)."""
    lib = load()
    cnt = C.c_int64()
    st = lib.mp_potrf_dag_schedule(nb, None, 0, C.byref(cnt))
    if st != MP_OK:
        raise MPError(st, "mp_potrf_dag_schedule")
    out = np.empty(4 * cnt.value, dtype=np.uint8)
    st = lib.mp_potrf_dag_schedule(nb, out.ctypes.data_as(C.c_void_p), cnt.value, C.byref(cnt))
    if st != MP_OK:
        raise MPError(st, "mp_potrf_dag_schedule")
    return out.reshape(-1, 4).astype(np.int64)


def solve_dag_schedule(nt, p_blocks, trans):
    """A triangular solve's task order: int array (tasks, 4) of op, i, j, p
    (host only)."""
    lib = load()
    cnt = C.c_int64()
    st = lib.mp_solve_dag_schedule(nt, p_blocks, trans, None, 0, C.byref(cnt))
    if st != MP_OK:
        raise MPError(st, "mp_solve_dag_schedule")
    out = np.empty(cnt.value, dtype=np.uint64)
    st = lib.mp_solve_dag_schedule(nt, p_blocks, trans, out.ctypes.data_as(C.c_void_p), cnt.value,
                                   C.byref(cnt))
    if st != MP_OK:
        raise MPError(st, "mp_solve_dag_schedule")
    w = out.astype(np.uint64)
    return np.stack([(w >> np.uint64(24)) & np.uint64(0xf), (w >> np.uint64(28)) & np.uint64(0xfff),
                     (w >> np.uint64(40)) & np.uint64(0xfff), (w >> np.uint64(52)) & np.uint64(0xff)],
                    axis=1).astype(np.int64)


def map_bound(n, b, sorted_locs, cov, band, near, far, eps):
    lib = load()
    nt = -(-n // b)
    m = np.empty((nt, nt), dtype=np.uint8)
    locs = np.ascontiguousarray(sorted_locs, dtype=np.float64)
    st = lib.mp_map_bound(n, b, locs.ctypes.data_as(C.c_void_p), mp_matern(*cov), band, near, far,
                          eps, m.ctypes.data_as(C.c_void_p))
    if st != MP_OK:
        raise MPError(st, "mp_map_bound")
    return m


# ---- host-side codecs of the storage formats (for tile upload/download) ----

def decode(raw: np.ndarray, dt: int) -> np.ndarray:
    import torch
    if dt == MP_F64:
        return raw.view(np.float64).copy()
    if dt == MP_F32:
        return raw.view(np.float32).astype(np.float64)
    if dt == MP_F16:
        return raw.view(np.float16).astype(np.float64)
    t = torch.from_numpy(raw.copy())
    if dt == MP_BF16:
        return t.view(torch.bfloat16).to(torch.float64).numpy()
    return t.view(torch.float8_e4m3fn).to(torch.float64).numpy()


def encode(vals: np.ndarray, dt: int) -> np.ndarray:
    """Packs values that are already representable in `dt` (exact)."""
    import torch
    if dt == MP_F64:
        return vals.astype(np.float64).view(np.uint8)
    if dt == MP_F32:
        return vals.astype(np.float32).view(np.uint8)
    if dt == MP_F16:
        return vals.astype(np.float16).view(np.uint8)
    t = torch.from_numpy(vals.astype(np.float32))
    if dt == MP_BF16:
        return t.to(torch.bfloat16).view(torch.uint8).numpy().copy()
    return t.to(torch.float8_e4m3fn).view(torch.uint8).numpy().copy()
