/*
 * mpchol.h -- C ABI of the mixed-precision tiled Cholesky log-likelihood
 * library for NVIDIA GB300 (sm_103a).
 *
 * The calls follow the operations of the MPCR paper (arXiv 2406.02701):
 * a matrix object in a chosen precision (Sec. 4.1, `as.MPCR` with its
 * precision argument), `chol` (Sec. 6.2), `forwardsolve` / `backsolve`
 * (Sec. 5 and 6.2), `%*%` / `crossprod` (Sec. 5), `log(diag(U))` summed
 * into the log-determinant and the negative log-likelihood recipe (Sec. 6.2),
 * and the tiled multi-precision extension named as future work (Sec. 7):
 * every tile of the matrix carries its own precision.
 *
 * Conventions shared by every call
 *   - Pointers named d_* are DEVICE pointers (cudaMalloc / torch tensors on
 *     the library's device); they are borrowed, never freed by the library.
 *     Host pointers are named h_* or are plain structs/arrays.
 *   - `stream` arguments are cudaStream_t values passed as void*; NULL means
 *     the legacy default stream.  Every call that takes or owns a stream is
 *     asynchronous on it: results in device memory are valid after the
 *     stream is synchronised.  Host-visible results are returned only by the
 *     calls documented as synchronous.
 *   - Errors are returned as mp_status codes; nothing aborts.  A failing
 *     CUDA call yields MP_ERR_CUDA and its text is kept for mp_last_error.
 *     Failures found on the device (a pivot that is not positive, a wait
 *     that ran out) are written to device status words named in each call.
 *   - Matrices and right-hand sides are column-major with a leading
 *     dimension (R's convention): element (r, c) of B is B[r + c * ldb].
 *   - The library stores the LOWER factor L (Sigma = L L^T); the paper's R
 *     `chol` returns U = L^T.  The log-determinant is the same.
 *   - One mp_ctx per thread at a time; different contexts are independent.
 */
#ifndef MPCHOL_H
#define MPCHOL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MP_OK = 0,
  MP_ERR_ARG = 1,      /* invalid argument (sizes, map, dtype, pointer) */
  MP_ERR_NOT_SPD = 2,  /* a diagonal pivot was not > 0 (see d_info)     */
  MP_ERR_OOM = 3,      /* device or host allocation failed              */
  MP_ERR_CUDA = 4,     /* a CUDA runtime/driver call failed             */
  MP_ERR_TIMEOUT = 5,  /* a bounded device-side wait ran out            */
  MP_ERR_STATE = 6     /* call out of order (e.g. loglik before chol)   */
} mp_status;

/* Tile storage formats (Sec. 2 and 4.1: half/single/double; extended with
 * BF16 and OCP FP8 E4M3).  E4M3 tiles carry a power-of-two scale s chosen
 * per tile so that amax / s <= 448; a stored code c represents c * s. */
typedef enum { MP_F64 = 0, MP_F32 = 1, MP_BF16 = 2, MP_F16 = 3, MP_E4M3 = 4 } mp_dtype;

/* Matérn covariance parameters (Sec. 6.2): C(r) = sigma2 2^(1-nu) /
 * Gamma(nu) x^nu K_nu(x), x = r / range (K_nu the modified Bessel function
 * of the second kind; C(0) = sigma2), for 0 < nu <= 16: the half-integer
 * closed forms for nu in {0.5, 1.5, 2.5}, a Chebyshev table of x^nu K_nu(x)
 * (built on the host per nu, relative error about 1e-15) for any other nu.
 * `nugget` is added to the diagonal.  Other nu give MP_ERR_ARG. */
typedef struct {
  double sigma2;
  double range;
  double nu;
  double nugget;
} mp_matern;

typedef struct mp_ctx mp_ctx;
typedef struct mp_tmat mp_tmat;
typedef struct mp_batch mp_batch;

/* ---------------------------------------------------------------- context */

/* Creates a context on CUDA device `device` (made current for the calls
 * of this context).  *out receives the handle; free with mp_ctx_destroy. */
mp_status mp_ctx_create(int device, mp_ctx** out);
void mp_ctx_destroy(mp_ctx* ctx);

/* Static text for a status code. */
const char* mp_status_string(mp_status s);

/* Copies the last error message of `ctx` (NUL-terminated, truncated to
 * len) into buf.  Synchronous, host only. */
mp_status mp_last_error(mp_ctx* ctx, char* buf, size_t len);

/* Library build string (compiler, target architecture). */
const char* mp_version(void);

/* ------------------------------------------------------------ tiled matrix */

/* Creates an n x n symmetric tiled matrix with tile size b (a multiple of
 * 128, 128 <= b <= 1024) and NT = ceil(n / b) tiles per side.
 *   h_map   : NT*NT bytes, row-major, entry [i*NT + j] is the mp_dtype of
 *             tile (i, j); only the lower triangle i >= j is read; the
 *             diagonal must be MP_F64.  NULL means all MP_F64.
 *   flags   : MP_TMAT_KEEP_SIGMA keeps a copy of the generated lower
 *             tiles for the FP64 refinement residual, in 62-bit fixed
 *             point under one power of two (see mp_loglik; needs
 *             8 * NT(NT+1)/2 * b^2 more bytes).  MP_TMAT_SIMT_UPDATES runs
 *             the lower-precision trailing updates on CUDA cores (FP32
 *             FMA) instead of the tcgen05 tensor cores (BF16/FP16/E4M3
 *             MMAs; FP32 products as three TF32 products of hi/lo splits
 *             in two MMAs).
 *             MP_TMAT_STREAM_ALLOC allocates and frees the matrix's device
 *             memory with cudaMallocAsync / cudaFreeAsync on `stream` (and
 *             uploads with cudaMemcpyAsync), so that creating or destroying
 *             a matrix never waits for other streams' work.
 *             By default the panel solve of every panel tile stored in
 *             FP32 or below is the product X = A_ik W with W = L_kk^{-T}
 *             (FP64, formed with the diagonal tile's factorisation), on
 *             the tensor cores: both operands are split into 8 integer
 *             digits of 6 bits, every digit level accumulates exactly in
 *             FP32, and the levels are summed in float-float; the dropped
 *             levels bound the error by b (1 + 11/3) 2^-48 times the
 *             product of the row bound of A and the column bound of W,
 *             far below the FP32 rounding the result then receives.
 *             FP64-stored panel tiles keep the FP64 solve.
 *             MP_TMAT_FP64_PANEL solves every panel tile by FP64
 *             substitution instead.
 *             MP_TMAT_DIRECT: mp_chol and mp_loglik enqueue their kernels
 *             directly instead of capturing and replaying CUDA graphs, for
 *             matrices that are factored once (capturing and instantiating
 *             a graph of thousands of nodes costs more host time than its
 *             replay saves; the server uses it).  Same kernels, same bits.
 *             MP_TMAT_TRACE records the critical chain of the diagonal
 *             tiles' factorisations (mp_tmat_chain_trace).
 *             MP_TMAT_DAG16 / MP_TMAT_DAG32 / MP_TMAT_LOWP_RING4 are
 *             schedule choices (the autotuner's, see mp_tune_batch): they
 *             change speed, not the arithmetic of any product, but the
 *             task-graph block changes the summation order inside the
 *             diagonal tiles, so results agree to rounding, not bits.
 *             Accuracy of the two update paths: the tensor cores' FP32
 *             accumulation rounds toward zero, a bias of about 1e-6 of a
 *             K = 512 product per update (measured), which refinement does
 *             not remove from the log-determinant; MP_TMAT_SIMT_UPDATES
 *             accumulates with IEEE FP32 fused multiply-adds (the method's
 *             FP32 accumulation exactly, about 2.5x the factorisation time).
 *             Keep one path for all updates of a matrix: SYRK on one and
 *             GEMM on the other leaves a factor that FP64 refinement no
 *             longer converges with at n = 65536.
 *   stream  : stream all later calls on this matrix are ordered on.
 * The library allocates tile storage and workspace on the device (see
 * mp_tmat_info for the byte count).  Rows/columns n..NT*b-1 are padding
 * and hold the identity, which leaves the log-determinant and the
 * quadratic form unchanged.  Synchronous. */
#define MP_TMAT_KEEP_SIGMA 1u
#define MP_TMAT_SIMT_UPDATES 2u  /* trailing updates on CUDA cores instead of tcgen05 */
#define MP_TMAT_STREAM_ALLOC 4u  /* stream-ordered allocation on `stream` (no device sync) */
#define MP_TMAT_FP64_PANEL 8u    /* panel solves by FP64 substitution (default: integer-digit tcgen05 products) */
#define MP_TMAT_DAG16 32u        /* diagonal tile's task graph on 16 x 16 blocks (default: 16 for b in [384, 768], else 32) */
#define MP_TMAT_DAG32 64u        /* ... on 32 x 32 blocks */
#define MP_TMAT_LOWP_RING4 128u  /* 16-/8-bit tensor-core updates: 4-slot ring, 1 CTA per SM (default: 2-slot, 2 per SM) */
#define MP_TMAT_DIRECT 256u      /* mp_chol / mp_loglik launch directly instead of capturing CUDA graphs */
#define MP_TMAT_TRACE 512u       /* record the diagonal tiles' critical-chain stamps (mp_tmat_chain_trace) */
mp_status mp_tmat_create(mp_ctx* ctx, int64_t n, int32_t b, const uint8_t* h_map,
                         uint32_t flags, void* stream, mp_tmat** out);
void mp_tmat_destroy(mp_tmat* t);

/* Sizes of a tiled matrix: order, tile size, tiles per side, device bytes
 * held (tiles + workspace).  Any output pointer may be NULL.  Synchronous. */
mp_status mp_tmat_info(mp_tmat* t, int64_t* n, int32_t* b, int32_t* nt, int64_t* bytes);

/* Copies tile (i, j), i >= j, between the device and host memory: b*b
 * elements, row-major (element (r, c) at r*b + c), in the tile's storage
 * format (8/4/2/2/1 bytes); *scale is the E4M3 scale (1 otherwise).  For
 * diagonal tiles only the lower triangle is meaningful.  Synchronous
 * (waits for the matrix's stream).  Used to inspect factors and to load a
 * matrix that was not generated by mp_generate_matern (`as.MPCR`). */
mp_status mp_tile_get(mp_tmat* t, int32_t i, int32_t j, void* h_dst, double* scale);
mp_status mp_tile_set(mp_tmat* t, int32_t i, int32_t j, const void* h_src, double scale);

/* --------------------------------------------------------------- points */

/* Morton (Z-curve) order of n locations in [0,1]^2: d_locs_in is n x 2
 * row-major float64 (x, y per point); each coordinate is quantised to
 * q = min(floor(v * 65536), 65535) and the key interleaves x bits (even
 * positions) with y bits (odd positions); points are sorted by key, ties
 * by original index.  Writes d_locs_out (n x 2, may not alias d_locs_in)
 * and d_perm (n int64, d_locs_out[k] = d_locs_in[d_perm[k]]).  Uses a
 * device workspace owned by ctx.  Asynchronous on `stream`. */
mp_status mp_morton_order(mp_ctx* ctx, int64_t n, const double* d_locs_in,
                          double* d_locs_out, int64_t* d_perm, void* stream);

/* Allocation-free Morton ordering (no counterpart in the paper; it is a
 * service of this library).  Same result as mp_morton_order, but the sort
 * keys live in a fixed buffer inside the library's device image instead of
 * a cudaMalloc'd workspace, for callers that must not allocate device
 * memory: work enqueued during CUDA graph capture, latency-critical loops
 * that cannot absorb the allocator's implicit synchronisation, and
 * programs whose device memory belongs to another allocator or budget.
 *   - Runs on the calling thread's current device and on `stream`.
 *   - n must be in [1, MP_NOALLOC_MAX_POINTS]; larger n returns MP_ERR_ARG
 *     (use mp_morton_order).  The buffer (8 bytes per point of the limit,
 *     1 MiB) is held by every device that loads the library until exit.
 *   - The first call on a device looks the buffer's device address up
 *     (cudaGetSymbolAddress), and so does the first call after a
 *     cudaDeviceReset (the address belongs to the device's context); make
 *     that first call before any stream capture that includes this entry
 *     point.
 *   - A CUDA error already pending when the call starts is reported as
 *     MP_ERR_CUDA (and left pending) before anything is enqueued.
 *   - All calls share the one buffer: two calls whose work overlaps on the
 *     GPU (different streams, or different threads without ordering) race
 *     and corrupt each other's result; order them on one stream.
 *   - Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 * d_locs_in, d_locs_out, d_perm are as in mp_morton_order. */
#define MP_NOALLOC_MAX_POINTS 131072
mp_status mp_morton_order_noalloc(int64_t n, const double* d_locs_in, double* d_locs_out,
                                  int64_t* d_perm, void* stream);

/* ------------------------------------------------------------ generation */

/* Fills every lower tile with the Matérn covariance of the locations
 * d_locs (n x 2 row-major float64; borrowed until the generation kernels
 * have run on the matrix's stream).  With MP_TMAT_KEEP_SIGMA the values
 * are also kept, in fixed point, for the refinement residual.  Each entry
 * is computed to float64 accuracy (the closed forms in 64-bit fixed point,
 * within 0.55 + x/128 ulp of the exact value at the float64 squared
 * distance) and rounded once to its tile's format (RNE; E4M3 with
 * satfinite and a per-tile scale from the tile's amax).  Resets the
 * factorisation state.  Asynchronous. */
mp_status mp_generate_matern(mp_tmat* t, const double* d_locs, mp_matern p);

/* --------------------------------------------------------- factorisation */

/* Tiled right-looking Cholesky in place (Sec. 6.2 `chol`, tiled as in
 * Sec. 7): per step k, POTRF of the FP64 diagonal tile (with its inverse
 * W = L_kk^{-T}), the panel TRSM (integer-digit tensor-core products with W
 * by default, FP64 substitution with MP_TMAT_FP64_PANEL or for FP64-stored
 * panel tiles; the result rounded to each tile's format), and the trailing
 * SYRK/GEMM updates, each in the precision min(p(target), max(p(A),
 * p(B))) with FP32 accumulation (FP64 for FP64 products).  The whole
 * schedule is one CUDA graph launch on the matrix's stream.
 *   d_info   : 1 int64: 0, or the smallest 1-based global row whose pivot
 *              was not > 0 (then L is not valid), or -MP_ERR_TIMEOUT when a
 *              bounded device-side wait of a tensor-core kernel ran out
 *              (the kernel returned without hanging).  May be NULL.
 *   d_logdet : 1 float64: log det Sigma = 2 sum log L_tt.  May be NULL.
 * Returns MP_OK once enqueued (a non-SPD matrix is reported in d_info
 * only).  Asynchronous. */
mp_status mp_chol(mp_tmat* t, int64_t* d_info, double* d_logdet);

/* Runs only steps k0 .. k1-1 of the factorisation (0 <= k0 <= k1 <= NT),
 * with direct launches (no graph).  For inspecting the per-step kernels;
 * mp_chol is the same as mp_chol_steps(t, 0, NT) plus the outputs.
 * Asynchronous. */
mp_status mp_chol_steps(mp_tmat* t, int32_t k0, int32_t k1);

/* Budget of the bounded device-side waits of the task-graph kernels (the
 * diagonal tile's factorisation and the triangular solves): a wait gives up
 * after `polls` polls of about 64 ns each (0: the default, 2^21 polls,
 * about 0.1-0.3 s), sets the matrix's error word and its kernel returns;
 * mp_chol then reports -MP_ERR_TIMEOUT in d_info and mp_loglik writes NaN
 * log-likelihoods until the matrix is factored again.  A small budget makes
 * waits run out on purpose (failure handling can be tested without a
 * hung GPU).  Waits for the matrix's stream, drops its captured graphs
 * (recaptured at the next call).  Synchronous. */
mp_status mp_tmat_set_wait_budget(mp_tmat* t, int32_t polls);

/* The order in which the FP64 diagonal tile's task graph hands out its
 * tasks for nb = b / DB blocks (1 <= nb <= 64); host only, for checking
 * the schedule without a GPU.  4 bytes per task: op (0 factor (0, 0),
 * 1 solve (r, k), 2 update (r, c) with column k, 3 solve (k, k-1) +
 * update and factor (k, k), 4 solve of W block (c, r), 5 update of W block
 * (c, r) with column k), r, c, k.  *count = tasks; h_out (cap >= *count
 * tasks) may be NULL to query the count. */
mp_status mp_potrf_dag_schedule(int32_t nb, uint8_t* h_out, int64_t cap, int64_t* count);

/* The order in which a triangular solve's task graph hands out its tasks
 * for one matrix of nt tile rows split into p_blocks row blocks per tile
 * (b / 32); trans = 0 forward (L x = z), 1 backward (L^T x = z).  Host
 * only, for checking the schedule without a GPU.  One word per task: bits
 * 24-27 op (0 diagonal block: out_i[p] from in_i - chain_i; 1 update in
 * place: in_i[p] -= L_ij out_j, or L_ji^T out_j backward; 2 the same
 * product with the row j solved just before i, stored in chain_i[p]),
 * bits 28-39 i, 40-51 j, 52-59 p (bits 0-23: the matrix, 0 here).  *count = tasks; h_out (cap >= *count)
 * may be NULL to query the count. */
mp_status mp_solve_dag_schedule(int32_t nt, int32_t p_blocks, int32_t trans, uint64_t* h_out, int64_t cap,
                                int64_t* count);

/* Critical-chain stamps of the last factorisation of a matrix created with
 * MP_TMAT_TRACE (instrumentation, off by default; the arithmetic is the
 * same with it on).  The FP64 diagonal tile's task graph runs one chain
 * task per DB x DB diagonal block k (DB = *block, 16 or 32): factor block
 * (0, 0), or for k >= 1 solve block (k, k-1), update block (k, k) and
 * factor it (Sec. 6.2 `chol` in FP64, tile by tile as in Sec. 7).  Per
 * block, tile by tile (index (i * b / DB + k) * 16 for diagonal tile i),
 * 16 words: %globaltimer in ns, then clock64 of the same SM, at 8 points
 *   0 task taken, 1 its A blocks final, 2 the previous block's inverse
 *   ready, 3 block (k, k-1) solved and published, 4 block (k, k) updated,
 *   5 block (k, k) factored, 6 published, 7 task done.
 * When one CTA runs the chain (the default), point 1 is when that CTA had
 * loaded block k's inputs (during block k-1's factorisation, so before
 * point 0), points 0 and 2 coincide, and 5-7 coincide (the publication
 * runs beside the next block's work).
 * *count = words held (nt * b / DB * 16); h_out (cap >= *count words) may
 * be NULL to query the size.  Waits for the matrix's stream.
 * MP_ERR_STATE without MP_TMAT_TRACE. */
mp_status mp_tmat_chain_trace(mp_tmat* t, uint64_t* h_out, int64_t cap, int64_t* count, int32_t* block);

/* Copies log det Sigma of the factorised matrix into d_out (1 float64).
 * MP_ERR_STATE if mp_chol has not been enqueued.  Asynchronous. */
mp_status mp_logdet(mp_tmat* t, double* d_out);

/* In-place triangular solve with the factor, FP64 arithmetic on the
 * exactly upcast tiles (Sec. 6.2 `forwardsolve`, Sec. 5 `backsolve`):
 * trans = 0 solves L X = B, trans = 1 solves L^T X = B.  d_B is n x nrhs
 * column-major float64 with leading dimension ldb >= n.  Asynchronous. */
mp_status mp_trsm(mp_tmat* t, int trans, double* d_B, int64_t ldb, int32_t nrhs);

/* Solve with the factor, Sigma X = B (R's `solve` through the Cholesky
 * factor, Sec. 4.1's operation list): X = L^-T (L^-1 B) by two mp_trsm
 * calls, FP64 arithmetic on the exactly upcast tiles, no refinement (the
 * result carries the factor's lower-precision rounding; mp_loglik refines).
 * d_B: n x nrhs column-major, ld >= n, overwritten by X.  Right-hand sides
 * go through in chunks of 2048 (bounded workspace).  Waits for the
 * matrix's stream between chunks; asynchronous after the last. */
mp_status mp_solve(mp_tmat* t, double* d_B, int64_t ldb, int32_t nrhs);

/* Inverse from the factor, (L L^T)^-1 = L^-T L^-1 (R's `chol2inv`, Sec. 4.1):
 * d_out n x n column-major (ld >= n) receives the inverse of the matrix the
 * factor represents, column block by column block (identity columns solved
 * with mp_solve).  n^3 FP64 work; as mp_solve otherwise. */
mp_status mp_chol2inv(mp_tmat* t, double* d_out, int64_t ldo);

/* Gaussian log-likelihood (Sec. 6.2):
 *   loglik = -n/2 log(2 pi) - logdet/2 - quad/2
 * for each of nrhs right-hand sides z (d_z: n x nrhs column-major float64,
 * leading dimension ldz >= n).
 * refine_iters = 0: quad = ||L^{-1} z||^2.
 * refine_iters > 0: FP64 iterative refinement of Sigma x = z (the paper's
 *   "double precision for refinement", Sec. 1): x0 = L^-T L^-1 z, then up to
 *   refine_iters times r = z - Sigma x from the copy of Sigma kept by
 *   MP_TMAT_KEEP_SIGMA (MP_ERR_STATE without it, or when a tile was set by
 *   mp_tile_set after the last mp_generate_matern).  The copy holds each
 *   entry as a 62-bit integer below 2^E, 2^E the power of two above
 *   sigma^2 + nugget (within 2^(E-63) of the float64 entry); x is
 *   scaled to 54-bit integers per b-long segment, so the products and each
 *   tile's sums are exact, rounded to float64 once per tile and summed in
 *   float64 over the tiles of a row; a column stops when
 *   ||r||_inf <= n 2^-53 (||Sigma||_inf ||x||_inf + ||z||_inf), otherwise
 *   x += L^-T L^-1 r; quad = z^T x.
 * Outputs (device, may be NULL except d_ll): d_ll[nrhs] loglik,
 * d_quad[nrhs], d_iters[nrhs] corrections applied per column.
 * The solve and refinement schedule is captured into a CUDA graph and
 * re-used while the arguments stay the same.  Asynchronous. */
mp_status mp_loglik(mp_tmat* t, const double* d_z, int64_t ldz, int32_t nrhs,
                    int32_t refine_iters, double* d_ll, double* d_quad, int32_t* d_iters);

/* ------------------------------------------------------ planning, stats */

/* Frobenius norm of every lower tile of the Matérn matrix that
 * mp_generate_matern would produce for (n, b, d_locs, p), computed on the
 * device in float64 without storing the matrix: d_norms is NT*NT float64,
 * row-major, entry [i*NT + j] for i >= j (others set to 0).  Deterministic
 * (fixed reduction order).  Allocates a small scratch; synchronous. */
mp_status mp_tile_norms(mp_ctx* ctx, int64_t n, int32_t b, const double* d_locs, mp_matern p,
                        double* d_norms, void* stream);

/* The Matérn covariance C(r) of `p` (nugget not added) at count distances
 * h_r, into h_out; host only, the same method as the generation kernels
 * (closed forms or the per-nu Chebyshev table).  Synchronous. */
mp_status mp_matern_host(mp_matern p, int64_t count, const double* h_r, double* h_out);

/* Norm-guarded band precision map (host only).  The multi-precision tiled
 * extension (Sec. 7) leaves the choice of precisions open; this rule keeps
 * the diagonal in MP_F64, tiles with i - j <= band in near_dt, and gives a
 * farther tile far_dt only when u(far_dt) ||A_ij||_F <= eps ||A||_F / NT
 * (u = unit roundoff: 2^-24 F32, 2^-8 BF16, 2^-11 F16, 2^-4 E4M3), which
 * bounds the rounding perturbation of all far tiles by eps ||A||_F; the
 * others fall back to near_dt.  h_norms as written by mp_tile_norms;
 * h_map (NT*NT, row-major) receives the map, 255 above the diagonal. */
mp_status mp_map_guarded(int32_t nt, const double* h_norms, int32_t band, uint8_t near_dt,
                         uint8_t far_dt, double eps, uint8_t* h_map);

/* Kernel launches of one mp_chol (its graph's kernel nodes, known after the
 * first mp_chol), of one mp_generate_matern, and of one mp_loglik with the
 * arguments of its last call.  Any pointer may be NULL. */
mp_status mp_tmat_stats(mp_tmat* t, int64_t* chol_kernels, int64_t* gen_kernels,
                        int64_t* loglik_kernels);

/* Runs the factorisation once with direct launches and a CUDA event after
 * every launch, and returns per kernel class c (0 diagonal-tile task graph:
 * POTRF and W = L^{-T}, 1 panel TRSM, 2 panel rounding, 3 FP64 updates,
 * 4 CUDA-core lower-precision updates, 5 tensor-core updates of FP32 kind
 * (three TF32 products), 6 E4M3 target rounding, 7 other, 8 panel TRSM of
 * the first tile of each step (the lookahead chain's part), 9 integer-digit
 * panel products, 10 their digit splits, 11 tensor-core updates of 16- and
 * 8-bit kinds): h_ms[c] summed event time, h_launches[c] launches,
 * h_flops[c] algorithmic flops (diagonal tile 2b^3/3 for the factor and
 * its inverse, TRSM b^3 per tile, GEMM 2b^3, SYRK b^2(b+1)).  Arrays hold
 * nclass >= MP_PROFILE_CLASSES entries.  Leaves the matrix factored (as
 * mp_chol).  Synchronous. */
#define MP_PROFILE_CLASSES 12
mp_status mp_chol_profile(mp_tmat* t, int32_t nclass, float* h_ms, int64_t* h_launches,
                          double* h_flops);

/* Measures the device's FP64 FMA throughput (TFLOP/s) with a loop of
 * independent DFMA chains over every SM: the peak against which the FP64
 * kernels (panel TRSM, diagonal POTRF) are rated.  Synchronous. */
mp_status mp_probe_fp64_peak(int device, double* h_tflops);

/* ------------------------------------------------------------------ GEMM */

/* C = alpha op(A) op(B) + beta C (Sec. 5 `%*%` / `crossprod` per
 * precision), all three matrices stored in `dtype`, column-major with
 * leading dimensions; op(X) = X for 'N', X^T for 'T'.  op(A) is m x k,
 * op(B) is k x n, C is m x n.  Products accumulate in FP32 (FP64 for
 * MP_F64); alpha, beta and the final sum are applied in float64 for
 * MP_F64/MP_F32 targets and FP32 otherwise; the result is rounded once
 * to `dtype` (E4M3 codes with scale 1, satfinite).  BF16, FP16, E4M3 and
 * FP32 run on the tcgen05 tensor cores (FP32 as three TF32 products of
 * hi/lo splits): the operands are packed into K-major tiles of a stream-
 * ordered workspace (about (m + n) k element bytes, twice for FP32, plus
 * 4 m n), each 128 x 128 output block accumulates up to K = 4096 in tensor
 * memory (whose FP32 accumulation rounds toward zero), and blocks of K
 * are added with IEEE FP32 subtractions.  FP64 (and sizes beyond the
 * tile layout's limits) runs on the CUDA cores.  Asynchronous on
 * `stream`. */
mp_status mp_gemm(mp_ctx* ctx, mp_dtype dtype, char ta, char tb, int64_t m, int64_t n,
                  int64_t k, double alpha, const void* d_A, int64_t lda, const void* d_B,
                  int64_t ldb, double beta, void* d_C, int64_t ldc, void* stream);

/* ----------------------------------------------------------------- batch */

/* One log-likelihood request of a batch. */
typedef struct {
  int64_t n;              /* matrix order (>= 1)                             */
  const uint8_t* h_map;   /* NT*NT precision map as in mp_tmat_create, or NULL */
  const double* d_locs;   /* n x 2 row-major float64 locations (borrowed)     */
  const double* d_z;      /* n x nrhs column-major float64, ld = n (borrowed) */
  int32_t nrhs;           /* right-hand sides (>= 1)                          */
  int32_t refine_iters;   /* as in mp_loglik (0 = none)                       */
  mp_matern cov;          /* covariance parameters                            */
  /* Precision map by rule, used when h_map is NULL and rule_eps > 0: the
   * map of mp_map_bound(n, b, locations, cov, rule_band, rule_near,
   * rule_far, rule_eps) at the plan's own b (the locations are read back
   * from d_locs, which must then be in the order the matrix uses).  A map
   * by rule follows b; an explicit h_map fixes it.  rule_eps = 0 with
   * h_map NULL: all FP64. */
  int32_t rule_band;
  uint8_t rule_near, rule_far, rule_pad_[2];
  double rule_eps;
} mp_request;

/* Builds a batch plan for `count` independent requests sharing tile size b
 * (b = 0: the autotuner picks b and the schedule flags, see mp_tune_batch,
 * with its cache at the path in the environment variable MPCHOL_TUNE_CACHE
 * when set; the first call for a new kind of batch then times candidate
 * plans, several seconds): one tile
 * arena for all matrices and one merged schedule -- generation,
 * factorisation, solve, refinement and log-likelihood of every request --
 * captured as a single CUDA graph.  Panel solves follow mp_tmat_create's
 * default (integer-digit tensor-core products for tiles stored in FP32 or
 * below), so each request's result is bit-identical to its evaluation
 * alone.  Pointers in `reqs` are borrowed and must stay valid for the
 * plan's lifetime.  Synchronous. */
mp_status mp_batch_create(mp_ctx* ctx, int32_t count, const mp_request* reqs, int32_t b,
                          void* stream, mp_batch** out);
void mp_batch_destroy(mp_batch* batch);

/* mp_batch_create with explicit schedule flags: MP_TMAT_SIMT_UPDATES,
 * MP_TMAT_FP64_PANEL, MP_TMAT_DAG16 or MP_TMAT_DAG32, MP_TMAT_LOWP_RING4
 * (others give MP_ERR_ARG).  A request's result is bit-identical to its
 * evaluation by mp_tmat_create with the same b and flags.  Synchronous. */
mp_status mp_batch_create_ex(mp_ctx* ctx, int32_t count, const mp_request* reqs, int32_t b,
                             uint32_t flags, void* stream, mp_batch** out);

/* Schedule flags a batch plan was built with. */
mp_status mp_batch_flags(mp_batch* batch, uint32_t* flags);

/* ------------------------------------------------------------- autotuner */

/* A schedule chosen by the autotuner: tile size, schedule flags (as for
 * mp_tmat_create), the measured time of the workload it was chosen on,
 * whether it came from the cache, and how many candidates were timed. */
typedef struct {
  int32_t b;
  uint32_t flags;
  double ms;
  int32_t from_cache;
  int32_t tried;
} mp_tuned;

/* Autotuner of batch plans (the tiled extension of Sec. 7 leaves tile sizes
 * and schedules open; they are measured, not assumed).  Times whole batch
 * graphs of these very requests (one warm-up and the best of two launches,
 * CUDA events on `stream`) for candidate schedules, by coordinate descent
 * from b = 256 with the default flags: every b in {128, 256, 384, 512} up
 * to the largest request, then at the best b the other task-graph block,
 * the FP64 panel solve, the 4-slot ring of the 16-/8-bit updates.  The
 * fastest goes to *out.  cache_path (may be NULL: no cache) is a text file
 * of "key b flags ms" lines; the key names the GPU (name, SM count) and the
 * batch (request count, quartiles of n in steps of 256, share of tiles
 * stored below FP32 in steps of 1/10, right-hand sides); a matching line is
 * returned without timing, a new result is appended.  The requests'
 * pointers must be valid (their data are read).  Allocates and frees each
 * candidate plan; synchronous. */
mp_status mp_tune_batch(mp_ctx* ctx, int32_t count, const mp_request* reqs, const char* cache_path,
                        void* stream, mp_tuned* out);
/* (A request with an explicit h_map fixes b: then mp_tune_batch and
 * mp_batch_create with b = 0 give MP_ERR_ARG; give its map by rule.) */

/* Autotuner of single-matrix evaluations (the server's and the MLE
 * driver's): times one log-likelihood evaluation (generation, factorisation,
 * solve with `refine_iters` FP64 refinement sweeps) of an n-point synthetic
 * Matérn field (a jittered grid of the unit square, nu 3/2, range 0.05,
 * nugget 1e-4, precision map of mp_map_bound with band 2, FP32 near tiles,
 * far_dt where the bound allows it with eps) for b in {128, 256, 384, 512,
 * 1024} up to n and, at the best b, the other task-graph block and the
 * FP64 panel solve.  Cache as for mp_tune_batch (key: GPU, "tmat", n,
 * far_dt, eps, refine_iters).  Synchronous. */
mp_status mp_tune_tmat(mp_ctx* ctx, int64_t n, uint8_t far_dt, double eps, int32_t refine_iters,
                       const char* cache_path, void* stream, mp_tuned* out);

/* Device bytes held by a batch plan and the tile size it uses. */
mp_status mp_batch_info(mp_batch* batch, int64_t* bytes, int32_t* b);

/* Launches the batch graph.  d_ll: sum of nrhs over requests float64, the
 * log-likelihoods of request 0's columns first; d_status: count int32,
 * MP_OK or MP_ERR_NOT_SPD per request (a failing request does not stop the
 * others).  Asynchronous on the plan's stream. */
mp_status mp_batch_run(mp_batch* batch, double* d_ll, int32_t* d_status);

/* Same as mp_batch_create + mp_batch_run + a stream synchronisation.
 * Synchronous. */
mp_status mp_loglik_batch(mp_ctx* ctx, int32_t count, const mp_request* reqs,
                          double* d_ll, int32_t* d_status, void* stream);

/* --------------------------------------------------------------- serving */

/* Continuous-batching server of log-likelihood requests (an MLE search is
 * a stream of likelihood evaluations, Sec. 6.2).  Requests arrive with HOST
 * buffers and queue; mp_server_poll retires finished requests and admits
 * queued ones -- in arrival order, later ones backfilling when an earlier
 * one does not fit -- while one of `max_slots` streams is free and the
 * request's device footprint fits `hbm_budget` bytes.  Admitted requests
 * run concurrently, each on its own stream: locations are Morton-ordered
 * on the host, the precision map comes from mp_map_bound (diagonal FP64,
 * |i-j| <= 2 FP32, far tiles in `far_dt` where the norm bound allows it
 * with `eps`), and generation, factorisation and log-likelihood run on
 * the device; tile size 128 (n <= 2048), 256 (n <= 8192) or 512.  A
 * finished request keeps its factor on the device until released; when
 * a request needs the memory, the least recently finished unreleased
 * factors are evicted.  One thread drives a server. */
typedef struct mp_server mp_server;

typedef struct {
  int64_t id;
  int32_t status;       /* MP_OK, MP_ERR_NOT_SPD, MP_ERR_TIMEOUT, ...           */
  int32_t nrhs;
  int64_t n;
  int32_t b;
  int32_t low_tiles;    /* off-diagonal tiles stored in far_dt                 */
  int32_t offdiag_tiles;
  int32_t pad_;
  double t_submit, t_admit, t_done;   /* host clock (seconds)                 */
  double logdet;
  double loglik0;       /* log-likelihood of the first right-hand side         */
} mp_serve_result;

/* Creates a server (max_slots in [1, 64] streams).  Synchronous. */
mp_status mp_server_create(mp_ctx* ctx, int64_t hbm_budget, int32_t max_slots, double eps,
                           uint8_t far_dt, mp_server** out);
/* Waits for all work, frees everything. */
void mp_server_destroy(mp_server* s);

/* Queues a request: h_locs n x 2 row-major, h_z n x nrhs column-major (ld
 * n), both copied at the call; refine_iters as in mp_loglik.  *id is the
 * request's id (1, 2, ...).  Host only. */
mp_status mp_server_submit(mp_server* s, int64_t n, const double* h_locs, const double* h_z,
                           int32_t nrhs, int32_t refine_iters, mp_matern cov, int64_t* id);

/* Progress without blocking: writes up to max_out results of requests that
 * finished since the last poll (completion time = the poll that saw them)
 * and admits queued requests.  Call it in a loop. */
mp_status mp_server_poll(mp_server* s, mp_serve_result* out, int32_t max_out, int32_t* n_out);

/* Host copies of a finished request's log-likelihoods and quadratic forms
 * (nrhs each; either pointer may be NULL).  Returns the request's status
 * (MP_ERR_STATE while it has not finished). */
mp_status mp_server_result(mp_server* s, int64_t id, double* h_ll, double* h_quad);

/* The device factor a finished, not yet evicted request keeps (valid until
 * mp_server_release or eviction). */
mp_status mp_server_factor(mp_server* s, int64_t id, mp_tmat** t);

/* Frees a finished request's device memory. */
mp_status mp_server_release(mp_server* s, int64_t id);

/* Failure injection for the admission path: the next `count` admissions
 * fail their input allocation as if the device had no memory left (made on
 * the host; the request's tiled matrix already exists and is freed by the
 * failure path).  Those requests finish with MP_ERR_OOM; the others are
 * unaffected.  Host only. */
mp_status mp_server_inject_alloc_failures(mp_server* s, int32_t count);

/* Tunes the server's tile size and schedule for requests of the given
 * sizes with mp_tune_tmat (its far_dt and eps, refine_iters as given);
 * afterwards a request of order n takes the choice of the smallest tuned
 * size >= n (the largest beyond all), instead of the fixed rule (b = 128
 * up to n = 2048, 256 up to 8192, else 512).  cache_path as for
 * mp_tune_batch.  Synchronous; call before submitting requests. */
mp_status mp_server_tune(mp_server* s, const int64_t* sizes, int32_t count, int32_t refine_iters,
                         const char* cache_path);

/* Queue length, requests on the GPU, kept factors, device bytes in use. */
mp_status mp_server_stats(mp_server* s, int64_t* queued, int64_t* running, int64_t* kept,
                          int64_t* bytes_used);

/* Precision map from closed-form norm bounds (host only; the server's map).
 * h_sorted_locs: n x 2, already in the order the matrix will use.  As
 * mp_map_guarded, with ||A_ij||_F replaced by the upper bound
 * sqrt(rows_i cols_j) C(d_ij) (d_ij: distance between the bounding boxes
 * of the two tiles' points; C decreases with distance) and ||A||_F by the
 * lower bound sqrt(n) (sigma2 + nugget); both make the map more
 * conservative than the exact-norm rule.  h_map: NT*NT, 255 above the
 * diagonal. */
mp_status mp_map_bound(int64_t n, int32_t b, const double* h_sorted_locs, mp_matern c,
                       int32_t band, uint8_t near_dt, uint8_t far_dt, double eps, uint8_t* h_map);

#ifdef __cplusplus
}
#endif

#endif /* MPCHOL_H */
