// Internal types of the mpchol runtime: the tile arena, work items of every
// launch, and the host launchers each kernel file exports.
//
// A plan owns one arena: one device pool per storage format, each pool a
// stack of b x b row-major tiles.  A tile is named by an int32 id into the
// tile table (format, index in its pool).  Every kernel reads its work from
// a device array of items, so one launch can serve tiles of many matrices
// (the batched schedule) as well as one.
#pragma once

#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

namespace mp {

enum : int { F64 = 0, F32 = 1, BF16 = 2, F16 = 3, E4M3 = 4, NDT = 5 };

__host__ __device__ inline int esize(int dt) {
  return dt == F64 ? 8 : dt == F32 ? 4 : dt == E4M3 ? 1 : 2;
}
// precision rank of the update rule: F64 > F32 > 16-bit > E4M3
__host__ __device__ inline int level(int dt) {
  return dt == F64 ? 4 : dt == F32 ? 3 : dt == E4M3 ? 1 : 2;
}

struct TileRef {
  int32_t dt;
  int32_t idx;   // index in pool[dt]
};

// Device view of an arena, passed by value to kernels.
struct Arena {
  char* pool[NDT];
  const TileRef* tiles;           // tile table
  double* scale;                  // per tile: E4M3 scale (1 otherwise)
  unsigned long long* amax;       // per tile: amax as float64 bits (atomicMax)
  int* err;                       // set to 1 when a bounded device wait ran out
  int b;
  int wait_polls;                 // polls of a task-graph wait before it gives up (0: DAG_WAIT_LIMIT)
  // chain trace of the diagonal tiles' task graphs (NULL: off): per
  // diagonal block (log-determinant slot order) TRACE_WORDS stamps
  unsigned long long* trace;
};
constexpr int TRACE_WORDS = 16;   // 8 %globaltimer (ns) then 8 clock64 stamps per block

template <typename T>
__host__ __device__ inline T* tile_ptr(const Arena& A, int id) {
  TileRef r = A.tiles[id];
  return reinterpret_cast<T*>(A.pool[r.dt] + (int64_t)r.idx * A.b * A.b * esize(r.dt));
}
__host__ __device__ inline char* tile_bytes(const Arena& A, int id) {
  TileRef r = A.tiles[id];
  return A.pool[r.dt] + (int64_t)r.idx * A.b * A.b * esize(r.dt);
}

// ---- work items -----------------------------------------------------------

// Factorisation of one FP64 diagonal tile by a task graph over its NB x NB
// blocks, NB = 16 or 32 (k_potrf_dag); ver and the launch's ticket are zero
// when it starts.  One SM's FP64 pipe retires about two lane-FMAs per clock,
// so the block solve and update on the graph's critical chain cost NB^3 on
// a single SM while the chain of pivots (one per column) does not depend on
// NB: 16 keeps the chain short when few tiles share a launch, 32 has fewer
// tasks when many do.
struct ItemPotrf {
  int32_t tile;       // FP64 diagonal tile
  int32_t mat;        // matrix index (info word)
  int32_t ldslot;     // first of b/NB log-determinant partial slots
  int32_t pad_;
  int64_t row0;       // global row of the tile's first row
  double* dinv;       // b/NB inverses of the diagonal blocks (row-major)
  double* w;          // b x b: W = L^{-T} of the tile (upper triangular)
  float* whi;         // W as FP32 hi + lo pair (upper part only; NULL: not wanted)
  float* wlo;
  int32_t* ver;       // 2 (b/NB)^2 progress counters: factor blocks, then blocks of W
};
struct DagTask {
  uint8_t op;         // 0 factor (0, 0), 1 solve (r, k), 2 update (r, c), 3 solve (k, k-1) +
                      //   update and factor (k, k), 4 solve of W block (c, r), 5 update of
                      //   W block (c, r) with column k
  uint8_t r, c, k;
};

// Panel TRSM: X = A_ik L_kk^{-T} in float64 into a scratch slot.
struct ItemPanel {
  int32_t tile;       // A_ik
  int32_t diag;       // L_kk
  int32_t amax;       // amax slot of the result
  int32_t mat;        // matrix of the plan (host bookkeeping)
  const double* w;    // W = L_kk^{-T} (b x b); its diagonal 32-blocks are the
                      // transposed inverses of L_kk's diagonal 32-blocks
  double* x;          // b x b float64 scratch
};

// Rounds a panel scratch slot into its tile and its shadow copies (the tile
// rounded into each lower format a consumer's product runs in).
constexpr int MAX_SHADOW = 3;
struct ItemRound {
  int32_t tile;
  int32_t shadow[MAX_SHADOW];   // -1: unused
  int32_t hi, lo;               // FP32 tiles: value split as TF32 hi + remainder (-1: none)
  int32_t amax;                 // amax slot written by the panel solve
  int32_t pad_;
  const double* x;
};

// Trailing update C -= A B^T of one target tile.
struct ItemUpd {
  int32_t c, a, b;    // tile ids (a, b may be shadows already in the kind)
  int32_t syrk;       // 1: C is a diagonal tile (lower sub-blocks only)
  float* v;           // E4M3 target: b x b FP32 scratch for the new values
  int32_t vslot;      // E4M3 target: amax slot (index into Arena.amax)
  int32_t pad_;
};

// Tensor-core update of one target tile; for three-TF32 products a/a2 and
// b/b2 are the hi/lo splits of the operands.
struct ItemTC {
  int32_t c, a, b, a2, b2;
  int32_t syrk;
  int32_t vslot;
  int32_t kspan;      // contraction over tiles a .. a+kspan-1 with b .. b+kspan-1 (0, 1: one tile)
  float* v;
};

// Panel solve on the tensor cores (k_ozaki.cu): digit tiles of the rows of
// A_ik and of the columns of W = L_kk^{-T}.
constexpr int OZ_SMAX = 8;
struct ItemOzA {            // split of one panel tile's rows
  int32_t tile;
  int32_t slices[OZ_SMAX];  // BF16 digit tiles
  float* sigma;             // b row bounds
};
struct ItemOzW {            // split of W's columns (transposed digit tiles)
  int32_t wtile;            // FP64 tile holding W
  int32_t slices[OZ_SMAX];
  float* tau;               // b column bounds
};
struct ItemOz {             // X = A W for one panel tile
  int32_t a[OZ_SMAX];       // digit tiles of A
  int32_t w[OZ_SMAX];       // digit tiles of W^T
  int32_t amax;
  int32_t fuse;             // 1: round X into the tile, its shadows and TF32 splits here
  int32_t tile;             // (fuse) the panel tile
  int32_t shadow[MAX_SHADOW];
  int32_t hi, lo;
  int32_t s;                // digits per operand used (ozaki_digits of the tile's format)
  const float* sigma;
  const float* tau;
  double* x;                // b x b float64 result (when not fused)
};

// Digits per operand of the integer-digit panel product for a panel tile
// stored in format dt: the smallest S whose truncation bound
// b (1 + (S + 3) / 3) 2^(-6S) sigma_r tau_c, at b = 1024, sits 2^11 below
// half a unit in the last place of the format (FP32 8, BF16 and FP16 6,
// E4M3 5).
inline int ozaki_digits(int dt) {
  return dt == F32 ? 8 : (dt == BF16 || dt == F16) ? 6 : dt == E4M3 ? 5 : 8;
}

// Rounds an E4M3 target from its FP32 scratch with the new scale.
struct ItemFp8 {
  int32_t tile;
  int32_t vslot;
  const float* v;
};

// Generation of one lower tile.
struct ItemGen {
  int32_t tile;
  int32_t mat;
  int32_t ti, tj;     // tile coordinates
  const double* locs; // n x 2
  int64_t n;
  double sigma2, range, nu, nugget;
  // optional copy of Sigma for the refinement residual, b x b row-major, in
  // fixed point: round(Sigma 2^(62 - sig_e)) (every entry below 2^sig_e);
  // null: no copy.  The CTA of tile (0, 0) stores sig_e at *sig_e_out.
  uint64_t* sigfix;
  // nu without a closed form: the Matérn table of matern_nu_table (device
  // copy) and its first octave; null for nu in {1/2, 3/2, 5/2}
  const double* ktab;
  int32_t ke0;
  int32_t sig_e;
  int32_t* sig_e_out;
};

// Solve items.  Diagonal: tile = L_ii^{-T} (FP64), xj = X-product of xi
// (out of place).  Off-diagonal: tile = L tile, xi = solved segment,
// xj = segment still to be solved (updated in place).
// One matrix's triangular solve run by the solve task graph (k_solve_dag):
// forward out = L^{-1} in or backward out = L^{-T} in, `in` updated in
// place.  cnt holds nt (b/32 + 1) progress counters, zero at launch: per
// tile row i, the updates applied to each 32-row block, then the number of
// finished 32-row blocks of out_i.
struct ItemSolveDag {
  const int32_t* tiles;   // nt x nt tile ids of the factor (lower part)
  const int32_t* linv;    // nt tile ids of L_ii^{-T} (FP64, upper triangular), then nt ids
                          // of its FP32 hi parts and nt of its lo parts (ffdiag)
  double* in;             // N x nrhs (column stride ld), consumed
  double* out;            // N x nrhs (column stride ld)
  double* chain;          // N x nrhs (column stride ld): each tile row's update with the
                          // row solved just before it (kept apart, subtracted by the
                          // diagonal step)
  int* cnt;               // per tile row 2 P + 1 counters (P = b / 32): updates applied
                          // in place to each block, finished diagonal blocks, chain
                          // update of each block done
  int64_t ld;
  int32_t nt, nrhs;
  int32_t ffdiag;         // 1: diagonal steps in float-float from the hi/lo parts
  int32_t pad_;
};
// Task of the solve graph: matrix (bits 0-23), op (24-27: 0 diagonal block,
// 1 off-diagonal block applied in place, 2 off-diagonal block into the
// chain vector), target tile row i (28-39), source tile row j (40-51),
// 32-row block p (52-59).
typedef uint64_t SolveTask;

// Refinement residual r = z - Sigma x from the float64 copy of Sigma's lower
// tiles.  Pass 1, one item per lower tile (i, j): its row product
// Sigma_ij x_j into part(i, j) and, for i > j, its transposed product
// Sigma_ij^T x_i into part(j, i) (a diagonal tile's upper half is its lower
// half transposed), so every tile is read once.  Pass 2, one item per tile
// row i: r_i = z_i - sum_j part(i, j), j in increasing order.  part(i, j)
// holds b x nrhs doubles at ((i nt + j) nrhs + c) b; pabs the same for the
// absolute row sums (float, one column; NULL: not wanted).
struct ItemResTile {
  int32_t tile;       // tile of the fixed-point copy of Sigma
  int32_t ti, tj, nt;
  const double* x;    // N x nrhs (column stride ld)
  double* part;
  float* pabs;
  int64_t ld;
  int32_t nrhs, pad_;
  const int32_t* sig_e;   // the copy's exponent (written by the generation)
};
struct ItemResRow {
  int32_t ti, nt;
  const double* part;
  const float* pabs;
  const double* z;    // N x nrhs (column stride ld)
  double* r;          // N x nrhs (column stride ld)
  double* rowabs;     // N: sum_j |Sigma_ij| (NULL: not wanted)
  int64_t ld;
  int32_t nrhs, pad_;
};

// ---- host launchers (each .cu file exports its own) -----------------------

// k_gen.cu
void launch_morton_keys(const double* locs, int64_t n, int64_t n2, unsigned long long* keys,
                        cudaStream_t s);
void launch_bitonic(unsigned long long* keys, int64_t n2, cudaStream_t s);
void launch_morton_gather(const unsigned long long* keys, const double* in, int64_t n,
                          double* out, int64_t* perm, cudaStream_t s);
void launch_gen_amax(const Arena& A, const ItemGen* items, int count, cudaStream_t s);
void launch_generate(const Arena& A, const ItemGen* items, int count, cudaStream_t s);
// Uploads the generation kernels' e^{-x} tables to the current device; 0 on success.
int init_gen_tables();
// Matérn correlation for nu without a closed form (host side of the
// generation kernels): KNU_COEF Chebyshev coefficients per half octave
// [2^E, 1.5 2^E) and [1.5 2^E, 2^(E+1)), E = e0 .. KNU_EMAX - 1, of
// g(x) = 2^(1-nu) / Gamma(nu) x^nu K_nu(x) for x < 1 and of g(x) e^x for
// x >= 1; g(x) = 1 below 2^e0 and 0 from 2^KNU_EMAX on.
constexpr int KNU_COEF = 16;
constexpr int KNU_EMAX = 10;
constexpr double KNU_NU_MAX = 16.0;
bool matern_nu_closed(double nu);          // nu in {1/2, 3/2, 5/2}
bool matern_nu_valid(double nu);           // 0 < nu <= KNU_NU_MAX
// Builds the table (0 on success); e0 receives the first octave.
int matern_nu_table(double nu, std::vector<double>& coef, int* e0);
// g(x) e^{-x} ... the correlation at x = r / range from a host table.
double matern_nu_host(const double* coef, int e0, double x);
// Frobenius norm of every generated lower tile into norms[ti * nt + tj]
// (partial: count * b/16 doubles of scratch).
// partial sums per tile that launch_tile_norms writes (its `partial` holds
// count times this many doubles)
int tile_norm_parts(int b);
void launch_tile_norms(int b, const ItemGen* items, int count, int nt, double* partial,
                       double* norms, cudaStream_t s);

// k_fp64.cu
std::vector<DagTask> potrf_dag_tasks(int nb);
void launch_potrf_dag(const Arena& A, const ItemPotrf* items, int count, const DagTask* tasks,
                      int ntasks, int* ticket, double* ldparts, long long* info, int db,
                      cudaStream_t s);
// reserve_sms: SMs left free by the persistent grid (for concurrent work)
void launch_panel_trsm(const Arena& A, const ItemPanel* items, int count, int reserve_sms,
                       cudaStream_t s);
void launch_panel_round(const Arena& A, const ItemRound* items, int count, cudaStream_t s);

// k_update.cu
void launch_update_f32(const Arena& A, const ItemUpd* items, int count, cudaStream_t s);
void launch_update_f64(const Arena& A, const ItemUpd* items, int count, cudaStream_t s);
void launch_fp8_round(const Arena& A, const ItemFp8* items, int count, cudaStream_t s);

// k_ozaki.cu (8 digits per operand for every tile size up to 1024)
int oz_slices(int b);
void launch_oz_split_rows(const Arena& A, const ItemOzA* items, int count, cudaStream_t s);
void launch_oz_split_cols(const Arena& A, const ItemOzW* items, int count, cudaStream_t s);
void launch_oz_gemm(const Arena& A, const ItemOz* items, int count, const struct CUtensorMap_st& mapA,
                    const struct CUtensorMap_st& mapB64, const struct CUtensorMap_st& mapB32,
                    cudaStream_t s);

// k_tc.cu (kind: BF16, F16, E4M3, or F32 as three TF32 products; the map
// is a const CUtensorMap& of the operands' pool)
void launch_update_tc(const Arena& A, int kind, const ItemTC* items, int count,
                      const struct CUtensorMap_st& map, cudaStream_t s, bool ring4 = false);

// k_solve.cu  (a non-null `gate` pointing at 0 turns a launch into a no-op)
std::vector<SolveTask> solve_dag_tasks(const std::vector<int>& nts, int p_blocks, int trans);
void launch_solve_dag(const Arena& A, const ItemSolveDag* items, const SolveTask* tasks, int ntasks,
                      int* ticket, int trans, int nrhs_max, const int* gate, cudaStream_t s);
void launch_residual(const Arena& A, const ItemResTile* tiles, int ntiles, const ItemResRow* rows,
                     int nrows, int nrhs, int want_rowabs, const int* gate, cudaStream_t s);
void launch_logdet(const double* ldparts, const int32_t* ldoff, const int32_t* ldcnt, int nmat,
                   double* logdet, cudaStream_t s);
void launch_colmax(const double* v, int64_t n, int64_t ld, int nrhs, double* out,
                   const int* gate, cudaStream_t s);
void launch_refine_check(const double* rmax, const double* xmax, const double* zmax,
                         const double* snorm, int64_t n, int nrhs, int* active, int* iters,
                         int* any, const int* gate, cudaStream_t s);
void launch_axpy_active(double* x, const double* d, int64_t n, int64_t ld, int nrhs,
                        const int* active, const int* gate, cudaStream_t s);
void launch_copy_pad(const double* src, int64_t lds, double* dst, int64_t ldd, int64_t n,
                     int64_t N, int nrhs, const int* gate, cudaStream_t s);
void launch_dot(const double* a, const double* b, int64_t n, int64_t ld, int nrhs, double* out,
                cudaStream_t s);
void launch_loglik(const double* logdet, const double* quad, int64_t n, int nrhs, double* ll,
                   const int* err, cudaStream_t s);

// k_gemm.cu
// k_gemm_tc.cu: the same product on the tensor cores (0 ok, 1 no memory,
// 2 CUDA failure, 3 sizes beyond its tile layout: nothing enqueued)
int launch_gemm_tc(int dt, int ta, int tb, int64_t m, int64_t n, int64_t k, double alpha,
                   const void* A, int64_t lda, const void* B, int64_t ldb, double beta, void* C,
                   int64_t ldc, cudaStream_t s);
void launch_gemm(int dt, int ta, int tb, int64_t m, int64_t n, int64_t k, double alpha,
                 const void* A, int64_t lda, const void* B, int64_t ldb, double beta, void* C,
                 int64_t ldc, cudaStream_t s);

}  // namespace mp
