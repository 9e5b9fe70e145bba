// Host runtime behind include/mpchol.h: tile arenas, the static schedule of
// the tiled factorisation (merged over all matrices of a plan), solve and
// refinement schedules, and their capture into CUDA graphs.
//
// The schedule is the right-looking tiled Cholesky of the tiled
// multi-precision extension (Sec. 7) applied to the `chol` / `forwardsolve`
// recipe of Sec. 6.2.  Every step k is a fixed sequence of launches, each
// carrying the work items of every matrix that still has a step k:
//   amax reset, for each 32-block of the diagonal tile: POTRF block (+ inner
//   TRSM, inner SYRK), panel TRSM, panel rounding, trailing updates (FP64
//   products, lower-precision products), E4M3 target rounding.
// Because the whole schedule depends only on sizes and precision maps, it is
// built once per plan and replayed as one CUDA graph launch.
#include <algorithm>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <functional>
#include <vector>

#include <array>
#include <cuda.h>

#include "../../include/mpchol.h"
#include "mp_device.cuh"

using namespace mp;

struct mp_ctx {
  int device = 0;
  std::string err;
  unsigned long long* keys = nullptr;
  int64_t keys_cap = 0;
  std::mutex mu;
  // pinned host buffers lent to matrices for their uploads and taken back
  // when they are destroyed (freeing page-locked memory synchronises the
  // device, which a serving loop must not do per request)
  std::mutex pin_mu;
  std::vector<std::pair<char*, size_t>> pin_free;
};

namespace {
// Lends a pinned buffer of at least `bytes` (the smallest free one that
// fits, else a new one); nullptr if none can be had.
char* pin_borrow(mp_ctx* ctx, size_t bytes, size_t* cap) {
  {
    std::lock_guard<std::mutex> lk(ctx->pin_mu);
    size_t best = (size_t)-1;
    for (size_t k = 0; k < ctx->pin_free.size(); ++k)
      if (ctx->pin_free[k].second >= bytes && (best == (size_t)-1 || ctx->pin_free[k].second < ctx->pin_free[best].second))
        best = k;
    if (best != (size_t)-1) {
      auto e = ctx->pin_free[best];
      ctx->pin_free.erase(ctx->pin_free.begin() + best);
      *cap = e.second;
      return e.first;
    }
  }
  char* p = nullptr;
  if (cudaMallocHost((void**)&p, bytes) != cudaSuccess) return nullptr;
  *cap = bytes;
  return p;
}
void pin_return(mp_ctx* ctx, char* p, size_t cap) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(ctx->pin_mu);
  ctx->pin_free.push_back({p, cap});
}
}  // namespace

namespace {

thread_local char g_err_fallback[256];

mp_status fail(mp_ctx* ctx, mp_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  else snprintf(g_err_fallback, sizeof g_err_fallback, "%s", buf);
  return st;
}

}  // namespace

// Error text for calls that have no context (read by mp_last_error(NULL)).
namespace mp {
void set_error_text(const char* msg) { snprintf(g_err_fallback, sizeof g_err_fallback, "%s", msg); }
}  // namespace mp

namespace {

#define CK(ctx, call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return fail((ctx), MP_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                             \
  } while (0)

// R-MMA: precision of the product A_ik A_jk^T for a target of format q.
int kind_of(int q, int pa, int pb) {
  int lk = std::min(level(q), std::max(level(pa), level(pb)));
  if (lk == level(q)) return q;
  bool ha = level(pa) == lk, hb = level(pb) == lk;
  if (ha && hb && pa != pb) return F32;   // BF16 with F16 below a wider target
  return ha ? pa : pb;
}
// does an operand stored in format p need rounding to run in `kind`?
bool needs_round(int p, int kind) { return p != kind && level(p) >= level(kind); }

enum Op {
  OP_AMAX0, OP_INFO0, OP_POTRF_DAG, OP_PANEL, OP_ROUND, OP_UPD32, OP_UPD64, OP_TC,
  OP_REC, OP_WAIT, OP_AMAXR, OP_OZA, OP_OZW, OP_OZG,
  OP_FP8R, OP_LOGDET, OP_DIAG_F, OP_OFF_F, OP_DIAG_B, OP_OFF_B, OP_GEN_AMAX, OP_GEN
};

struct Launch {
  int op;
  size_t off;     // byte offset of the item array (OP_AMAXR: first amax slot)
  int count;      // items (OP_AMAXR: slots; OP_REC/OP_WAIT: event index)
  int kb;
  int stream = 0; // 0: the critical chain, 1: the bulk (lookahead)
};

}  // namespace

// One matrix inside a plan.
struct MatDesc {
  int64_t n = 0;
  int nt = 0;
  std::vector<int32_t> tile, sig;           // nt*nt each (-1 = none)
  std::vector<uint8_t> need;                // nt*nt: operand forms tile (i,j) must provide
                                            // (bit d: rounded copy in format d; bit 5:
                                            // TF32 hi/lo split)
  std::vector<int32_t> linv;                // nt: FP64 tile holding L_ii^{-T}
  std::vector<int32_t> linv_hi, linv_lo;    // nt each: its FP32 hi/lo parts (-1: all-FP64 matrix)
  bool mixed = false;                       // some tile stored below FP64
  int32_t ldoff = 0;
  double* dinv = nullptr;                   // nt * (b/dag_nb) blocks of dag_nb x dag_nb
};

struct Plan {
  mp_ctx* ctx = nullptr;
  int b = 0;
  cudaStream_t stream = nullptr;   // user stream
  cudaStream_t cap = nullptr;      // internal stream for graph capture (chain)
  cudaStream_t cap2 = nullptr;     // second capture stream (bulk work)
  std::vector<cudaEvent_t> events; // dependencies between the two streams
  int64_t pslots = 0;              // panel slots per step parity
  int64_t amax_panel0 = 0, amax_v0 = 0, amax_dummy = 0;
  bool keep_sigma = false;
  // arena
  std::vector<TileRef> h_tiles;
  int pool_count[NDT] = {};
  int dag_nb = 32;                 // block of the diagonal-tile task graph (16 or 32)
  int dag_nb_req = 0;              // requested block (0: chosen by b)
  bool lowp_ring4 = false;         // 16-/8-bit tensor-core updates: 4-slot ring, one CTA per SM
  bool no_graph = false;           // factorisation and solves launched directly (no capture)
  int wait_polls = 0;              // task-graph wait budget (0: the kernels' default)
  bool trace = false;              // record the diagonal tiles' chain stamps
  unsigned long long* d_trace = nullptr;
  int64_t trace_words = 0;
  int* d_dag = nullptr;            // diagonal-tile task graph: ticket, then per matrix 2 (b/dag_nb)^2 counters
  int32_t* d_ltab = nullptr;       // per matrix: nt*nt factor tile ids, then nt ids of L_ii^{-T}
  std::vector<int64_t> ltab_off;
  int* d_scnt = nullptr;           // solve task graph: ticket, then per matrix nt (2 b/32 + 1) counters
  size_t scnt_bytes = 0;
  std::vector<int64_t> scnt_off;
  size_t dag_bytes = 0;
  size_t dag_tasks_off = 0;        // task list (items buffer offset)
  int dag_ntasks = 0;
  bool use_tc = true;              // tensor-core updates (else CUDA cores)
  bool ozaki = false;              // panel solve on the tensor cores (integer digits)
  int oz_s = 0;                    // digits per operand
  std::vector<std::array<int32_t, OZ_SMAX>> slot_oz;   // digit tiles per panel slot
  std::vector<std::array<int32_t, OZ_SMAX>> wdig;      // digit tiles of W, per parity x matrix
  float* d_sigma = nullptr;        // row bounds per panel slot (b each)
  float* d_tau = nullptr;          // column bounds per parity x matrix (b each)
  CUtensorMap tmap_bf16_64;        // BF16 pool, box 128 bytes x 64 rows (digit products)
  CUtensorMap tmap_bf16_32;        // BF16 pool, box 128 bytes x 32 rows (single-tile digit products)
  // operand forms of the panel tiles, per panel slot of a step
  std::vector<std::array<int32_t, NDT>> slot_shadow;
  std::vector<int32_t> slot_hi, slot_lo;
  CUtensorMap tmap[NDT];
  bool have_tmap[NDT] = {};
  int* d_err = nullptr;
  char* pool[NDT] = {};
  TileRef* d_tiles = nullptr;
  double* d_scale = nullptr;
  unsigned long long* d_amax = nullptr;
  int n_amax = 0;
  // matrices
  std::vector<MatDesc> mats;
  double* d_dinv_all = nullptr;
  double* d_ldparts = nullptr;
  int32_t* d_ldoff = nullptr;
  int32_t* d_ldcnt = nullptr;
  long long* d_info = nullptr;
  double* d_logdet = nullptr;
  double* d_panel = nullptr;        // panel scratch slots (float64)
  float* d_v = nullptr;             // E4M3 update scratch slots (FP32)
  int32_t* d_sig = nullptr;         // sigma tile tables (all matrices)
  // work items and schedules
  std::vector<char> h_items;
  char* d_items = nullptr;
  size_t d_items_cap = 0;
  std::vector<Launch> chol;          // full factorisation
  std::vector<size_t> step_begin;    // index into chol of each step's first launch
  std::vector<int64_t> first_split;  // per step: launch splitting its first panel tiles' digits
                                     // (issued by the previous step's bulk), or -1
  cudaGraphExec_t chol_exec = nullptr;
  int64_t chol_kernels = 0;
  bool factored = false;
  int64_t bytes = 0;
  std::vector<void*> allocs;
  bool stream_alloc = false;       // cudaMallocAsync / cudaFreeAsync on `stream`

  Arena arena() const {
    Arena A{};
    for (int d = 0; d < NDT; ++d) A.pool[d] = pool[d];
    A.tiles = d_tiles;
    A.scale = d_scale;
    A.amax = d_amax;
    A.err = d_err;
    A.b = b;
    A.wait_polls = wait_polls;
    A.trace = d_trace;
    return A;
  }

  template <typename T>
  size_t push(const std::vector<T>& v) {
    size_t off = (h_items.size() + 255) & ~size_t(255);
    h_items.resize(off + v.size() * sizeof(T));
    if (!v.empty()) memcpy(h_items.data() + off, v.data(), v.size() * sizeof(T));
    return off;
  }
  template <typename T>
  const T* item(size_t off) const { return reinterpret_cast<const T*>(d_items + off); }

  cudaError_t raw_alloc(void** p, size_t bytes_) {
    return stream_alloc ? cudaMallocAsync(p, bytes_, stream) : cudaMalloc(p, bytes_);
  }
  void raw_free(void* p) {
    if (!p) return;
    if (stream_alloc) cudaFreeAsync(p, stream);
    else cudaFree(p);
  }
  // Host-to-device copies are ordered on the plan's stream: the kernels that
  // read them run there, and a plain cudaMemcpy (legacy stream) is not
  // ordered with a non-blocking stream -- from pageable memory it returns
  // once the data is staged, and a kernel on such a stream could still read
  // the previous contents.  A pageable source is staged before the call
  // returns, so the host buffer may be freed right after.
  cudaError_t upload(void* dst, const void* src, size_t bytes_) {
    return cudaMemcpyAsync(dst, src, bytes_, cudaMemcpyHostToDevice, stream);
  }
  mp_status alloc(void** p, size_t bytes_) {
    if (bytes_ == 0) { *p = nullptr; return MP_OK; }
    cudaError_t e = raw_alloc(p, bytes_);
    if (e != cudaSuccess) return fail(ctx, MP_ERR_OOM, "cudaMalloc(%zu): %s", bytes_, cudaGetErrorString(e));
    allocs.push_back(*p);
    bytes += (int64_t)bytes_;
    return MP_OK;
  }

  ~Plan() {
    if (chol_exec) cudaGraphExecDestroy(chol_exec);
    for (auto e : events) cudaEventDestroy(e);
    if (cap2) cudaStreamDestroy(cap2);
    for (void* p : allocs) raw_free(p);
    if (d_items) raw_free(d_items);
    if (cap) cudaStreamDestroy(cap);
  }
};

// Single-matrix handle: a plan with one matrix plus solve state.
struct mp_tmat {
  Plan P;
  const double* locs = nullptr;
  mp_matern cov{};
  bool generated = false;
  // generation items (re-built when the inputs change)
  std::vector<char> gen_key;
  size_t gen_off_amax = 0, gen_off_all = 0;
  int gen_n_amax = 0, gen_n_all = 0;
  char* d_gen = nullptr;
  size_t d_gen_cap = 0;
  // Matérn table for nu without a closed form (device), the nu it holds
  double* d_ktab = nullptr;
  size_t d_ktab_cap = 0;
  double ktab_nu = 0.0;
  int ktab_e0 = 0;
  // exponent of the fixed-point copy of Sigma (device, set by the
  // generation); whether the copy holds the matrix (no mp_tile_set since)
  int32_t* d_sig_e = nullptr;
  bool sig_valid = false;
  // loglik workspace + graph
  int ws_nrhs = 0;
  double *zp = nullptr, *x = nullptr, *r = nullptr, *w = nullptr, *d = nullptr;
  double* c = nullptr;              // the solves' chain products (scratch)
  double *rowabs = nullptr, *red = nullptr;
  double* rpart = nullptr;          // residual partial products: nt * nt * b * nrhs
  float* rpabs = nullptr;           // residual partial absolute sums: nt * nt * b
  int *active = nullptr, *iters = nullptr, *any = nullptr;
  cudaGraphExec_t ll_exec = nullptr;
  int64_t ll_kernels = 0;
  std::vector<char> ll_key;
  char* d_sitems = nullptr;
  size_t d_sitems_cap = 0;
  // pinned staging of the solve items: a copy from pageable memory waits
  // for the stream (here: for the factorisation just enqueued)
  char* h_pin = nullptr;
  size_t h_pin_cap = 0;
  cudaEvent_t pin_ev = nullptr;
  bool pin_used = false;
  std::vector<void*> ws_allocs;
  ~mp_tmat() {
    if (ll_exec) cudaGraphExecDestroy(ll_exec);
    for (void* p : ws_allocs) P.raw_free(p);
    P.raw_free(d_gen);
    P.raw_free(d_sitems);
    P.raw_free(d_ktab);
    P.raw_free(d_sig_e);
    if (pin_ev) { if (pin_used) cudaEventSynchronize(pin_ev); cudaEventDestroy(pin_ev); }
    pin_return(P.ctx, h_pin, h_pin_cap);
  }
};

struct mp_batch {
  Plan P;
  int count = 0;
  uint32_t flags = 0;
  std::vector<mp_request> reqs;
  cudaGraphExec_t exec = nullptr;
  double* d_llbuf = nullptr;    // internal outputs
  int32_t* d_stbuf = nullptr;
  int total_rhs = 0;
  ~mp_batch() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

namespace {

// ------------------------------------------------------------ plan building

mp_status validate_map(mp_ctx* ctx, int nt, const uint8_t* map) {
  if (!map) return MP_OK;
  for (int i = 0; i < nt; ++i) {
    if (map[i * nt + i] != F64) return fail(ctx, MP_ERR_ARG, "diagonal tile %d must be MP_F64", i);
    for (int j = 0; j < i; ++j)
      if (map[i * nt + j] >= NDT) return fail(ctx, MP_ERR_ARG, "tile (%d,%d): bad dtype %d", i, j, map[i * nt + j]);
  }
  return MP_OK;
}

int new_tile(Plan& P, int dt) {
  TileRef r{dt, P.pool_count[dt]++};
  P.h_tiles.push_back(r);
  return (int)P.h_tiles.size() - 1;
}

// Lays out the tiles of one matrix (and its shadows / float64 Sigma copy).
mp_status add_matrix(Plan& P, int64_t n, const uint8_t* map) {
  MatDesc M;
  M.n = n;
  if ((n + P.b - 1) / P.b > 4095) return fail(P.ctx, MP_ERR_ARG, "at most 4095 tiles per side");
  M.nt = (int)((n + P.b - 1) / P.b);
  const int nt = M.nt;
  if (mp_status st = validate_map(P.ctx, nt, map)) return st;
  auto dt = [&](int i, int j) { return map ? (int)map[i * nt + j] : (int)F64; };
  M.tile.assign((size_t)nt * nt, -1);
  M.need.assign((size_t)nt * nt, 0);
  for (int i = 0; i < nt; ++i)
    for (int j = 0; j <= i; ++j) M.tile[i * nt + j] = new_tile(P, dt(i, j));
  // operand forms needed by each off-diagonal tile (i, s): a rounded copy
  // per format in which a product that reads it runs below its storage
  // format, and the TF32 split when a tensor-core FP32 product reads it
  for (int s = 0; s < nt; ++s)
    for (int i = s + 1; i < nt; ++i) {
      const int p = dt(i, s);
      uint8_t need = 0;
      auto use = [&](int kd) {
        if (needs_round(p, kd)) need |= (uint8_t)(1u << kd);
        if (P.use_tc && kd == F32) need |= 1u << 5;
      };
      for (int j = s + 1; j <= i; ++j) use(kind_of(dt(i, j), p, dt(j, s)));     // as A
      for (int i2 = i + 1; i2 < nt; ++i2) use(kind_of(dt(i2, i), dt(i2, s), p)); // as B
      int cnt = 0;
      for (int d = 0; d < NDT; ++d) cnt += (need >> d) & 1;
      if (cnt > MAX_SHADOW) return fail(P.ctx, MP_ERR_ARG, "tile (%d,%d) needs too many rounded copies", i, s);
      M.need[(size_t)i * nt + s] = need;
    }
  M.linv.assign(nt, -1);
  for (int i = 0; i < nt; ++i) M.linv[i] = new_tile(P, F64);
  for (int i = 0; i < nt; ++i)
    for (int j = 0; j <= i; ++j) M.mixed |= dt(i, j) != F64;
  M.linv_hi.assign(nt, -1);
  M.linv_lo.assign(nt, -1);
  if (M.mixed)
    for (int i = 0; i < nt; ++i) {
      M.linv_hi[i] = new_tile(P, F32);
      M.linv_lo[i] = new_tile(P, F32);
    }
  if (P.keep_sigma) {
    M.sig.assign((size_t)nt * nt, -1);
    for (int i = 0; i < nt; ++i)
      for (int j = 0; j <= i; ++j) M.sig[i * nt + j] = new_tile(P, F64);
  }
  P.mats.push_back(std::move(M));
  return MP_OK;
}

// Builds the factorisation schedule of every matrix in the plan, merged by
// step index, as two streams with lookahead:
//   chain (stream 0): POTRF(k); the panel solve of the first tile (k+1, k)
//     and its rounding; the SYRK of (k+1, k+1);
//   bulk (stream 1):  the rest of panel k (and L_kk^{-T}) and its rounding;
//     the updates of column k+1 below the diagonal; all other updates.
// Events order them: POTRF(k) after the bulk of step k-2; the first panel
// tile after the column-(k) updates of step k-1; the SYRK of (k+1, k+1)
// after the bulk of step k-1; the bulk of step k after POTRF(k) and, for
// its column updates, after the first tile.  Panel scratch, operand copies
// and panel amax slots alternate between two sets by step parity, so the
// chain of step k+1 never touches what the bulk of step k reads.
void build_chol_schedule(Plan& P, int64_t* panel_slots, int64_t* v_slots) {
  const int b = P.b, nbb = b / P.dag_nb;
  int maxnt = 0;
  for (auto& M : P.mats) maxnt = std::max(maxnt, M.nt);
  int64_t max_v = 0;
  P.chol.clear();
  P.step_begin.clear();
  P.first_split.assign(maxnt + 1, -1);
  {
    const std::vector<DagTask> tasks = potrf_dag_tasks(nbb);
    P.dag_tasks_off = P.push(tasks);
    P.dag_ntasks = (int)tasks.size();
  }
  P.chol.push_back({OP_INFO0, 0, 0, 0, 0});
  auto ev = [](int s, int which) { return 4 * s + which; };   // 0 potrf 1 first 2 col 3 rest
  auto add = [&](int op, size_t off, int count, int kb, int stream) {
    P.chol.push_back({op, off, count, kb, stream});
  };
  auto rec = [&](int e, int st) { add(OP_REC, 0, e, 0, st); };
  auto wait = [&](int e, int st) { add(OP_WAIT, 0, e, 0, st); };
  auto amax_reset = [&](int64_t first, int64_t n, int st) {
    if (n > 0) add(OP_AMAXR, (size_t)first, (int)n, 0, st);
  };
  for (int s = 0; s < maxnt; ++s) {
    P.step_begin.push_back(P.chol.size());
    const int par = s & 1;
    const int64_t slot0 = par * P.pslots;
    // ---------------- chain: POTRF(s)
    if (s >= 2) wait(ev(s - 2, 3), 0);
    {
      std::vector<ItemPotrf> items;
      for (int m = 0; m < (int)P.mats.size(); ++m) {
        auto& M = P.mats[m];
        if (M.nt <= s) continue;
        ItemPotrf it{};
        it.tile = M.tile[s * M.nt + s];
        it.mat = m;
        it.ldslot = M.ldoff + s * nbb;
        it.row0 = (int64_t)s * b;
        it.dinv = M.dinv + (int64_t)s * nbb * P.dag_nb * P.dag_nb;
        it.w = (double*)(P.pool[F64] + (size_t)P.h_tiles[M.linv[s]].idx * b * b * 8);
        if (M.mixed) {
          it.whi = (float*)(P.pool[F32] + (size_t)P.h_tiles[M.linv_hi[s]].idx * b * b * 4);
          it.wlo = (float*)(P.pool[F32] + (size_t)P.h_tiles[M.linv_lo[s]].idx * b * b * 4);
        }
        it.ver = P.d_dag + 32 + (int64_t)m * 2 * nbb * nbb;
        items.push_back(it);
      }
      add(OP_POTRF_DAG, P.push(items), (int)items.size(), 0, 0);
    }
    // Ozaki mode: digits of W = L_ss^{-T} (formed by the POTRF graph), used
    // by the first tile's product here and by the rest of the panel
    if (P.ozaki) {
      std::vector<ItemOzW> ozw;
      for (int m = 0; m < (int)P.mats.size(); ++m) {
        auto& M = P.mats[m];
        bool any = false;
        for (int i = s + 1; i < M.nt; ++i) any |= P.h_tiles[M.tile[i * M.nt + s]].dt != F64;
        if (!any) continue;
        ItemOzW w{};
        w.wtile = M.linv[s];
        for (int d = 0; d < OZ_SMAX; ++d) w.slices[d] = P.wdig[par * P.mats.size() + m][d];
        w.tau = P.d_tau + (par * P.mats.size() + m) * (int64_t)b;
        ozw.push_back(w);
      }
      if (!ozw.empty()) add(OP_OZW, P.push(ozw), (int)ozw.size(), 0, 0);
    }
    rec(ev(s, 0), 0);
    // slot of panel tile (i, s) of matrix m: first tiles first, then the rest
    std::vector<int64_t> first_slot(P.mats.size(), -1), rest_base(P.mats.size(), 0);
    int64_t nfirst = 0, nrest = 0;
    for (int m = 0; m < (int)P.mats.size(); ++m) {
      if (P.mats[m].nt > s + 1) first_slot[m] = nfirst++;
    }
    for (int m = 0; m < (int)P.mats.size(); ++m) {
      rest_base[m] = nfirst + nrest;
      if (P.mats[m].nt > s + 2) nrest += P.mats[m].nt - s - 2;
    }
    auto slot_of = [&](int m, int i) {
      return slot0 + (i == s + 1 ? first_slot[m] : rest_base[m] + (i - s - 2));
    };
    auto form = [&](int m, int i, int d) { return P.slot_shadow[slot_of(m, i)][d]; };
    auto panel_items = [&](int m, int i, std::vector<ItemPanel>& panel, std::vector<ItemRound>& round) {
      auto& M = P.mats[m];
      const int nt = M.nt;
      const int64_t q = slot_of(m, i);
      ItemPanel it{};
      it.tile = M.tile[i * nt + s];
      it.diag = M.tile[s * nt + s];
      it.mat = m;
      it.amax = (int)(P.amax_panel0 + q);
      it.w = (const double*)(P.pool[F64] + (size_t)P.h_tiles[M.linv[s]].idx * b * b * 8);
      it.x = P.d_panel + q * (int64_t)b * b;
      panel.push_back(it);
      ItemRound r{};
      r.tile = it.tile;
      for (int d = 0; d < MAX_SHADOW; ++d) r.shadow[d] = -1;
      const uint8_t need = M.need[(size_t)i * nt + s];
      int c = 0;
      for (int d = 0; d < NDT; ++d)
        if ((need >> d) & 1) r.shadow[c++] = form(m, i, d);
      r.hi = (need & (1u << 5)) ? P.slot_hi[q] : -1;
      r.lo = (need & (1u << 5)) ? P.slot_lo[q] : -1;
      r.amax = it.amax;
      r.x = it.x;
      round.push_back(r);
    };
    // update items of targets (i, j) with operands from column s
    int64_t vslot = 0;
    struct Group {
      std::vector<ItemUpd> u32, u64;
      std::vector<ItemTC> tc[NDT];
      std::vector<ItemFp8> f8;
    };
    auto add_update = [&](Group& g, int m, int i, int j) {
      auto& M = P.mats[m];
      const int nt = M.nt;
      const int tc_ = M.tile[i * nt + j], ta = M.tile[i * nt + s], tb = M.tile[j * nt + s];
      const int q = P.h_tiles[tc_].dt, pa = P.h_tiles[ta].dt, pb = P.h_tiles[tb].dt;
      const int kd = kind_of(q, pa, pb);
      float* v = nullptr;
      int vs = -1;
      if (q == E4M3) {
        v = P.d_v + vslot * (int64_t)b * b;
        vs = (int)(P.amax_v0 + vslot);
        g.f8.push_back(ItemFp8{tc_, vs, v});
        ++vslot;
      }
      const bool tc_ok = P.use_tc;
      if (kd == F64) {
        g.u64.push_back(ItemUpd{tc_, ta, tb, i == j, v, vs, 0});
      } else if (tc_ok && kd == F32) {
        ItemTC u{};
        u.c = tc_;
        u.a = P.slot_hi[slot_of(m, i)];
        u.a2 = P.slot_lo[slot_of(m, i)];
        u.b = P.slot_hi[slot_of(m, j)];
        u.b2 = P.slot_lo[slot_of(m, j)];
        u.syrk = i == j;
        u.vslot = vs;
        u.v = v;
        g.tc[F32].push_back(u);
      } else {
        const int a = needs_round(pa, kd) ? form(m, i, kd) : ta;
        const int bb = needs_round(pb, kd) ? form(m, j, kd) : tb;
        if (tc_ok) {
          ItemTC u{};
          u.c = tc_;
          u.a = a;
          u.b = bb;
          u.a2 = u.b2 = -1;
          u.syrk = i == j;
          u.vslot = vs;
          u.v = v;
          g.tc[kd].push_back(u);
        } else {
          g.u32.push_back(ItemUpd{tc_, a, bb, i == j, v, vs, 0});
        }
      }
    };
    auto emit = [&](Group& g, int st) {
      if (!g.u64.empty()) add(OP_UPD64, P.push(g.u64), (int)g.u64.size(), 0, st);
      if (!g.u32.empty()) add(OP_UPD32, P.push(g.u32), (int)g.u32.size(), 0, st);
      for (int d : {F32, BF16, F16, E4M3})
        if (!g.tc[d].empty()) add(OP_TC, P.push(g.tc[d]), (int)g.tc[d].size(), d, st);
      if (!g.f8.empty()) add(OP_FP8R, P.push(g.f8), (int)g.f8.size(), 0, st);
    };
    // panel tiles stored in FP32 or below take X = A W on the tensor cores
    // (Ozaki mode); the others keep the FP64 solve
    auto split_panel = [&](std::vector<ItemPanel>& panel, std::vector<ItemRound>& round,
                           std::vector<ItemOzA>& oza, std::vector<ItemOz>& ozg) {
      if (!P.ozaki) return;
      std::vector<ItemPanel> native;
      std::vector<ItemRound> rest_round;
      for (size_t k = 0; k < panel.size(); ++k) {
        const ItemPanel& it = panel[k];
        const ItemRound& rd = round[k];
        if (P.h_tiles[it.tile].dt == F64) {
          native.push_back(it);
          rest_round.push_back(rd);
          continue;
        }
        const int64_t q = (it.x - P.d_panel) / ((int64_t)b * b);
        const int m = it.mat;
        ItemOzA a{};
        a.tile = it.tile;
        for (int d = 0; d < OZ_SMAX; ++d) a.slices[d] = P.slot_oz[q][d];
        a.sigma = P.d_sigma + q * b;
        oza.push_back(a);
        ItemOz g{};
        for (int d = 0; d < OZ_SMAX; ++d) { g.a[d] = P.slot_oz[q][d]; g.w[d] = P.wdig[par * P.mats.size() + m][d]; }
        g.amax = it.amax;
        g.sigma = a.sigma;
        g.tau = P.d_tau + (par * P.mats.size() + m) * (int64_t)b;
        g.x = it.x;
        // rounding fused into the product unless an E4M3 scale (from the
        // tile's amax) is involved
        bool e4 = P.h_tiles[it.tile].dt == E4M3;
        for (int d = 0; d < MAX_SHADOW; ++d) e4 |= rd.shadow[d] >= 0 && P.h_tiles[rd.shadow[d]].dt == E4M3;
        g.fuse = e4 ? 0 : 1;
        g.tile = it.tile;
        for (int d = 0; d < MAX_SHADOW; ++d) g.shadow[d] = rd.shadow[d];
        g.hi = rd.hi;
        g.lo = rd.lo;
        g.s = ozaki_digits(P.h_tiles[it.tile].dt);
        ozg.push_back(g);
        if (e4) rest_round.push_back(rd);
      }
      panel.swap(native);
      round.swap(rest_round);
    };
    auto emit_panel = [&](std::vector<ItemPanel>& panel, std::vector<ItemRound>& round, int st,
                          bool split_done) {
      std::vector<ItemOzA> oza;
      std::vector<ItemOz> ozg;
      split_panel(panel, round, oza, ozg);
      if (!oza.empty() && !split_done) add(OP_OZA, P.push(oza), (int)oza.size(), 0, st);
      if (!panel.empty()) add(OP_PANEL, P.push(panel), (int)panel.size(), 0, st);
      if (!ozg.empty()) add(OP_OZG, P.push(ozg), (int)ozg.size(), 0, st);
      if (!round.empty()) add(OP_ROUND, P.push(round), (int)round.size(), 0, st);
    };
    // ---------------- chain: first panel tile, its rounding, SYRK (s+1, s+1)
    {
      std::vector<ItemPanel> panel;
      std::vector<ItemRound> round;
      Group syrk;
      for (int m = 0; m < (int)P.mats.size(); ++m)
        if (P.mats[m].nt > s + 1) panel_items(m, s + 1, panel, round);
      if (s >= 1) wait(ev(s - 1, 2), 0);
      amax_reset(P.amax_panel0 + slot0, nfirst, 0);
      // from step 1 on, the bulk of the previous step split this tile's rows
      // right after finishing it
      emit_panel(panel, round, 0, P.ozaki && s >= 1);
      rec(ev(s, 1), 0);
      for (int m = 0; m < (int)P.mats.size(); ++m)
        if (P.mats[m].nt > s + 1) add_update(syrk, m, s + 1, s + 1);
      if (s >= 1) wait(ev(s - 1, 3), 0);
      emit(syrk, 0);
    }
    // ---------------- bulk: rest of the panel, column s+1, rest
    {
      std::vector<ItemPanel> panel;
      std::vector<ItemRound> round;
      for (int m = 0; m < (int)P.mats.size(); ++m)
        for (int i = s + 2; i < P.mats[m].nt; ++i) panel_items(m, i, panel, round);
      wait(ev(s, 0), 1);
      amax_reset(P.amax_panel0 + slot0 + nfirst, nrest, 1);
      emit_panel(panel, round, 1, false);
      Group col, rest;
      for (int m = 0; m < (int)P.mats.size(); ++m)
        for (int i = s + 2; i < P.mats[m].nt; ++i) add_update(col, m, i, s + 1);
      for (int m = 0; m < (int)P.mats.size(); ++m)
        for (int j = s + 2; j < P.mats[m].nt; ++j)
          for (int i = j; i < P.mats[m].nt; ++i) add_update(rest, m, i, j);
      wait(ev(s, 1), 1);
      amax_reset(P.amax_v0, vslot, 1);
      emit(col, 1);
      // Ozaki mode: digits of the next step's first panel tiles (s+2, s+1),
      // final after these column updates, split here off the critical chain
      if (P.ozaki) {
        const int64_t nslot0 = ((s + 1) & 1) * P.pslots;
        std::vector<ItemOzA> nxt;
        int64_t nf = 0;
        for (int m = 0; m < (int)P.mats.size(); ++m) {
          auto& M = P.mats[m];
          if (M.nt <= s + 2) continue;
          const int64_t q = nslot0 + nf++;
          const int tile = M.tile[(s + 2) * M.nt + s + 1];
          if (P.h_tiles[tile].dt == F64) continue;
          ItemOzA a{};
          a.tile = tile;
          for (int d = 0; d < OZ_SMAX; ++d) a.slices[d] = P.slot_oz[q][d];
          a.sigma = P.d_sigma + q * b;
          nxt.push_back(a);
        }
        if (!nxt.empty()) {
          P.first_split[s + 1] = (int64_t)P.chol.size();
          add(OP_OZA, P.push(nxt), (int)nxt.size(), 0, 1);
        }
      }
      rec(ev(s, 2), 1);
      emit(rest, 1);
      rec(ev(s, 3), 1);
    }
    max_v = std::max(max_v, vslot);
  }
  P.step_begin.push_back(P.chol.size());
  wait(ev(maxnt - 1, 3), 0);
  add(OP_LOGDET, 0, (int)P.mats.size(), 0, 0);
  *panel_slots = P.pslots;
  *v_slots = max_v;
}

// Counts scratch needs without item pointers (first pass), so that scratch
// can be allocated before the items that point into it are built.
void count_scratch(const Plan& P, int64_t* panel_slots, int64_t* v_slots) {
  int maxnt = 0;
  for (auto& M : P.mats) maxnt = std::max(maxnt, M.nt);
  int64_t mp_ = 0, mv = 0;
  for (int s = 0; s < maxnt; ++s) {
    int64_t slot = 0, vslot = 0;
    for (auto& M : P.mats) {
      if (M.nt <= s) continue;
      slot += M.nt - 1 - s;
      for (int j = s + 1; j < M.nt; ++j)
        for (int i = j; i < M.nt; ++i)
          if (P.h_tiles[M.tile[i * M.nt + j]].dt == E4M3) ++vslot;
    }
    mp_ = std::max(mp_, slot);
    mv = std::max(mv, vslot);
  }
  *panel_slots = mp_;
  *v_slots = mv;
}

mp_status upload_items(Plan& P) {
  if (P.h_items.size() > P.d_items_cap) {
    P.raw_free(P.d_items);
    P.d_items = nullptr;
    CK(P.ctx, P.raw_alloc((void**)&P.d_items, P.h_items.size()));
    P.d_items_cap = P.h_items.size();
  }
  if (!P.h_items.empty()) CK(P.ctx, P.upload(P.d_items, P.h_items.data(), P.h_items.size()));
  return MP_OK;
}

// One 2-D tensor map per format pool that tensor-core products read: the
// pool seen as a (tiles * b) x b row-major matrix, box 128 bytes x 128 rows,
// 128-byte swizzle (the K-major operand layout of the MMA descriptors).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

mp_status make_tensor_maps(Plan& P) {
  static EncodeTiledFn encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return fail(P.ctx, MP_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    encode = (EncodeTiledFn)fn;
  }
  const int b = P.b;
  for (int d : {F32, BF16, F16, E4M3}) {
    if (P.pool_count[d] == 0) continue;
    CUtensorMapDataType ty = d == F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                           : d == BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                           : d == F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                      : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    const int es = esize(d);
    cuuint64_t dims[2] = {(cuuint64_t)b, (cuuint64_t)P.pool_count[d] * b};
    cuuint64_t strides[1] = {(cuuint64_t)b * es};
    cuuint32_t box[2] = {(cuuint32_t)(128 / es), 128};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(&P.tmap[d], ty, 2, P.pool[d], dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(P.ctx, MP_ERR_CUDA, "tensor map of pool %d: error %d", d, (int)r);
    P.have_tmap[d] = true;
    if (d == BF16) {
      cuuint32_t box64[2] = {(cuuint32_t)(128 / es), 64};
      r = encode(&P.tmap_bf16_64, ty, 2, P.pool[d], dims, strides, box64, estr,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return fail(P.ctx, MP_ERR_CUDA, "tensor map (64 rows): error %d", (int)r);
      cuuint32_t box32[2] = {(cuuint32_t)(128 / es), 32};
      r = encode(&P.tmap_bf16_32, ty, 2, P.pool[d], dims, strides, box32, estr,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return fail(P.ctx, MP_ERR_CUDA, "tensor map (32 rows): error %d", (int)r);
    }
  }
  return MP_OK;
}

// Allocates the arena and scratch of a plan whose matrices were added.
mp_status finish_plan(Plan& P) {
  // the block of the diagonal tile's task graph depends on b alone (a batch
  // and a single matrix of the same b factor bit-identically): 16-blocks
  // shorten the critical chain; at b = 1024 they make 91k tasks per tile and
  // at b <= 256 the chain is short anyway, so those keep 32-blocks
  P.dag_nb = P.dag_nb_req ? P.dag_nb_req : (P.b >= 384 && P.b <= 768) ? 16 : 32;
  const int b = P.b, nbb = b / 32, ndb = b / P.dag_nb;
  {
    int64_t panel_slots = 0, v_slots = 0;
    count_scratch(P, &panel_slots, &v_slots);
    P.pslots = panel_slots;
    uint8_t all = 0;
    for (auto& M : P.mats)
      for (uint8_t v : M.need) all |= v;
    const int64_t nslot = 2 * panel_slots;            // two sets: step parity
    P.slot_shadow.assign(nslot, {});
    P.slot_hi.assign(nslot, -1);
    P.slot_lo.assign(nslot, -1);
    for (int64_t q = 0; q < nslot; ++q) {
      for (int d = 0; d < NDT; ++d) P.slot_shadow[q][d] = (all >> d) & 1 ? new_tile(P, d) : -1;
      if (all & (1u << 5)) {
        P.slot_hi[q] = new_tile(P, F32);
        P.slot_lo[q] = new_tile(P, F32);
      }
    }
    if (P.ozaki) {
      P.oz_s = oz_slices(b);
      P.slot_oz.assign(nslot, {});
      for (int64_t q = 0; q < nslot; ++q)
        for (int d = 0; d < OZ_SMAX; ++d) P.slot_oz[q][d] = d < P.oz_s ? new_tile(P, BF16) : -1;
      P.wdig.assign(2 * P.mats.size(), {});
      for (auto& w : P.wdig)
        for (int d = 0; d < OZ_SMAX; ++d) w[d] = d < P.oz_s ? new_tile(P, BF16) : -1;
    }
  }
  for (int d = 0; d < NDT; ++d) {
    void* p = nullptr;
    size_t bytes = (size_t)P.pool_count[d] * b * b * esize(d);
    if (mp_status st = P.alloc(&p, bytes)) return st;
    P.pool[d] = (char*)p;
    // zero once: the blocks of W = L^{-T} below its diagonal are never
    // written (the factorisation writes W's diagonal and upper blocks only)
    if (d == F64 && bytes) CK(P.ctx, cudaMemsetAsync(p, 0, bytes, P.stream));
  }
  int64_t panel_slots = 0, v_slots = 0;
  count_scratch(P, &panel_slots, &v_slots);
  void* p;
  if (mp_status st = P.alloc(&p, (size_t)2 * panel_slots * b * b * 8)) return st;
  P.d_panel = (double*)p;
  if (P.ozaki) {
    if (mp_status st = P.alloc(&p, sizeof(float) * (size_t)2 * std::max<int64_t>(panel_slots, 1) * b)) return st;
    P.d_sigma = (float*)p;
    if (mp_status st = P.alloc(&p, sizeof(float) * 2 * P.mats.size() * b)) return st;
    P.d_tau = (float*)p;
  }
  if (mp_status st = P.alloc(&p, (size_t)v_slots * b * b * 4)) return st;
  P.d_v = (float*)p;
  const int ntiles = (int)P.h_tiles.size();
  P.amax_panel0 = ntiles;
  P.amax_v0 = ntiles + 2 * panel_slots;
  P.amax_dummy = P.amax_v0 + v_slots;
  P.n_amax = (int)(P.amax_dummy + 1);
  if (mp_status st = P.alloc(&p, sizeof(TileRef) * ntiles)) return st;
  P.d_tiles = (TileRef*)p;
  if (mp_status st = P.alloc(&p, sizeof(double) * ntiles)) return st;
  P.d_scale = (double*)p;
  if (mp_status st = P.alloc(&p, sizeof(unsigned long long) * P.n_amax)) return st;
  P.d_amax = (unsigned long long*)p;
  // per-matrix: block inverses, log-det partials
  int64_t ninv = 0;
  int32_t ldo = 0;
  std::vector<int32_t> ldoff, ldcnt;
  for (auto& M : P.mats) {
    M.ldoff = ldo;
    ldoff.push_back(ldo);
    ldcnt.push_back(M.nt * ndb);
    ldo += M.nt * ndb;
    ninv += (int64_t)M.nt * ndb;
  }
  if (mp_status st = P.alloc(&p, sizeof(double) * P.dag_nb * P.dag_nb * ninv)) return st;
  P.d_dinv_all = (double*)p;
  int64_t io = 0;
  for (auto& M : P.mats) {
    M.dinv = P.d_dinv_all + io * P.dag_nb * P.dag_nb;
    io += (int64_t)M.nt * ndb;
  }
  const int nm = (int)P.mats.size();
  if (mp_status st = P.alloc(&p, sizeof(double) * std::max(ldo, 1))) return st;
  P.d_ldparts = (double*)p;
  if (P.trace) {
    P.trace_words = (int64_t)std::max(ldo, 1) * TRACE_WORDS;
    if (mp_status st = P.alloc(&p, sizeof(unsigned long long) * P.trace_words)) return st;
    P.d_trace = (unsigned long long*)p;
    CK(P.ctx, cudaMemsetAsync(P.d_trace, 0, sizeof(unsigned long long) * P.trace_words, P.stream));
  }
  if (mp_status st = P.alloc(&p, sizeof(int32_t) * nm)) return st;
  P.d_ldoff = (int32_t*)p;
  if (mp_status st = P.alloc(&p, sizeof(int32_t) * nm)) return st;
  P.d_ldcnt = (int32_t*)p;
  if (mp_status st = P.alloc(&p, sizeof(long long) * nm)) return st;
  P.d_info = (long long*)p;
  if (mp_status st = P.alloc(&p, sizeof(double) * nm)) return st;
  P.d_logdet = (double*)p;
  if (mp_status st = P.alloc(&p, sizeof(int))) return st;
  P.d_err = (int*)p;
  P.dag_bytes = sizeof(int) * (32 + (size_t)nm * 2 * ndb * ndb);
  if (mp_status st = P.alloc(&p, P.dag_bytes)) return st;
  P.d_dag = (int*)p;
  {
    std::vector<int32_t> ltab;
    size_t cnt = 32;
    for (auto& M : P.mats) {
      P.ltab_off.push_back((int64_t)ltab.size());
      ltab.insert(ltab.end(), M.tile.begin(), M.tile.end());
      ltab.insert(ltab.end(), M.linv.begin(), M.linv.end());
      ltab.insert(ltab.end(), M.linv_hi.begin(), M.linv_hi.end());
      ltab.insert(ltab.end(), M.linv_lo.begin(), M.linv_lo.end());
      P.scnt_off.push_back((int64_t)cnt);
      cnt += (size_t)M.nt * (2 * nbb + 1);
    }
    if (mp_status st = P.alloc(&p, sizeof(int32_t) * ltab.size())) return st;
    P.d_ltab = (int32_t*)p;
    CK(P.ctx, P.upload(P.d_ltab, ltab.data(), sizeof(int32_t) * ltab.size()));
    P.scnt_bytes = sizeof(int) * cnt;
    if (mp_status st = P.alloc(&p, P.scnt_bytes)) return st;
    P.d_scnt = (int*)p;
  }
  CK(P.ctx, cudaMemsetAsync(P.d_err, 0, sizeof(int), P.stream));
  if (P.use_tc || P.ozaki) {
    if (mp_status st = make_tensor_maps(P)) return st;
  }
  if (P.keep_sigma) {
    int64_t tot = 0;
    for (auto& M : P.mats) tot += (int64_t)M.nt * M.nt;
    if (mp_status st = P.alloc(&p, sizeof(int32_t) * tot)) return st;
    P.d_sig = (int32_t*)p;
    int64_t o = 0;
    for (auto& M : P.mats) {
      CK(P.ctx, P.upload(P.d_sig + o, M.sig.data(), sizeof(int32_t) * M.sig.size()));
      o += (int64_t)M.nt * M.nt;
    }
  }
  CK(P.ctx, P.upload(P.d_tiles, P.h_tiles.data(), sizeof(TileRef) * ntiles));
  std::vector<double> ones(ntiles, 1.0);
  CK(P.ctx, P.upload(P.d_scale, ones.data(), sizeof(double) * ntiles));
  CK(P.ctx, P.upload(P.d_ldoff, ldoff.data(), sizeof(int32_t) * nm));
  CK(P.ctx, P.upload(P.d_ldcnt, ldcnt.data(), sizeof(int32_t) * nm));
  int64_t ps = 0, vs = 0;
  build_chol_schedule(P, &ps, &vs);
  if (mp_status st = upload_items(P)) return st;
  P.bytes += (int64_t)P.h_items.size();
  // the critical chain gets the highest stream priority, the bulk the lowest
  int lo_pri = 0, hi_pri = 0;
  CK(P.ctx, cudaDeviceGetStreamPriorityRange(&lo_pri, &hi_pri));
  CK(P.ctx, cudaStreamCreateWithPriority(&P.cap, cudaStreamNonBlocking, hi_pri));
  CK(P.ctx, cudaStreamCreateWithPriority(&P.cap2, cudaStreamNonBlocking, lo_pri));
  int maxnt = 0;
  for (auto& M : P.mats) maxnt = std::max(maxnt, M.nt);
  P.events.resize(4 * maxnt + 4);     // last four: chain fork/join, direct-launch fork/join
  for (auto& e : P.events) CK(P.ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  // the uploads above are ordered on the plan's stream; creation stays
  // synchronous unless the plan allocates stream-ordered
  if (!P.stream_alloc) CK(P.ctx, cudaStreamSynchronize(P.stream));
  return MP_OK;
}


// Runs one entry of a schedule.  With s2 == nullptr everything goes to s in
// list order (a valid sequential order) and event entries are skipped.
void run_launch(const Plan& P, const Launch& L, cudaStream_t s0, cudaStream_t s2 = nullptr) {
  const Arena A = P.arena();
  cudaStream_t s = (s2 && L.stream == 1) ? s2 : s0;
  switch (L.op) {
    case OP_OZA: launch_oz_split_rows(A, P.item<ItemOzA>(L.off), L.count, s); break;
    case OP_OZW: launch_oz_split_cols(A, P.item<ItemOzW>(L.off), L.count, s); break;
    case OP_OZG:
      launch_oz_gemm(A, P.item<ItemOz>(L.off), L.count, P.tmap[BF16], P.tmap_bf16_64, P.tmap_bf16_32, s);
      break;
    case OP_REC: if (s2) cudaEventRecord(P.events[L.count], s); break;
    case OP_WAIT: if (s2) cudaStreamWaitEvent(s, P.events[L.count], 0); break;
    case OP_AMAXR:
      cudaMemsetAsync(P.d_amax + L.off, 0, sizeof(unsigned long long) * L.count, s);
      break;
    case OP_INFO0:
      cudaMemsetAsync(P.d_info, 0x7f, sizeof(long long) * P.mats.size(), s);
      cudaMemsetAsync(P.d_err, 0, sizeof(int), s);
      break;
    case OP_AMAX0: cudaMemsetAsync(P.d_amax, 0, sizeof(unsigned long long) * P.n_amax, s); break;
    case OP_POTRF_DAG:
      cudaMemsetAsync(P.d_dag, 0, P.dag_bytes, s);
      launch_potrf_dag(A, P.item<ItemPotrf>(L.off), L.count, P.item<DagTask>(P.dag_tasks_off),
                       P.dag_ntasks, P.d_dag, P.d_ldparts, P.d_info, P.dag_nb, s);
      break;
    case OP_PANEL:
      // the bulk panel leaves SMs free for the chain running beside it
      launch_panel_trsm(A, P.item<ItemPanel>(L.off), L.count, (s2 && L.stream == 1) ? 16 : 0, s);
      break;
    case OP_ROUND: launch_panel_round(A, P.item<ItemRound>(L.off), L.count, s); break;
    case OP_UPD32: launch_update_f32(A, P.item<ItemUpd>(L.off), L.count, s); break;
    case OP_UPD64: launch_update_f64(A, P.item<ItemUpd>(L.off), L.count, s); break;
    case OP_TC: {
      // FP32 products read the TF32 splits from the FP32 pool; the others
      // read their own format's pool
      launch_update_tc(A, L.kb, P.item<ItemTC>(L.off), L.count, P.tmap[L.kb], s, P.lowp_ring4);
      break;
    }
    case OP_FP8R: launch_fp8_round(A, P.item<ItemFp8>(L.off), L.count, s); break;
    case OP_LOGDET:
      launch_logdet(P.d_ldparts, P.d_ldoff, P.d_ldcnt, (int)P.mats.size(), P.d_logdet, s);
      break;
    default: break;
  }
}

// Enqueues the factorisation schedule on `s` with the bulk work forked to
// the plan's second stream (inside a graph capture: two graph branches).
void run_chol_forked(const Plan& P, cudaStream_t s);

// Direct launches (no graph) with the same two-stream structure: the
// chain on the high-priority stream, the bulk on the low-priority one,
// ordered after and before the work of the plan's stream.
void run_chol_direct(const Plan& P) {
  cudaEvent_t fork = P.events[P.events.size() - 4], join = P.events[P.events.size() - 3];
  cudaEventRecord(fork, P.stream);
  cudaStreamWaitEvent(P.cap, fork, 0);
  run_chol_forked(P, P.cap);
  cudaEventRecord(join, P.cap);
  cudaStreamWaitEvent(P.stream, join, 0);
}

void run_chol_forked(const Plan& P, cudaStream_t s) {
  cudaEvent_t fork = P.events[P.events.size() - 2], join = P.events.back();
  cudaEventRecord(fork, s);
  cudaStreamWaitEvent(P.cap2, fork, 0);
  for (const Launch& L : P.chol) run_launch(P, L, s, P.cap2);
  cudaEventRecord(join, P.cap2);
  cudaStreamWaitEvent(s, join, 0);
}

}  // namespace

namespace {

template <typename F>
mp_status capture_graph(mp_ctx* ctx, cudaStream_t cap, F&& body, cudaGraphExec_t* exec,
                        int64_t* kernel_nodes = nullptr) {
  cudaGraph_t g = nullptr;
  CK(ctx, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
  body(cap);
  cudaError_t e = cudaStreamEndCapture(cap, &g);
  if (e != cudaSuccess) return fail(ctx, MP_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  if (kernel_nodes) {
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
    int64_t k = 0;
    for (auto nd : nodes) {
      cudaGraphNodeType ty;
      if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++k;
    }
    *kernel_nodes = k;
  }
  if (*exec) { cudaGraphExecDestroy(*exec); *exec = nullptr; }
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(ctx, MP_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  return MP_OK;
}

// Launches `exec` on the user stream; the capture stream is independent.
mp_status launch_graph(mp_ctx* ctx, cudaGraphExec_t exec, cudaStream_t s) {
  CK(ctx, cudaGraphLaunch(exec, s));
  return MP_OK;
}

mp_status check_launch(mp_ctx* ctx) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, MP_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
  return MP_OK;
}

}  // namespace

// ================================================================== C ABI ==

extern "C" {

const char* mp_status_string(mp_status s) {
  switch (s) {
    case MP_OK: return "ok";
    case MP_ERR_ARG: return "invalid argument";
    case MP_ERR_NOT_SPD: return "matrix is not positive definite";
    case MP_ERR_OOM: return "out of memory";
    case MP_ERR_CUDA: return "CUDA error";
    case MP_ERR_TIMEOUT: return "device wait timed out";
    case MP_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

const char* mp_version(void) {
#define MP_STR2(x) #x
#define MP_STR(x) MP_STR2(x)
  return "mpchol 0.1 (sm_103a, nvcc " MP_STR(__CUDACC_VER_MAJOR__) "." MP_STR(__CUDACC_VER_MINOR__) ")";
}

mp_status mp_ctx_create(int device, mp_ctx** out) {
  if (!out) return fail(nullptr, MP_ERR_ARG, "out is null");
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n)
    return fail(nullptr, MP_ERR_ARG, "no CUDA device %d", device);
  CK(nullptr, cudaSetDevice(device));
  if (init_gen_tables() != 0) return fail(nullptr, MP_ERR_CUDA, "cannot set the generation tables");
  mp_ctx* c = new mp_ctx;
  c->device = device;
  *out = c;
  return MP_OK;
}

void mp_ctx_destroy(mp_ctx* ctx) {
  if (!ctx) return;
  if (ctx->keys) cudaFree(ctx->keys);
  for (auto& e : ctx->pin_free) cudaFreeHost(e.first);
  delete ctx;
}

mp_status mp_last_error(mp_ctx* ctx, char* buf, size_t len) {
  if (!buf || len == 0) return MP_ERR_ARG;
  snprintf(buf, len, "%s", ctx ? ctx->err.c_str() : g_err_fallback);
  return MP_OK;
}

mp_status mp_tmat_create(mp_ctx* ctx, int64_t n, int32_t b, const uint8_t* h_map, uint32_t flags,
                         void* stream, mp_tmat** out) {
  if (!ctx || !out) return fail(ctx, MP_ERR_ARG, "null argument");
  if (n < 1) return fail(ctx, MP_ERR_ARG, "n must be >= 1");
  if (b < 128 || b > 1024 || b % 128) return fail(ctx, MP_ERR_ARG, "b must be a multiple of 128 in [128, 1024]");
  CK(ctx, cudaSetDevice(ctx->device));
  mp_tmat* t = new mp_tmat;
  t->P.ctx = ctx;
  t->P.b = b;
  t->P.stream = (cudaStream_t)stream;
  t->P.keep_sigma = (flags & MP_TMAT_KEEP_SIGMA) != 0;
  t->P.use_tc = (flags & MP_TMAT_SIMT_UPDATES) == 0;
  t->P.ozaki = (flags & MP_TMAT_FP64_PANEL) == 0;
  t->P.stream_alloc = (flags & MP_TMAT_STREAM_ALLOC) != 0;
  if ((flags & MP_TMAT_DAG16) && (flags & MP_TMAT_DAG32)) {
    delete t;
    return fail(ctx, MP_ERR_ARG, "MP_TMAT_DAG16 and MP_TMAT_DAG32 exclude each other");
  }
  t->P.dag_nb_req = (flags & MP_TMAT_DAG16) ? 16 : (flags & MP_TMAT_DAG32) ? 32 : 0;
  t->P.lowp_ring4 = (flags & MP_TMAT_LOWP_RING4) != 0;
  t->P.no_graph = (flags & MP_TMAT_DIRECT) != 0;
  t->P.trace = (flags & MP_TMAT_TRACE) != 0;
  mp_status st = add_matrix(t->P, n, h_map);
  if (st == MP_OK) st = finish_plan(t->P);
  if (st != MP_OK) { delete t; return st; }
  // pinned staging for the solve items, sized for the three solve plans and
  // the residual items of mp_loglik (grown later if ever short), allocated
  // here while the stream has no work of this matrix yet
  {
    const size_t nt = (size_t)t->P.mats[0].nt, pb = (size_t)b / 32;
    const size_t bytes = 3 * (sizeof(SolveTask) * pb * nt * (nt + 3) / 2 + 2 * sizeof(ItemSolveDag) + 512) +
                         sizeof(ItemResTile) * nt * (nt + 1) / 2 + sizeof(ItemResRow) * nt + 4096;
    t->h_pin = pin_borrow(ctx, bytes, &t->h_pin_cap);
  }
  *out = t;
  return MP_OK;
}

void mp_tmat_destroy(mp_tmat* t) { delete t; }

mp_status mp_tmat_info(mp_tmat* t, int64_t* n, int32_t* b, int32_t* nt, int64_t* bytes) {
  if (!t) return MP_ERR_ARG;
  if (n) *n = t->P.mats[0].n;
  if (b) *b = t->P.b;
  if (nt) *nt = t->P.mats[0].nt;
  if (bytes) *bytes = t->P.bytes;
  return MP_OK;
}

static mp_status tile_xfer(mp_tmat* t, int32_t i, int32_t j, void* h, double* scale, bool get) {
  if (!t) return MP_ERR_ARG;
  Plan& P = t->P;
  const MatDesc& M = P.mats[0];
  if (i < 0 || j < 0 || i >= M.nt || j > i) return fail(P.ctx, MP_ERR_ARG, "tile (%d,%d) out of range", i, j);
  if (!h) return fail(P.ctx, MP_ERR_ARG, "host buffer is null");
  const int id = M.tile[i * M.nt + j];
  const TileRef r = P.h_tiles[id];
  const size_t bytes = (size_t)P.b * P.b * esize(r.dt);
  char* dev = P.pool[r.dt] + (size_t)r.idx * bytes;
  // ordered on the matrix's stream, complete on return
  if (get) {
    double s = 1.0;
    CK(P.ctx, cudaMemcpyAsync(h, dev, bytes, cudaMemcpyDeviceToHost, P.stream));
    CK(P.ctx, cudaMemcpyAsync(&s, P.d_scale + id, sizeof(double), cudaMemcpyDeviceToHost, P.stream));
    CK(P.ctx, cudaStreamSynchronize(P.stream));
    if (scale) *scale = s;
  } else {
    const double s = scale ? *scale : 1.0;
    CK(P.ctx, cudaMemcpyAsync(dev, h, bytes, cudaMemcpyHostToDevice, P.stream));
    CK(P.ctx, cudaMemcpyAsync(P.d_scale + id, &s, sizeof(double), cudaMemcpyHostToDevice, P.stream));
    CK(P.ctx, cudaStreamSynchronize(P.stream));
    t->generated = true;
    t->sig_valid = false;   // the refinement's copy of Sigma no longer matches
    P.factored = false;
  }
  return MP_OK;
}

mp_status mp_tile_get(mp_tmat* t, int32_t i, int32_t j, void* h_dst, double* scale) {
  return tile_xfer(t, i, j, h_dst, scale, true);
}

mp_status mp_tile_set(mp_tmat* t, int32_t i, int32_t j, const void* h_src, double scale) {
  return tile_xfer(t, i, j, const_cast<void*>(h_src), &scale, false);
}

mp_status mp_morton_order(mp_ctx* ctx, int64_t n, const double* d_locs_in, double* d_locs_out,
                          int64_t* d_perm, void* stream) {
  if (!ctx || !d_locs_in || !d_locs_out || !d_perm) return fail(ctx, MP_ERR_ARG, "null argument");
  if (n < 1 || n > (int64_t)1 << 31) return fail(ctx, MP_ERR_ARG, "n out of range");
  if (d_locs_in == d_locs_out) return fail(ctx, MP_ERR_ARG, "d_locs_out may not alias d_locs_in");
  std::lock_guard<std::mutex> lk(ctx->mu);
  CK(ctx, cudaSetDevice(ctx->device));
  int64_t n2 = 1024;
  while (n2 < n) n2 <<= 1;
  if (ctx->keys_cap < n2) {
    if (ctx->keys) cudaFree(ctx->keys);
    ctx->keys = nullptr;
    ctx->keys_cap = 0;
    cudaError_t e = cudaMalloc(&ctx->keys, sizeof(unsigned long long) * n2);
    if (e != cudaSuccess) return fail(ctx, MP_ERR_OOM, "morton workspace: %s", cudaGetErrorString(e));
    ctx->keys_cap = n2;
  }
  cudaStream_t s = (cudaStream_t)stream;
  launch_morton_keys(d_locs_in, n, n2, ctx->keys, s);
  launch_bitonic(ctx->keys, n2, s);
  launch_morton_gather(ctx->keys, d_locs_in, n, d_locs_out, d_perm, s);
  return check_launch(ctx);
}

// Generation items for a single-matrix handle.
static mp_status build_gen_items(mp_tmat* t) {
  Plan& P = t->P;
  const MatDesc& M = P.mats[0];
  std::vector<ItemGen> amax, all;
  // the exponent of the fixed-point copy of Sigma: every entry (at most
  // sigma^2 + nugget) below 2^sig_e
  int sig_e = 0;
  std::frexp(t->cov.sigma2 + t->cov.nugget, &sig_e);
  for (int i = 0; i < M.nt; ++i)
    for (int j = 0; j <= i; ++j) {
      ItemGen g{};
      g.tile = M.tile[i * M.nt + j];
      g.mat = 0;
      g.ti = i;
      g.tj = j;
      g.locs = t->locs;
      g.n = M.n;
      g.sigma2 = t->cov.sigma2;
      g.range = t->cov.range;
      g.nu = t->cov.nu;
      g.nugget = t->cov.nugget;
      g.sigfix = nullptr;
      if (!matern_nu_closed(t->cov.nu)) {
        g.ktab = t->d_ktab;
        g.ke0 = t->ktab_e0;
      }
      if (P.keep_sigma) {
        const TileRef r = P.h_tiles[M.sig[i * M.nt + j]];
        g.sigfix = (uint64_t*)(P.pool[F64] + (size_t)r.idx * P.b * P.b * 8);
        g.sig_e = sig_e;
        g.sig_e_out = t->d_sig_e;
      }
      if (P.h_tiles[g.tile].dt == E4M3) amax.push_back(g);
      all.push_back(g);
    }
  size_t bytes = sizeof(ItemGen) * (amax.size() + all.size());
  if (bytes > t->d_gen_cap) {
    P.raw_free(t->d_gen);
    t->d_gen = nullptr;
    CK(P.ctx, P.raw_alloc((void**)&t->d_gen, bytes));
    t->d_gen_cap = bytes;
  }
  t->gen_off_amax = 0;
  t->gen_off_all = sizeof(ItemGen) * amax.size();
  t->gen_n_amax = (int)amax.size();
  t->gen_n_all = (int)all.size();
  if (!amax.empty()) CK(P.ctx, P.upload(t->d_gen, amax.data(), sizeof(ItemGen) * amax.size()));
  CK(P.ctx, P.upload(t->d_gen + t->gen_off_all, all.data(), sizeof(ItemGen) * all.size()));
  return MP_OK;
}

static bool valid_nu(double nu) { return matern_nu_valid(nu); }

// Builds the Matérn table of nu on the host and uploads it into a device
// buffer (grown with `alloc`, a stream-ordered or plain allocation) on
// `stream`; the host table may be reused once the call returns (a copy
// from pageable memory is staged before cudaMemcpyAsync returns).
static mp_status upload_knu_table(mp_ctx* ctx, double nu, double** d_tab, size_t* cap, int* e0,
                                  cudaStream_t stream,
                                  const std::function<cudaError_t(void**, size_t)>& alloc) {
  std::vector<double> tab;
  if (matern_nu_table(nu, tab, e0)) return fail(ctx, MP_ERR_ARG, "nu must be in (0, 16]");
  const size_t bytes = sizeof(double) * tab.size();
  if (bytes > *cap) {
    cudaError_t e = alloc((void**)d_tab, bytes);
    if (e != cudaSuccess) return fail(ctx, MP_ERR_OOM, "Matérn table: %s", cudaGetErrorString(e));
    *cap = bytes;
  }
  CK(ctx, cudaMemcpyAsync(*d_tab, tab.data(), bytes, cudaMemcpyHostToDevice, stream));
  return MP_OK;
}

mp_status mp_generate_matern(mp_tmat* t, const double* d_locs, mp_matern p) {
  if (!t || !d_locs) return fail(t ? t->P.ctx : nullptr, MP_ERR_ARG, "null argument");
  Plan& P = t->P;
  if (!valid_nu(p.nu)) return fail(P.ctx, MP_ERR_ARG, "nu must be in (0, 16]");
  if (!(p.range > 0.0) || !(p.sigma2 > 0.0) || !(p.nugget >= 0.0))
    return fail(P.ctx, MP_ERR_ARG, "need range > 0, sigma2 > 0, nugget >= 0");
  CK(P.ctx, cudaSetDevice(P.ctx->device));
  if (!matern_nu_closed(p.nu) && (!t->d_ktab || p.nu != t->ktab_nu)) {
    size_t cap = t->d_ktab_cap;
    bool freed = false;
    mp_status st = upload_knu_table(P.ctx, p.nu, &t->d_ktab, &cap, &t->ktab_e0, P.stream,
                                    [&](void** q, size_t bytes) {
                                      P.raw_free(t->d_ktab);   // stream-ordered or synchronising
                                      freed = true;
                                      *q = nullptr;
                                      return P.raw_alloc(q, bytes);
                                    });
    if (st) {
      if (freed) {
        if (t->d_ktab) P.raw_free(t->d_ktab);
        t->d_ktab = nullptr;
        t->d_ktab_cap = 0;
      }
      t->ktab_nu = 0.0;
      t->gen_key.clear();
      return st;
    }
    t->d_ktab_cap = cap;
    t->ktab_nu = p.nu;
    t->gen_key.clear();          // the items carry the table's pointer and octave
  }
  if (P.keep_sigma && !t->d_sig_e) {
    CK(P.ctx, P.raw_alloc((void**)&t->d_sig_e, sizeof(int32_t)));
    t->gen_key.clear();
  }
  std::vector<char> key(sizeof(void*) + sizeof(mp_matern));
  memcpy(key.data(), &d_locs, sizeof(void*));
  memcpy(key.data() + sizeof(void*), &p, sizeof(mp_matern));
  if (key != t->gen_key) {
    t->locs = d_locs;
    t->cov = p;
    if (mp_status st = build_gen_items(t)) return st;
    t->gen_key = key;
  }
  const Arena A = P.arena();
  cudaStream_t s = P.stream;
  CK(P.ctx, cudaMemsetAsync(P.d_amax, 0, sizeof(unsigned long long) * P.n_amax, s));
  launch_gen_amax(A, (const ItemGen*)(t->d_gen + t->gen_off_amax), t->gen_n_amax, s);
  launch_generate(A, (const ItemGen*)(t->d_gen + t->gen_off_all), t->gen_n_all, s);
  t->generated = true;
  t->sig_valid = P.keep_sigma;
  P.factored = false;
  return check_launch(P.ctx);
}

mp_status mp_chol_steps(mp_tmat* t, int32_t k0, int32_t k1) {
  if (!t) return MP_ERR_ARG;
  Plan& P = t->P;
  const int nt = P.mats[0].nt;
  if (k0 < 0 || k1 > nt || k0 > k1) return fail(P.ctx, MP_ERR_ARG, "steps out of range");
  if (!t->generated) return fail(P.ctx, MP_ERR_STATE, "matrix not generated or loaded");
  CK(P.ctx, cudaSetDevice(P.ctx->device));
  if (k0 == 0) run_launch(P, P.chol[0], P.stream);   // info reset
  // the digit split of step k0's first panel tiles is issued by step k0-1
  if (k0 >= 1 && k0 < k1 && P.first_split[k0] >= 0) run_launch(P, P.chol[P.first_split[k0]], P.stream);
  for (size_t l = P.step_begin[k0]; l < P.step_begin[k1]; ++l) run_launch(P, P.chol[l], P.stream);
  if (k1 == nt) {
    run_launch(P, P.chol.back(), P.stream);
    P.factored = true;
  }
  return check_launch(P.ctx);
}

namespace {
__global__ void k_info_out(const long long* info, const int* err, long long* out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = *err ? -(long long)MP_ERR_TIMEOUT : info[i] == 0x7f7f7f7f7f7f7f7fLL ? 0 : info[i];
}
}  // namespace

mp_status mp_chol(mp_tmat* t, int64_t* d_info, double* d_logdet) {
  if (!t) return MP_ERR_ARG;
  Plan& P = t->P;
  if (!t->generated) return fail(P.ctx, MP_ERR_STATE, "matrix not generated or loaded");
  CK(P.ctx, cudaSetDevice(P.ctx->device));
  if (P.no_graph) {
    run_chol_direct(P);
  } else {
    if (!P.chol_exec) {
      mp_status st = capture_graph(P.ctx, P.cap, [&](cudaStream_t s) {
        run_chol_forked(P, s);
      }, &P.chol_exec, &P.chol_kernels);
      if (st) return st;
    }
    if (mp_status st = launch_graph(P.ctx, P.chol_exec, P.stream)) return st;
  }
  if (d_info) k_info_out<<<1, 32, 0, P.stream>>>(P.d_info, P.d_err, (long long*)d_info, 1);
  if (d_logdet) CK(P.ctx, cudaMemcpyAsync(d_logdet, P.d_logdet, sizeof(double), cudaMemcpyDeviceToDevice, P.stream));
  P.factored = true;
  return check_launch(P.ctx);
}

mp_status mp_tmat_set_wait_budget(mp_tmat* t, int32_t polls) {
  if (!t || polls < 0) return MP_ERR_ARG;
  Plan& P = t->P;
  if (polls == P.wait_polls) return MP_OK;
  CK(P.ctx, cudaSetDevice(P.ctx->device));
  // the captured graphs hold the arena (and with it the budget) by value
  CK(P.ctx, cudaStreamSynchronize(P.stream));
  if (P.chol_exec) { cudaGraphExecDestroy(P.chol_exec); P.chol_exec = nullptr; }
  if (t->ll_exec) { cudaGraphExecDestroy(t->ll_exec); t->ll_exec = nullptr; t->ll_key.clear(); }
  P.wait_polls = polls;
  return MP_OK;
}

mp_status mp_potrf_dag_schedule(int32_t nb, uint8_t* h_out, int64_t cap, int64_t* count) {
  if (nb < 1 || nb > 64 || !count) return MP_ERR_ARG;
  const std::vector<DagTask> v = potrf_dag_tasks(nb);
  *count = (int64_t)v.size();
  if (!h_out) return MP_OK;
  if (cap < (int64_t)v.size()) return MP_ERR_ARG;
  for (size_t i = 0; i < v.size(); ++i) {
    h_out[4 * i] = v[i].op;
    h_out[4 * i + 1] = v[i].r;
    h_out[4 * i + 2] = v[i].c;
    h_out[4 * i + 3] = v[i].k;
  }
  return MP_OK;
}

mp_status mp_solve_dag_schedule(int32_t nt, int32_t p_blocks, int32_t trans, uint64_t* h_out, int64_t cap,
                                int64_t* count) {
  if (nt < 1 || nt > 4095 || p_blocks < 1 || p_blocks > 255 || !count) return MP_ERR_ARG;
  const std::vector<SolveTask> v = solve_dag_tasks({nt}, p_blocks, trans ? 1 : 0);
  *count = (int64_t)v.size();
  if (!h_out) return MP_OK;
  if (cap < (int64_t)v.size()) return MP_ERR_ARG;
  for (size_t i = 0; i < v.size(); ++i) h_out[i] = v[i];
  return MP_OK;
}

mp_status mp_tmat_chain_trace(mp_tmat* t, uint64_t* h_out, int64_t cap, int64_t* count, int32_t* block) {
  if (!t || !count) return MP_ERR_ARG;
  Plan& P = t->P;
  if (!P.d_trace) return fail(P.ctx, MP_ERR_STATE, "the matrix was created without MP_TMAT_TRACE");
  *count = P.trace_words;
  if (block) *block = P.dag_nb;
  if (!h_out) return MP_OK;
  if (cap < P.trace_words) return fail(P.ctx, MP_ERR_ARG, "trace needs %lld words", (long long)P.trace_words);
  CK(P.ctx, cudaSetDevice(P.ctx->device));
  CK(P.ctx, cudaMemcpyAsync(h_out, P.d_trace, sizeof(uint64_t) * P.trace_words, cudaMemcpyDeviceToHost,
                            P.stream));
  CK(P.ctx, cudaStreamSynchronize(P.stream));
  return MP_OK;
}

mp_status mp_logdet(mp_tmat* t, double* d_out) {
  if (!t || !d_out) return MP_ERR_ARG;
  Plan& P = t->P;
  if (!P.factored) return fail(P.ctx, MP_ERR_STATE, "mp_chol has not been called");
  CK(P.ctx, cudaMemcpyAsync(d_out, P.d_logdet, sizeof(double), cudaMemcpyDeviceToDevice, P.stream));
  return MP_OK;
}

}  // extern "C"

// --------------------------------------------------------------- solves

namespace {

// One triangular solve of the plan's matrices, run by the solve task graph.
struct SolvePlan {
  size_t items_off = 0, tasks_off = 0;
  int ntasks = 0, trans = 0, nrhs_max = 1;
};

// Forward (trans = 0: out = L^{-1} in) or backward (trans = 1: out = L^{-T}
// in) tiled solve of the plan's matrices, out of place; `in` is consumed,
// `chain` is scratch.  Vectors are given per matrix as padded N x nrhs
// blocks with leading dimension ld.
SolvePlan build_solve(Plan& P, const std::vector<double*>& in, const std::vector<double*>& out,
                      const std::vector<double*>& chain, const std::vector<int64_t>& ld,
                      const std::vector<int>& nrhs, int trans) {
  SolvePlan sp;
  std::vector<ItemSolveDag> items;
  std::vector<int> nts;
  for (int m = 0; m < (int)P.mats.size(); ++m) {
    const MatDesc& M = P.mats[m];
    ItemSolveDag it{};
    it.tiles = P.d_ltab + P.ltab_off[m];
    it.linv = it.tiles + (int64_t)M.nt * M.nt;
    it.in = in[m];
    it.out = out[m];
    it.chain = chain[m];
    it.cnt = P.d_scnt + P.scnt_off[m];
    it.ld = ld[m];
    it.nt = M.nt;
    it.nrhs = nrhs[m];
    it.ffdiag = M.mixed ? 1 : 0;
    sp.nrhs_max = std::max(sp.nrhs_max, nrhs[m]);
    items.push_back(it);
    nts.push_back(M.nt);
  }
  const std::vector<SolveTask> tasks = solve_dag_tasks(nts, P.b / 32, trans);
  sp.items_off = P.push(items);
  sp.tasks_off = P.push(tasks);
  sp.ntasks = (int)tasks.size();
  sp.trans = trans;
  return sp;
}

void run_solve(const Plan& P, const char* dbase, const SolvePlan& sp, const int* gate, cudaStream_t s) {
  cudaMemsetAsync(P.d_scnt, 0, P.scnt_bytes, s);
  launch_solve_dag(P.arena(), reinterpret_cast<const ItemSolveDag*>(dbase + sp.items_off),
                   reinterpret_cast<const SolveTask*>(dbase + sp.tasks_off), sp.ntasks, P.d_scnt,
                   sp.trans, sp.nrhs_max, gate, s);
}

}  // namespace

// Copies bytes of solve items into t->d_sitems through the pinned staging
// buffer, so that the host does not wait for the work already on the stream;
// the buffer is rewritten only after its previous copy has run.
static cudaError_t upload_pinned(mp_tmat* t, const char* src, size_t bytes) {
  Plan& P = t->P;
  cudaError_t e = cudaSuccess;
  if (!t->pin_ev && (e = cudaEventCreateWithFlags(&t->pin_ev, cudaEventDisableTiming)) != cudaSuccess) return e;
  if (t->pin_used && (e = cudaEventSynchronize(t->pin_ev)) != cudaSuccess) return e;
  if (bytes > t->h_pin_cap) {
    pin_return(P.ctx, t->h_pin, t->h_pin_cap);
    t->h_pin_cap = 0;
    t->h_pin = pin_borrow(P.ctx, bytes, &t->h_pin_cap);
    if (!t->h_pin) return cudaErrorMemoryAllocation;
  }
  memcpy(t->h_pin, src, bytes);
  if ((e = cudaMemcpyAsync(t->d_sitems, t->h_pin, bytes, cudaMemcpyHostToDevice, P.stream)) != cudaSuccess)
    return e;
  t->pin_used = true;
  return cudaEventRecord(t->pin_ev, P.stream);
}

// Solve workspace of a single-matrix handle for nrhs right-hand sides.
static mp_status ensure_ws(mp_tmat* t, int nrhs) {
  if (t->ws_nrhs >= nrhs) return MP_OK;
  Plan& P = t->P;
  for (void* p : t->ws_allocs) P.raw_free(p);
  t->ws_allocs.clear();
  const int64_t N = (int64_t)P.mats[0].nt * P.b;
  auto A = [&](void** p, size_t bytes) -> mp_status {
    cudaError_t e = P.raw_alloc(p, bytes);
    if (e != cudaSuccess) return fail(P.ctx, MP_ERR_OOM, "solve workspace: %s", cudaGetErrorString(e));
    t->ws_allocs.push_back(*p);
    return MP_OK;
  };
  mp_status st;
  if ((st = A((void**)&t->zp, sizeof(double) * N * nrhs))) return st;
  if ((st = A((void**)&t->x, sizeof(double) * N * nrhs))) return st;
  if ((st = A((void**)&t->r, sizeof(double) * N * nrhs))) return st;
  if ((st = A((void**)&t->w, sizeof(double) * N * nrhs))) return st;
  if ((st = A((void**)&t->d, sizeof(double) * N * nrhs))) return st;
  if ((st = A((void**)&t->c, sizeof(double) * N * nrhs))) return st;
  if ((st = A((void**)&t->rowabs, sizeof(double) * N))) return st;
  if (P.keep_sigma) {
    const size_t nt = (size_t)P.mats[0].nt;
    if ((st = A((void**)&t->rpart, sizeof(double) * nt * nt * P.b * nrhs))) return st;
    if ((st = A((void**)&t->rpabs, sizeof(float) * nt * nt * P.b))) return st;
  }
  if ((st = A((void**)&t->red, sizeof(double) * (5 * nrhs + 2)))) return st;
  if ((st = A((void**)&t->active, sizeof(int) * nrhs))) return st;
  if ((st = A((void**)&t->iters, sizeof(int) * nrhs))) return st;
  if ((st = A((void**)&t->any, sizeof(int) * 2))) return st;
  t->ws_nrhs = nrhs;
  if (t->ll_exec) { cudaGraphExecDestroy(t->ll_exec); t->ll_exec = nullptr; }
  t->ll_key.clear();
  return MP_OK;
}

namespace {
__global__ void k_refine_init(int* active, int* iters, int* any, int nrhs) {
  int c = threadIdx.x;
  for (int i = c; i < nrhs; i += blockDim.x) { active[i] = 1; iters[i] = 0; }
  if (c == 0) *any = 1;
}
__global__ void k_copy_iters(const int* src, int32_t* dst, int nrhs) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nrhs) dst[c] = src[c];
}
}  // namespace

namespace {
__global__ void k_identity(double* d, int64_t n, int64_t ld, int64_t c0, int64_t cols) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * cols) return;
  const int64_t r = idx % n, c = idx / n;
  d[r + c * ld] = r == c0 + c ? 1.0 : 0.0;
}
constexpr int32_t SOLVE_CHUNK = 2048;   // right-hand sides per solve (bounds the workspace)
}  // namespace

extern "C" mp_status mp_solve(mp_tmat* t, double* d_B, int64_t ldb, int32_t nrhs) {
  if (!t || !d_B || nrhs < 1) return MP_ERR_ARG;
  for (int32_t c0 = 0; c0 < nrhs; c0 += SOLVE_CHUNK) {
    const int32_t nc = std::min(SOLVE_CHUNK, nrhs - c0);
    double* B = d_B + (int64_t)c0 * ldb;
    if (mp_status st = mp_trsm(t, 0, B, ldb, nc)) return st;
    if (mp_status st = mp_trsm(t, 1, B, ldb, nc)) return st;
  }
  return MP_OK;
}

extern "C" mp_status mp_chol2inv(mp_tmat* t, double* d_out, int64_t ldo) {
  if (!t || !d_out) return MP_ERR_ARG;
  Plan& P = t->P;
  const int64_t n = P.mats[0].n;
  if (ldo < n) return fail(P.ctx, MP_ERR_ARG, "ldo must be >= n");
  if (!P.factored) return fail(P.ctx, MP_ERR_STATE, "mp_chol has not been called");
  CK(P.ctx, cudaSetDevice(P.ctx->device));
  for (int64_t c0 = 0; c0 < n; c0 += SOLVE_CHUNK) {
    const int64_t nc = std::min<int64_t>(SOLVE_CHUNK, n - c0);
    double* B = d_out + c0 * ldo;
    k_identity<<<(unsigned)((n * nc + 255) / 256), 256, 0, P.stream>>>(B, n, ldo, c0, nc);
    if (mp_status st = mp_solve(t, B, ldo, (int32_t)nc)) return st;
  }
  return MP_OK;
}

extern "C" mp_status mp_trsm(mp_tmat* t, int trans, double* d_B, int64_t ldb, int32_t nrhs) {
  if (!t || !d_B) return MP_ERR_ARG;
  Plan& P = t->P;
  const MatDesc& M = P.mats[0];
  if (!P.factored) return fail(P.ctx, MP_ERR_STATE, "mp_chol has not been called");
  if (nrhs < 1 || ldb < M.n) return fail(P.ctx, MP_ERR_ARG, "need nrhs >= 1 and ldb >= n");
  CK(P.ctx, cudaSetDevice(P.ctx->device));
  if (mp_status st = ensure_ws(t, nrhs)) return st;
  const int64_t N = (int64_t)M.nt * P.b;
  // solve on the padded copy, then copy the first n rows back
  std::vector<char> saved;
  saved.swap(P.h_items);
  const SolvePlan ls = build_solve(P, {t->x}, {t->w}, {t->c}, {N}, {nrhs}, trans ? 1 : 0);
  size_t bytes = P.h_items.size();
  if (bytes > t->d_sitems_cap) {
    P.raw_free(t->d_sitems);
    t->d_sitems = nullptr;
    cudaError_t e = P.raw_alloc((void**)&t->d_sitems, bytes);
    if (e != cudaSuccess) { P.h_items.swap(saved); return fail(P.ctx, MP_ERR_OOM, "solve items"); }
    t->d_sitems_cap = bytes;
  }
  cudaError_t e = cudaMemcpyAsync(t->d_sitems, P.h_items.data(), bytes, cudaMemcpyHostToDevice, P.stream);
  cudaStreamSynchronize(P.stream);
  P.h_items.swap(saved);
  if (e != cudaSuccess) return fail(P.ctx, MP_ERR_CUDA, "solve items copy");
  // the loglik graph caches item bytes in d_sitems: invalidate it
  if (t->ll_exec) { cudaGraphExecDestroy(t->ll_exec); t->ll_exec = nullptr; t->ll_key.clear(); }
  launch_copy_pad(d_B, ldb, t->x, N, M.n, N, nrhs, nullptr, P.stream);
  run_solve(P, t->d_sitems, ls, nullptr, P.stream);
  launch_copy_pad(t->w, N, d_B, ldb, M.n, M.n, nrhs, nullptr, P.stream);
  return check_launch(P.ctx);
}

extern "C" mp_status mp_loglik(mp_tmat* t, const double* d_z, int64_t ldz, int32_t nrhs,
                               int32_t refine_iters, double* d_ll, double* d_quad,
                               int32_t* d_iters) {
  if (!t || !d_z || !d_ll) return MP_ERR_ARG;
  Plan& P = t->P;
  const MatDesc& M = P.mats[0];
  if (!P.factored) return fail(P.ctx, MP_ERR_STATE, "mp_chol has not been called");
  if (nrhs < 1 || ldz < M.n) return fail(P.ctx, MP_ERR_ARG, "need nrhs >= 1 and ldz >= n");
  if (refine_iters < 0 || refine_iters > 100) return fail(P.ctx, MP_ERR_ARG, "refine_iters in [0, 100]");
  if (refine_iters > 0 && !P.keep_sigma)
    return fail(P.ctx, MP_ERR_STATE, "refinement needs MP_TMAT_KEEP_SIGMA");
  if (refine_iters > 0 && !t->sig_valid)
    return fail(P.ctx, MP_ERR_STATE, "refinement needs Sigma from mp_generate_matern (tiles set since)");
  CK(P.ctx, cudaSetDevice(P.ctx->device));
  if (mp_status st = ensure_ws(t, nrhs)) return st;
  std::vector<char> key(sizeof(void*) * 4 + sizeof(int64_t) + 2 * sizeof(int32_t));
  {
    char* k = key.data();
    memcpy(k, &d_z, 8); memcpy(k + 8, &d_ll, 8); memcpy(k + 16, &d_quad, 8); memcpy(k + 24, &d_iters, 8);
    memcpy(k + 32, &ldz, 8); memcpy(k + 40, &nrhs, 4); memcpy(k + 44, &refine_iters, 4);
  }
  if (!t->ll_exec || key != t->ll_key) {
    const int64_t N = (int64_t)M.nt * P.b;
    std::vector<char> saved;
    saved.swap(P.h_items);
    // r -> w (forward), w -> x or w -> d (backward)
    const SolvePlan fwd_rw = build_solve(P, {t->r}, {t->w}, {t->c}, {N}, {nrhs}, 0);
    const SolvePlan bwd_wx = build_solve(P, {t->w}, {t->x}, {t->c}, {N}, {nrhs}, 1);
    const SolvePlan bwd_wd = build_solve(P, {t->w}, {t->d}, {t->c}, {N}, {nrhs}, 1);
    std::vector<ItemResTile> rtiles;
    std::vector<ItemResRow> rrows;
    for (int i = 0; i < M.nt && refine_iters > 0; ++i) {
      for (int j = 0; j <= i; ++j) {
        ItemResTile it{};
        it.tile = M.sig[(size_t)i * M.nt + j];
        it.ti = i;
        it.tj = j;
        it.nt = M.nt;
        it.sig_e = t->d_sig_e;
        it.x = t->x;
        it.part = t->rpart;
        it.pabs = t->rpabs;
        it.ld = N;
        it.nrhs = nrhs;
        rtiles.push_back(it);
      }
      ItemResRow r{};
      r.ti = i;
      r.nt = M.nt;
      r.part = t->rpart;
      r.pabs = t->rpabs;
      r.z = t->zp;
      r.r = t->r;
      r.rowabs = t->rowabs;
      r.ld = N;
      r.nrhs = nrhs;
      rrows.push_back(r);
    }
    const size_t rtiles_off = P.push(rtiles), rrows_off = P.push(rrows);
    size_t bytes = P.h_items.size();
    if (bytes > t->d_sitems_cap) {
      P.raw_free(t->d_sitems);
      t->d_sitems = nullptr;
      cudaError_t e = P.raw_alloc((void**)&t->d_sitems, bytes);
      if (e != cudaSuccess) { P.h_items.swap(saved); return fail(P.ctx, MP_ERR_OOM, "solve items"); }
      t->d_sitems_cap = bytes;
    }
    cudaError_t e = upload_pinned(t, P.h_items.data(), bytes);
    P.h_items.swap(saved);
    if (e != cudaSuccess) return fail(P.ctx, MP_ERR_CUDA, "solve items copy");
    double* red = t->red;
    double *zmax = red, *xmax = red + nrhs, *rmax = red + 2 * nrhs, *quad = red + 3 * nrhs,
           *snorm = red + 4 * nrhs;
    const int64_t n = M.n;
    const char* db = t->d_sitems;
    const ItemResTile* rti = reinterpret_cast<const ItemResTile*>(db + rtiles_off);
    const ItemResRow* rro = reinterpret_cast<const ItemResRow*>(db + rrows_off);
    auto body = [&](cudaStream_t s) {
      launch_copy_pad(d_z, ldz, t->zp, N, n, N, nrhs, nullptr, s);
      launch_copy_pad(t->zp, N, t->r, N, N, N, nrhs, nullptr, s);
      k_refine_init<<<1, 128, 0, s>>>(t->active, t->iters, t->any, nrhs);
      run_solve(P, db, fwd_rw, nullptr, s);
      if (refine_iters == 0) {
        launch_dot(t->w, t->w, N, N, nrhs, quad, s);
      } else {
        run_solve(P, db, bwd_wx, nullptr, s);
        launch_colmax(t->zp, n, N, nrhs, zmax, nullptr, s);
        for (int itr = 0; itr < refine_iters; ++itr) {
          launch_residual(P.arena(), rti, (int)rtiles.size(), rro, (int)rrows.size(), nrhs, itr == 0,
                          t->any, s);
          if (itr == 0) launch_colmax(t->rowabs, n, N, 1, snorm, t->any, s);
          launch_colmax(t->r, n, N, nrhs, rmax, t->any, s);
          launch_colmax(t->x, n, N, nrhs, xmax, t->any, s);
          launch_refine_check(rmax, xmax, zmax, snorm, n, nrhs, t->active, t->iters, t->any,
                              t->any, s);
          run_solve(P, db, fwd_rw, t->any, s);
          run_solve(P, db, bwd_wd, t->any, s);
          launch_axpy_active(t->x, t->d, N, N, nrhs, t->active, t->any, s);
        }
        launch_dot(t->zp, t->x, N, N, nrhs, quad, s);
      }
      launch_loglik(P.d_logdet, quad, n, nrhs, d_ll, P.d_err, s);
      if (d_quad) cudaMemcpyAsync(d_quad, quad, sizeof(double) * nrhs, cudaMemcpyDeviceToDevice, s);
      if (d_iters) k_copy_iters<<<(nrhs + 127) / 128, 128, 0, s>>>(t->iters, d_iters, nrhs);
    };
    if (P.no_graph) {       // one-shot matrices: direct launches, no capture
      body(P.stream);
      return check_launch(P.ctx);
    }
    mp_status st = capture_graph(P.ctx, P.cap, body, &t->ll_exec, &t->ll_kernels);
    if (st) return st;
    t->ll_key = key;
  }
  return launch_graph(P.ctx, t->ll_exec, P.stream);
}

extern "C" mp_status mp_gemm(mp_ctx* ctx, mp_dtype dtype, char ta, char tb, int64_t m, int64_t n,
                             int64_t k, double alpha, const void* d_A, int64_t lda,
                             const void* d_B, int64_t ldb, double beta, void* d_C, int64_t ldc,
                             void* stream) {
  if (!ctx) return MP_ERR_ARG;
  if ((int)dtype < 0 || (int)dtype >= NDT) return fail(ctx, MP_ERR_ARG, "bad dtype");
  auto tr = [](char c) { return c == 'T' || c == 't' ? 1 : (c == 'N' || c == 'n' ? 0 : -1); };
  const int a = tr(ta), bb = tr(tb);
  if (a < 0 || bb < 0) return fail(ctx, MP_ERR_ARG, "ta/tb must be 'N' or 'T'");
  if (m < 0 || n < 0 || k < 0) return fail(ctx, MP_ERR_ARG, "negative size");
  if (m == 0 || n == 0) return MP_OK;
  if (!d_A || !d_B || !d_C) return fail(ctx, MP_ERR_ARG, "null matrix");
  if (ldc < m || lda < (a ? k : m) || ldb < (bb ? n : k))
    return fail(ctx, MP_ERR_ARG, "leading dimension too small");
  if (m >= (int64_t)65535 * 64 || n >= (int64_t)65535 * 64)
    return fail(ctx, MP_ERR_ARG, "m or n too large");
  CK(ctx, cudaSetDevice(ctx->device));
  if (dtype != MP_F64 && k > 0 && !getenv("MPCHOL_GEMM_SIMT")) {
    // BF16, FP16, E4M3, FP32 (three TF32 products) on the tcgen05 tensor cores
    const int rc = launch_gemm_tc((int)dtype, a, bb, m, n, k, alpha, d_A, lda, d_B, ldb, beta, d_C, ldc,
                                  (cudaStream_t)stream);
    if (rc == 1) return fail(ctx, MP_ERR_OOM, "mp_gemm: workspace allocation failed");
    if (rc == 2) return fail(ctx, MP_ERR_CUDA, "mp_gemm: %s", cudaGetErrorString(cudaGetLastError()));
    if (rc == 0) return check_launch(ctx);
  }
  launch_gemm((int)dtype, a, bb, m, n, k, alpha, d_A, lda, d_B, ldb, beta, d_C, ldc,
              (cudaStream_t)stream);
  return check_launch(ctx);
}

// ------------------------------------------------------------------ batch

namespace {

struct ItemBatchOut {
  const double* w;     // forward-solved vectors (N x nrhs, ld N)
  int64_t n, N;
  int32_t nrhs, mat;
  double* ll;          // output slot
  int32_t* status;
  int32_t pad_[2];
};

__global__ void k_batch_out(const ItemBatchOut* items, int count, const double* logdet,
                            const long long* info, const int* err) {
  const int m = blockIdx.x;
  if (m >= count) return;
  const ItemBatchOut it = items[m];
  __shared__ double red[8];
  const double log2pi = 1.8378770664093454836;
  for (int c = 0; c < it.nrhs; ++c) {
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < it.N; i += blockDim.x) {
      double v = it.w[(int64_t)c * it.N + i];
      s += v * v;
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < 8; ++w) s += red[w];
      it.ll[c] = -0.5 * (double)it.n * log2pi - 0.5 * logdet[it.mat] - 0.5 * s;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    it.status[0] = *err ? MP_ERR_TIMEOUT
                        : info[it.mat] == 0x7f7f7f7f7f7f7f7fLL ? MP_OK : MP_ERR_NOT_SPD;
}

struct ItemBatchCopy {
  const double* src;
  double* dst;
  int64_t n, N;
  int32_t nrhs, pad_;
};

__global__ void k_batch_copy(const ItemBatchCopy* items) {
  const ItemBatchCopy it = items[blockIdx.x];
  for (int c = 0; c < it.nrhs; ++c)
    for (int64_t i = threadIdx.x; i < it.N; i += blockDim.x)
      it.dst[(int64_t)c * it.N + i] = i < it.n ? it.src[(int64_t)c * it.n + i] : 0.0;
}

}  // namespace

extern "C" mp_status mp_batch_create(mp_ctx* ctx, int32_t count, const mp_request* reqs, int32_t b,
                                     void* stream, mp_batch** out) {
  if (b != 0) return mp_batch_create_ex(ctx, count, reqs, b, 0, stream, out);
  mp_tuned t{};
  if (mp_status st = mp_tune_batch(ctx, count, reqs, getenv("MPCHOL_TUNE_CACHE"), stream, &t)) return st;
  return mp_batch_create_ex(ctx, count, reqs, t.b, t.flags, stream, out);
}

extern "C" mp_status mp_batch_create_ex(mp_ctx* ctx, int32_t count, const mp_request* reqs, int32_t b,
                                        uint32_t flags, void* stream, mp_batch** out) {
  if (!ctx || !reqs || !out || count < 1) return fail(ctx, MP_ERR_ARG, "bad batch arguments");
  const uint32_t allowed = MP_TMAT_SIMT_UPDATES | MP_TMAT_FP64_PANEL | MP_TMAT_DAG16 | MP_TMAT_DAG32 |
                           MP_TMAT_LOWP_RING4;
  if ((flags & ~allowed) || ((flags & MP_TMAT_DAG16) && (flags & MP_TMAT_DAG32)))
    return fail(ctx, MP_ERR_ARG, "bad batch schedule flags 0x%x", flags);
  int64_t nmax = 0;
  for (int r = 0; r < count; ++r) {
    const mp_request& q = reqs[r];
    if (q.n < 1 || !q.d_locs || !q.d_z || q.nrhs < 1)
      return fail(ctx, MP_ERR_ARG, "request %d: bad n, pointers or nrhs", r);
    if (q.refine_iters != 0) return fail(ctx, MP_ERR_ARG, "request %d: batched refinement is not supported", r);
    if (!valid_nu(q.cov.nu) || !(q.cov.range > 0) || !(q.cov.sigma2 > 0) || !(q.cov.nugget >= 0))
      return fail(ctx, MP_ERR_ARG, "request %d: bad covariance parameters (nu in (0, 16])", r);
    nmax = std::max(nmax, q.n);
  }
  (void)nmax;
  if (b < 128 || b > 1024 || b % 128) return fail(ctx, MP_ERR_ARG, "b must be a multiple of 128 in [128, 1024]");
  CK(ctx, cudaSetDevice(ctx->device));
  mp_batch* B = new mp_batch;
  B->P.ctx = ctx;
  B->P.b = b;
  B->P.stream = (cudaStream_t)stream;
  // the same plan options as mp_tmat_create's flags, so that a request gives
  // the bits of its single evaluation with the same b and flags
  B->P.ozaki = (flags & MP_TMAT_FP64_PANEL) == 0;
  B->P.use_tc = (flags & MP_TMAT_SIMT_UPDATES) == 0;
  B->P.dag_nb_req = (flags & MP_TMAT_DAG16) ? 16 : (flags & MP_TMAT_DAG32) ? 32 : 0;
  B->P.lowp_ring4 = (flags & MP_TMAT_LOWP_RING4) != 0;
  B->flags = flags;
  B->count = count;
  B->reqs.assign(reqs, reqs + count);
  Plan& P = B->P;
  mp_status st = MP_OK;
  for (int r = 0; r < count && st == MP_OK; ++r) {
    const mp_request& q = reqs[r];
    std::vector<uint8_t> rule_map;
    if (!q.h_map && q.rule_eps > 0) {
      // the bound map at this plan's b, from the request's locations
      std::vector<double> h_locs(2 * (size_t)q.n);
      cudaError_t e = cudaMemcpy(h_locs.data(), q.d_locs, sizeof(double) * 2 * q.n, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) { st = fail(ctx, MP_ERR_CUDA, "request %d: locations: %s", r, cudaGetErrorString(e)); break; }
      const int nt = (int)((q.n + b - 1) / b);
      rule_map.resize((size_t)nt * nt);
      st = mp_map_bound(q.n, b, h_locs.data(), q.cov, q.rule_band, q.rule_near, q.rule_far, q.rule_eps,
                        rule_map.data());
      if (st) { fail(ctx, st, "request %d: map rule", r); break; }
    }
    st = add_matrix(P, q.n, rule_map.empty() ? q.h_map : rule_map.data());
  }
  if (st == MP_OK) st = finish_plan(P);
  if (st != MP_OK) { delete B; return st; }
  // workspace: padded vectors, outputs
  int64_t vec_total = 0;
  for (int r = 0; r < count; ++r) {
    vec_total += (int64_t)P.mats[r].nt * b * reqs[r].nrhs;
    B->total_rhs += reqs[r].nrhs;
  }
  void* p;
  if ((st = P.alloc(&p, sizeof(double) * vec_total))) { delete B; return st; }
  double* vec = (double*)p;
  if ((st = P.alloc(&p, sizeof(double) * vec_total))) { delete B; return st; }
  double* wout = (double*)p;
  if ((st = P.alloc(&p, sizeof(double) * vec_total))) { delete B; return st; }
  double* chn = (double*)p;
  if ((st = P.alloc(&p, sizeof(double) * B->total_rhs))) { delete B; return st; }
  B->d_llbuf = (double*)p;
  if ((st = P.alloc(&p, sizeof(int32_t) * count))) { delete B; return st; }
  B->d_stbuf = (int32_t*)p;
  // Matérn tables of the requests' nu without a closed form, one per value
  std::vector<std::pair<double, std::pair<double*, int>>> ktabs;
  for (int r = 0; r < count; ++r) {
    const double nu = reqs[r].cov.nu;
    if (matern_nu_closed(nu)) continue;
    bool have = false;
    for (auto& k : ktabs) have = have || k.first == nu;
    if (have) continue;
    double* d = nullptr;
    size_t cap = 0;
    int e0 = 0;
    st = upload_knu_table(ctx, nu, &d, &cap, &e0, P.stream, [&](void** q, size_t bytes) {
      return P.alloc(q, bytes) == MP_OK ? cudaSuccess : cudaErrorMemoryAllocation;
    });
    if (st) { delete B; return st; }
    ktabs.push_back({nu, {d, e0}});
  }
  // generation items
  std::vector<ItemGen> gamax, gall;
  std::vector<ItemBatchCopy> cp;
  std::vector<ItemBatchOut> outs;
  std::vector<double*> vp, wp, cp_;
  std::vector<int64_t> ld;
  std::vector<int> nr;
  int64_t vo = 0;
  int rhs_o = 0;
  for (int r = 0; r < count; ++r) {
    const MatDesc& M = P.mats[r];
    for (int i = 0; i < M.nt; ++i)
      for (int j = 0; j <= i; ++j) {
        ItemGen g{};
        g.tile = M.tile[i * M.nt + j];
        g.mat = r;
        g.ti = i;
        g.tj = j;
        g.locs = reqs[r].d_locs;
        g.n = M.n;
        g.sigma2 = reqs[r].cov.sigma2;
        g.range = reqs[r].cov.range;
        g.nu = reqs[r].cov.nu;
        g.nugget = reqs[r].cov.nugget;
        for (auto& k : ktabs)
          if (k.first == g.nu) {
            g.ktab = k.second.first;
            g.ke0 = k.second.second;
          }
        if (P.h_tiles[g.tile].dt == E4M3) gamax.push_back(g);
        gall.push_back(g);
      }
    const int64_t N = (int64_t)M.nt * b;
    ItemBatchCopy c{reqs[r].d_z, vec + vo, M.n, N, reqs[r].nrhs, 0};
    cp.push_back(c);
    ItemBatchOut o{};
    o.w = wout + vo;
    o.n = M.n;
    o.N = N;
    o.nrhs = reqs[r].nrhs;
    o.mat = r;
    o.ll = B->d_llbuf + rhs_o;
    o.status = B->d_stbuf + r;
    outs.push_back(o);
    vp.push_back(vec + vo);
    wp.push_back(wout + vo);
    cp_.push_back(chn + vo);
    ld.push_back(N);
    nr.push_back(reqs[r].nrhs);
    vo += N * reqs[r].nrhs;
    rhs_o += reqs[r].nrhs;
  }
  size_t off_ga = P.push(gamax), off_g = P.push(gall), off_cp = P.push(cp), off_out = P.push(outs);
  const SolvePlan fwd = build_solve(P, vp, wp, cp_, ld, nr, 0);
  if ((st = upload_items(P))) { delete B; return st; }
  st = capture_graph(ctx, P.cap, [&](cudaStream_t s) {
    const Arena A = P.arena();
    cudaMemsetAsync(P.d_amax, 0, sizeof(unsigned long long) * P.n_amax, s);
    launch_gen_amax(A, P.item<ItemGen>(off_ga), (int)gamax.size(), s);
    launch_generate(A, P.item<ItemGen>(off_g), (int)gall.size(), s);
    run_chol_forked(P, s);
    k_batch_copy<<<count, 256, 0, s>>>(P.item<ItemBatchCopy>(off_cp));
    run_solve(P, P.d_items, fwd, nullptr, s);
    k_batch_out<<<count, 256, 0, s>>>(P.item<ItemBatchOut>(off_out), count, P.d_logdet, P.d_info,
                                      P.d_err);
  }, &B->exec);
  if (st != MP_OK) { delete B; return st; }
  *out = B;
  return MP_OK;
}

extern "C" void mp_batch_destroy(mp_batch* batch) { delete batch; }

extern "C" mp_status mp_batch_info(mp_batch* batch, int64_t* bytes, int32_t* b) {
  if (!batch) return MP_ERR_ARG;
  if (bytes) *bytes = batch->P.bytes;
  if (b) *b = batch->P.b;
  return MP_OK;
}

extern "C" mp_status mp_batch_flags(mp_batch* batch, uint32_t* flags) {
  if (!batch || !flags) return MP_ERR_ARG;
  *flags = batch->flags;
  return MP_OK;
}

extern "C" mp_status mp_batch_run(mp_batch* batch, double* d_ll, int32_t* d_status) {
  if (!batch || !d_ll || !d_status) return MP_ERR_ARG;
  Plan& P = batch->P;
  CK(P.ctx, cudaSetDevice(P.ctx->device));
  if (mp_status st = launch_graph(P.ctx, batch->exec, P.stream)) return st;
  CK(P.ctx, cudaMemcpyAsync(d_ll, batch->d_llbuf, sizeof(double) * batch->total_rhs,
                            cudaMemcpyDeviceToDevice, P.stream));
  CK(P.ctx, cudaMemcpyAsync(d_status, batch->d_stbuf, sizeof(int32_t) * batch->count,
                            cudaMemcpyDeviceToDevice, P.stream));
  return MP_OK;
}

extern "C" mp_status mp_loglik_batch(mp_ctx* ctx, int32_t count, const mp_request* reqs,
                                     double* d_ll, int32_t* d_status, void* stream) {
  mp_batch* B = nullptr;
  if (mp_status st = mp_batch_create(ctx, count, reqs, 0, stream, &B)) return st;
  mp_status st = mp_batch_run(B, d_ll, d_status);
  if (st == MP_OK) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) st = fail(ctx, MP_ERR_CUDA, "batch: %s", cudaGetErrorString(e));
  }
  mp_batch_destroy(B);
  return st;
}

// ------------------------------------------------- planning and statistics

extern "C" mp_status mp_tile_norms(mp_ctx* ctx, int64_t n, int32_t b, const double* d_locs,
                                   mp_matern p, double* d_norms, void* stream) {
  if (!ctx || !d_locs || !d_norms) return fail(ctx, MP_ERR_ARG, "null argument");
  if (n < 1 || b < 128 || b > 1024 || b % 128) return fail(ctx, MP_ERR_ARG, "bad n or b");
  if (!valid_nu(p.nu) || !(p.range > 0.0) || !(p.sigma2 > 0.0) || !(p.nugget >= 0.0))
    return fail(ctx, MP_ERR_ARG, "bad covariance parameters (nu in (0, 16])");
  CK(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  double* d_ktab = nullptr;
  size_t kcap = 0;
  int ke0 = 0;
  if (!matern_nu_closed(p.nu)) {
    mp_status st = upload_knu_table(ctx, p.nu, &d_ktab, &kcap, &ke0, s,
                                    [](void** q, size_t bytes) { return cudaMalloc(q, bytes); });
    if (st) return st;
  }
  const int nt = (int)((n + b - 1) / b);
  std::vector<ItemGen> items;
  for (int i = 0; i < nt; ++i)
    for (int j = 0; j <= i; ++j) {
      ItemGen g{};
      g.ti = i; g.tj = j; g.locs = d_locs; g.n = n;
      g.sigma2 = p.sigma2; g.range = p.range; g.nu = p.nu; g.nugget = p.nugget;
      g.ktab = d_ktab; g.ke0 = ke0;
      items.push_back(g);
    }
  const int parts = tile_norm_parts(b);
  ItemGen* d_items = nullptr;
  double* partial = nullptr;
  cudaError_t e = cudaMalloc(&d_items, sizeof(ItemGen) * items.size());
  if (e != cudaSuccess) {
    if (d_ktab) { cudaStreamSynchronize(s); cudaFree(d_ktab); }
    return fail(ctx, MP_ERR_CUDA, "tile norms: %s", cudaGetErrorString(e));
  }
  e = cudaMalloc(&partial, sizeof(double) * items.size() * parts);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_items, items.data(), sizeof(ItemGen) * items.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_norms, 0, sizeof(double) * nt * nt, s);
  if (e == cudaSuccess) {
    launch_tile_norms(b, d_items, (int)items.size(), nt, partial, d_norms, s);
    e = cudaStreamSynchronize(s);
  }
  if (e != cudaSuccess) cudaStreamSynchronize(s);
  cudaFree(d_items);
  if (partial) cudaFree(partial);
  if (d_ktab) cudaFree(d_ktab);
  if (e != cudaSuccess) return fail(ctx, MP_ERR_CUDA, "tile norms: %s", cudaGetErrorString(e));
  return MP_OK;
}

extern "C" mp_status mp_matern_host(mp_matern p, int64_t count, const double* h_r, double* h_out) {
  if (count < 0 || (count > 0 && (!h_r || !h_out))) return MP_ERR_ARG;
  if (!valid_nu(p.nu) || !(p.range > 0.0) || !(p.sigma2 > 0.0)) {
    set_error_text("mp_matern_host: need 0 < nu <= 16, range > 0, sigma2 > 0");
    return MP_ERR_ARG;
  }
  std::vector<double> tab;
  int e0 = 0;
  const bool closed = matern_nu_closed(p.nu);
  if (!closed && matern_nu_table(p.nu, tab, &e0)) return MP_ERR_ARG;
  for (int64_t i = 0; i < count; ++i) {
    const double x = h_r[i] / p.range;
    if (closed) {
      const double poly = p.nu == 0.5 ? 1.0 : p.nu == 1.5 ? 1.0 + x : 1.0 + x + x * x / 3.0;
      h_out[i] = p.sigma2 * poly * std::exp(-x);
    } else {
      h_out[i] = p.sigma2 * matern_nu_host(tab.data(), e0, x);
    }
  }
  return MP_OK;
}

static double unit_roundoff(int dt) {
  switch (dt) {
    case F64: return 0x1p-53;
    case F32: return 0x1p-24;
    case BF16: return 0x1p-8;
    case F16: return 0x1p-11;
    default: return 0x1p-4;
  }
}

extern "C" mp_status mp_map_guarded(int32_t nt, const double* h_norms, int32_t band, uint8_t near_dt,
                                    uint8_t far_dt, double eps, uint8_t* h_map) {
  if (nt < 1 || !h_norms || !h_map || band < 0 || near_dt >= NDT || far_dt >= NDT || !(eps > 0))
    return fail(nullptr, MP_ERR_ARG, "bad map arguments");
  double tot = 0.0;
  for (int i = 0; i < nt; ++i)
    for (int j = 0; j <= i; ++j) {
      double v = h_norms[i * nt + j];
      tot += (i == j ? 1.0 : 2.0) * v * v;
    }
  const double bound = eps * sqrt(tot) / nt;
  for (int i = 0; i < nt; ++i)
    for (int j = 0; j < nt; ++j) {
      uint8_t m = 255;
      if (j == i) m = F64;
      else if (j < i) {
        if (i - j <= band) m = near_dt;
        else m = unit_roundoff(far_dt) * h_norms[i * nt + j] <= bound ? far_dt : near_dt;
      }
      h_map[i * nt + j] = m;
    }
  return MP_OK;
}

extern "C" mp_status mp_tmat_stats(mp_tmat* t, int64_t* chol_kernels, int64_t* gen_kernels,
                                   int64_t* loglik_kernels) {
  if (!t) return MP_ERR_ARG;
  if (chol_kernels) *chol_kernels = t->P.chol_kernels;
  if (gen_kernels) *gen_kernels = (t->gen_n_amax > 0 ? 1 : 0) + 1;
  if (loglik_kernels) *loglik_kernels = t->ll_kernels;
  return MP_OK;
}

namespace {
int op_class(const Launch& L) {
  const int op = L.op;
  if (op == OP_PANEL && L.stream == 0) return 8;
  switch (op) {
    case OP_POTRF_DAG: return 0;
    case OP_PANEL: return 1;
    case OP_ROUND: return 2;
    case OP_UPD64: return 3;
    case OP_UPD32: return 4;
    case OP_TC: return L.kb == F32 ? 5 : 11;
    case OP_FP8R: return 6;
    case OP_OZG: return 9;
    case OP_OZA:
    case OP_OZW: return 10;
    default: return 7;
  }
}
}  // namespace

extern "C" mp_status mp_chol_profile(mp_tmat* t, int32_t nclass, float* h_ms, int64_t* h_launches,
                                     double* h_flops) {
  if (!t || nclass < MP_PROFILE_CLASSES || !h_ms || !h_launches || !h_flops) return MP_ERR_ARG;
  Plan& P = t->P;
  if (!t->generated) return fail(P.ctx, MP_ERR_STATE, "matrix not generated or loaded");
  CK(P.ctx, cudaSetDevice(P.ctx->device));
  for (int c = 0; c < nclass; ++c) { h_ms[c] = 0.f; h_launches[c] = 0; h_flops[c] = 0.0; }
  const size_t nl = P.chol.size();
  std::vector<cudaEvent_t> ev(nl + 1);
  for (auto& e : ev) CK(P.ctx, cudaEventCreate(&e));
  CK(P.ctx, cudaEventRecord(ev[0], P.stream));
  for (size_t l = 0; l < nl; ++l) {
    run_launch(P, P.chol[l], P.stream);
    cudaEventRecord(ev[l + 1], P.stream);
  }
  cudaError_t e = cudaStreamSynchronize(P.stream);
  const double b = P.b;
  for (size_t l = 0; l < nl && e == cudaSuccess; ++l) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev[l], ev[l + 1]);
    const Launch& L = P.chol[l];
    const int c = op_class(L);
    h_ms[c] += ms;
    if (c == 7 && L.count == 0) continue;
    h_launches[c] += 1;
    switch (L.op) {
      case OP_POTRF_DAG: h_flops[c] += L.count * 2.0 * b * b * b / 3.0; break;  // POTRF + L^{-1}
      case OP_PANEL: h_flops[c] += L.count * b * b * b; break;  // incl. L_kk^{-T} rows
      case OP_OZG: h_flops[c] += L.count * b * b * b; break;    // the solve it stands for
      case OP_UPD64:
      case OP_UPD32: {
        const ItemUpd* it = reinterpret_cast<const ItemUpd*>(P.h_items.data() + L.off);
        for (int q = 0; q < L.count; ++q) h_flops[c] += it[q].syrk ? b * b * (b + 1) : 2.0 * b * b * b;
        break;
      }
      case OP_TC: {
        const ItemTC* it = reinterpret_cast<const ItemTC*>(P.h_items.data() + L.off);
        for (int q = 0; q < L.count; ++q) h_flops[c] += it[q].syrk ? b * b * (b + 1) : 2.0 * b * b * b;
        break;
      }
      default: break;
    }
  }
  for (auto& ev_ : ev) cudaEventDestroy(ev_);
  if (e != cudaSuccess) return fail(P.ctx, MP_ERR_CUDA, "profile: %s", cudaGetErrorString(e));
  P.factored = true;
  return check_launch(P.ctx);
}
