// FP64 kernels of the factorisation: the diagonal tile's Cholesky and the
// panel triangular solve (the `chol` / `forwardsolve` steps of Sec. 6.2 done
// tile by tile, as in the tiled extension of Sec. 7).
//
// The FP64 diagonal tile (b x b, b a multiple of 64) is factored by a
// blocked right-looking Cholesky over 16 x 16 or 32 x 32 blocks, run as a task graph
// by one persistent launch (k_potrf_dag): per block column k, one CTA
// factors block (k, k) in shared memory (adding 2 sum log L_tt to the
// log-determinant partials, flagging the first pivot that is not > 0, and
// forming the block's inverse), the blocks below are solved as
// X = A Dinv_k^T, and the trailing blocks are updated, A -= X X^T, each
// task starting as soon as its input blocks are final.
// The panel solve X = A_ik L_kk^{-T} keeps 16 rows of the panel tile in
// shared memory in float64 and sweeps L_kk's 32-column blocks left to right:
// acc = A[:, c] - X[:, <c] L[c, <c]^T, then X[:, c] = acc Dinv_c^T, with
// Dinv_c^T read from the diagonal 32-block of W = L_kk^{-T} (the diagonal
// blocks of a triangular matrix's inverse are the inverses of its diagonal
// blocks).  The
// float64 result goes to a scratch slot; `panel_round` then rounds it once
// into the tile's format (E4M3: scale from the tile's amax) and into the
// tile's shadow copy, the operand form that lower-precision updates read.
//
// GB300 has little FP64 throughput (about 1.2 TFLOP/s of DFMA), so these
// kernels are bound by the FP64 pipe, not by memory.
#include <algorithm>
#include <vector>

#include "mp_device.cuh"

namespace mp {

namespace {

constexpr int NB = 32;   // column block of the panel solve's sweep

// The task graph is instantiated for blocks DB = 16 and 32.  A block
// product runs on 256 threads, DJ outputs each, DTX threads along a row.
template <int DB>
struct DagShape {
  static_assert(DB == 16 || DB == 32, "task-graph block must be 16 or 32");
  static constexpr int DJ = DB * DB / 256;
  static constexpr int DTX = DB / DJ;
};

// Block (k, k) in S: Cholesky factor in place (lower part) and the block's
// inverse Y = L^{-1} in R, in one right-looking sweep over column pairs run
// as a two-stage pipeline.  In iteration p columns 2p and 2p + 1 of L are
// final; warp 0 then finishes the next pair (dag_pair): it applies columns
// 2p and 2p + 1 to columns n = 2p + 2 and n + 1 and takes both pivots from
// one rsqrt, because the second pivot is a ratio of leading minors,
// d_{n+1} = delta / a with a = A_nn, delta = A_nn A_{n+1,n+1} - A_{n+1,n}^2
// (the updated entries): so the sequential chain per pair of columns is
// two FMAs, the minor, one rsqrt and two multiplications, where a column
// at a time took one FMA, one rsqrt and one multiplication per column.
// Meanwhile warps 1-3 and 5-7 apply columns 2p and 2p + 1 to the columns
// beyond 2p + 3 and advance the inverse by the pair before:
// Y[c, .] = R[c, .] / L_cc, Y[c+1, .] = (R[c+1, .] - L_{c+1,c} Y[c, .]) /
// L_{c+1,c+1} (c = 2p - 2), then R[r, .] -= L_rc Y[c, .] + L_{r,c+1}
// Y[c+1, .] for the rows below.  Warp 4 shares warp 0's scheduler and sits
// the sweep out (the FP64 pipe issues one warp instruction per 64 cycles
// per scheduler, so any FP64 instruction there lengthens the chain).
// Writes L and the inverse to global memory; info gets the first pivot
// that is not > 0.

// Largest number of elements one pair of the sweep updates: the trailing
// triangle rows 2p+4.. on columns 2p+4..r and the inverse rows 2p.. on
// columns < 2p.
template <int DB>
__host__ __device__ constexpr int sweep_work_max() {
  int mx = 0;
  for (int p = 0; p < DB / 2; ++p) {
    const int m = DB - 4 - 2 * p;
    const int t = (m > 0 ? m * (m + 1) / 2 : 0) + (p >= 1 ? (DB - 2 * p) * 2 * p : 0);
    mx = t > mx ? t : mx;
  }
  return mx;
}

// Warp 0: columns n and n + 1 (n even) of the block factor.  Their entries
// in S carry the updates of the columns before n - 2; with PREV the final
// columns n - 2 and n - 1 are applied here.  Lanes 0-15 take column n,
// lanes 16-31 column n + 1, one row per lane and 16-row slot.  With v the
// updated column n, v' the updated column n + 1, a = v_n, beta = v_{n+1},
// delta = a v'_{n+1} - beta^2:
//   L_in      = v_i rsqrt(a)
//   L_{i,n+1} = (a v'_i - beta v_i) rsqrt(a) rsqrt(delta)
// (L_{n+1,n+1} = delta rsqrt(a) rsqrt(delta) = sqrt(delta / a)); lanes 0 and
// 1 form rsqrt(a) and rsqrt(delta) in the same instructions.  rps gets
// 1 / L_nn = rsqrt(a) and rsqrt(a) rsqrt(delta), pa gets a: 1 / L_{n+1,n+1}
// = a rsqrt(a) rsqrt(delta) is formed by the inverse's update, off the chain.
// A pivot that is not > 0 leaves L_nn or L_{n+1,n+1} NaN (rsqrt of a
// negative number, or 0 * inf), and every later pivot with it.
template <int DB, bool PREV>
__device__ __forceinline__ void dag_pair(double (*S)[DB + 1], int n, double* rps, double* pa) {
  constexpr int NS = DB / 16;                  // 16-row slots per lane
  const int lane = threadIdx.x & 31, hi = lane >> 4, col = n + hi;
  double g0 = 0.0, g1 = 0.0;
  if (PREV) { g0 = S[col][n - 2]; g1 = S[col][n - 1]; }
  double v[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const int i = (lane & 15) + 16 * s;
    double x = 0.0;
    if (16 * s + 16 > n) {                     // uniform: the slot reaches row n
      x = S[i][col];
      if (PREV) x = fma(-S[i][n - 1], g1, fma(-S[i][n - 2], g0, x));
    }
    v[s] = x;
  }
  const int r0 = n & 15;                       // rows n and n + 1 share a slot
  const double vs = (NS == 1 || n < 16) ? v[0] : v[NS - 1];
  const double a = __shfl_sync(0xffffffffu, vs, r0);
  const double beta = __shfl_sync(0xffffffffu, vs, r0 + 1);
  const double gam = __shfl_sync(0xffffffffu, vs, r0 + 17);
  const double delta = fma(a, gam, -(beta * beta));
  const double y = rsqrt((lane & 1) ? delta : a);
  const double rp = __shfl_sync(0xffffffffu, y, 0);
  const double rq = __shfl_sync(0xffffffffu, y, 1);
  const double m = rp * rq;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    if (16 * s + 16 <= n) continue;            // uniform
    const int i = (lane & 15) + 16 * s;
    const double u = __shfl_xor_sync(0xffffffffu, v[s], 16);   // the other column, row i
    const double w = fma(a, v[s], -(beta * u));
    const double out = (hi ? w : v[s]) * (hi ? m : rp);
    if (i >= col) S[i][col] = out;
  }
  if (lane == 0) {
    rps[n] = rp;
    rps[n + 1] = m;
    pa[n + 1] = a;
  }
}

// The sweep's warps synchronise among themselves (named barrier 2, 224
// threads); warp 4 waits at the end.
template <int DB>
__device__ void dag_factor(double (*S)[DB + 1], double (*R)[DB + 1], double* Tk, int b,
                           double* dinv, long long* info, long long row0, const uint16_t* tri) {
  const int tid = threadIdx.x, warp = tid >> 5;
  constexpr int NO = 192;                        // threads of warps 1-3 and 5-7
  constexpr int NP = DB / 2;                     // column pairs
  __shared__ double rps[DB];                     // see dag_pair
  __shared__ double pa[DB];
  for (int e = tid; e < DB * DB; e += blockDim.x) R[e / DB][e % DB] = (e / DB == e % DB) ? 1.0 : 0.0;
  if (tid < 32) dag_pair<DB, false>(S, 0, rps, pa);
  __syncthreads();
  if (warp != 4) for (int p = 0; p < NP; ++p) {
    if (p) asm volatile("bar.sync 2, 224;" ::: "memory");
    if (tid < 32) {
      if (p + 1 < NP) dag_pair<DB, true>(S, 2 * p + 2, rps, pa);
    } else {
      const int t = tid < 128 ? tid - 32 : tid - 64;
      const int c = 2 * p - 2;                   // the pair whose rows of Y finish here
      if (p >= 1 && t < c + 2) {
        const double y0 = R[c][t] * rps[c];
        R[c][t] = y0;
        R[c + 1][t] = (R[c + 1][t] - S[c + 1][c] * y0) * (pa[c + 1] * rps[c + 1]);
      }
      asm volatile("bar.sync 1, %0;" ::"r"(NO));
      // compact enumeration (the FP64 pipe charges a warp instruction in
      // full however many lanes it masks): trailing rows 2p+4.. on columns
      // 2p+4..r through the triangle table, then inverse rows 2p.. on
      // columns < 2p
      const int m = DB - 4 - 2 * p;
      const int ntri = m > 0 ? m * (m + 1) / 2 : 0;
      const int w2 = 2 * p;
      const int total = ntri + (p >= 1 ? (DB - w2) * w2 : 0);
      const float rc = p >= 1 ? 1.f / (float)w2 : 0.f;
      // at most UPT elements per thread (total <= UPT * 192); the updates of
      // one pair touch distinct entries and read only columns 2p - 2 .. 2p + 1
      // and rows 2p - 2, 2p - 1 of R, so all operands are loaded before any store
      constexpr int UPT = DB == 32 ? 3 : 1;
      static_assert(sweep_work_max<DB>() <= UPT * NO, "sweep elements exceed the update threads");
      double* dst[UPT];
      double x0[UPT], x1[UPT], x2[UPT], x3[UPT], x4[UPT];
#pragma unroll
      for (int u = 0; u < UPT; ++u) {
        const int e = t + u * NO;
        dst[u] = nullptr;
        if (e < ntri) {
          const int rr = tri[e] >> 8, cc = tri[e] & 0xff;
          const int r = w2 + 4 + rr, j = w2 + 4 + cc;
          dst[u] = &S[r][j];
          x1[u] = S[r][w2];
          x2[u] = S[j][w2];
          x3[u] = S[r][w2 + 1];
          x4[u] = S[j][w2 + 1];
        } else if (e < total) {
          const int q = e - ntri;
          const int qr = (int)(((float)q + 0.5f) * rc);   // q / 2p, exact for q < 2^12
          const int r = w2 + qr, j = q - qr * w2;
          dst[u] = &R[r][j];
          x1[u] = S[r][w2 - 2];
          x2[u] = R[w2 - 2][j];
          x3[u] = S[r][w2 - 1];
          x4[u] = R[w2 - 1][j];
        }
        if (dst[u]) x0[u] = *dst[u];
      }
#pragma unroll
      for (int u = 0; u < UPT; ++u)
        if (dst[u]) *dst[u] = x0[u] - x1[u] * x2[u] - x3[u] * x4[u];
    }
  }
  __syncthreads();
  if (tid < DB) {
    // rows DB - 2 and DB - 1 of Y (the last pair)
    const int c = DB - 2;
    const double y0 = R[c][tid] * rps[c];
    R[c][tid] = y0;
    R[c + 1][tid] = (R[c + 1][tid] - S[c + 1][c] * y0) * (pa[c + 1] * rps[c + 1]);
  }
  // a pivot d that is not > 0 leaves L_cc NaN (see dag_pair): the first
  // diagonal entry that is not > 0 is the first failed pivot
  if (tid < DB && !(S[tid][tid] > 0.0)) atomicMin(info, row0 + tid + 1);
  __syncthreads();
  // the inverse first: it is what the tasks waiting on this block read
  for (int e = tid; e < DB * DB; e += blockDim.x) dinv[e] = R[e / DB][e % DB];
  for (int e = tid; e < DB * DB; e += blockDim.x) {
    const int r = e / DB, c = e % DB;
    if (c <= r) Tk[(int64_t)r * b + c] = S[r][c];
  }
}

// 2 sum log L_tt of the block in S: one log per lane of warp 0 (lanes past
// the block add zero), fixed-order butterfly sum.
template <int DB>
__device__ void dag_logdet(double (*S)[DB + 1], double* ldpart) {
  if (threadIdx.x < 32) {
    double lg = threadIdx.x < DB ? log(S[threadIdx.x][threadIdx.x]) : 0.0;
    for (int o = 16; o > 0; o >>= 1) lg += __shfl_xor_sync(0xffffffffu, lg, o);
    if (threadIdx.x == 0) *ldpart = 2.0 * lg;
  }
}

// X = A Dinv^T for a DB x DB block (Dinv lower triangular): X[i][j] =
// sum_{t <= j} A[i][t] Dinv[j][t], in order of t (terms past j multiply
// Dinv's exact zeros above the diagonal and leave the sum unchanged).
// Output q of thread tid is element solve_rc(tid, q).  DB = 16: warp w
// takes the column pair p(w) = w (w < 4) or 11 - w, 16 rows each, and stops
// at t = 2p + 1 (a bound uniform over the warp): the FP64 pipe charges a
// warp instruction in full however many lanes it masks, so skipping the
// zeros by whole warps takes 72 FMA instructions instead of 128, and
// warps s and s + 4 (one scheduler) get 18 of them each.
// DB = 32: thread (ty, tx) takes row ty, columns tx + DTX q.
template <int DB>
__device__ __forceinline__ void solve_rc(int tid, int q, int& r, int& c) {
  if constexpr (DB == 16) {
    const int w = tid >> 5, l = tid & 31, p = w < 4 ? w : 11 - w;
    r = l & 15;
    c = 2 * p + (l >> 4);
  } else {
    constexpr int DTX = DagShape<DB>::DTX;
    r = tid / DTX;
    c = tid % DTX + DTX * q;
  }
}

template <int DB>
__device__ __forceinline__ void dag_solve(const double (*Ab)[DB + 1], const double (*D)[DB + 1],
                                          double out[DagShape<DB>::DJ]) {
  constexpr int DJ = DagShape<DB>::DJ, DTX = DagShape<DB>::DTX;
  if constexpr (DB == 16) {
    const int w = threadIdx.x >> 5, p = w < 4 ? w : 11 - w;
    int r, c;
    solve_rc<DB>(threadIdx.x, 0, r, c);
    double acc = 0.0;
    for (int q = 0; q <= 2 * p + 1; ++q) acc += Ab[r][q] * D[c][q];
    out[0] = acc;
  } else {
    const int ty = threadIdx.x / DTX, tx = threadIdx.x % DTX;
    double acc[DJ] = {};
    // DJ independent accumulation chains; D[c][q] = 0 for q > c, so column
    // group j stops at q = DTX j + DTX - 1 (a bound uniform over the warp)
#pragma unroll 4
    for (int q = 0; q < DB; ++q) {
      const double a = Ab[ty][q];
#pragma unroll
      for (int j = 0; j < DJ; ++j)
        if (q <= DTX * j + DTX - 1) acc[j] += a * D[tx + DTX * j][q];
    }
#pragma unroll
    for (int j = 0; j < DJ; ++j) out[j] = acc[j];
  }
}

// One persistent launch factors the FP64 diagonal tile of every item as a
// task graph over its DB x DB blocks (nb = b / DB) and forms
// W = L^{-T} (the operand of the panel products and of the solves):
//   F(0)       factor block (0, 0): L_00, Dinv_0 = L_00^{-1}, log-det part
//   G(k)       k >= 1, the critical chain: L_{k,k-1} = A_{k,k-1} Dinv_{k-1}^T
//              (published at once), A_kk -= L_{k,k-1} L_{k,k-1}^T (lower
//              part), then factor block (k, k)
//   T(r, k)    r > k + 1:  L_rk = A_rk Dinv_k^T
//   U(r, c, k) k < c <= r, (r, c) != (k+1, k+1):  A_rc -= L_rk L_ck^T
// and for Y = L^{-1} by block rows (Y_kk = Dinv_k, Y_rj = Dinv_r R_rj with
// R_rj = -sum_{k=j}^{r-1} L_rk Y_kj), stored transposed as W:
//   E(r, k, j) r > k >= j:  W_jr -= W_jk L_rk^T   (R_rj -= L_rk Y_kj)
//   V(r, j)    r > j:       W_jr = W_jr Dinv_r^T   (Y_rj = Dinv_r R_rj)
// F and G also write W_kk = Dinv_k^T (the blocks of W left of it are zero
// from the plan's creation on).
// ver[r nb + c] counts the operations finished on block (r, c) of the
// factor (its c updates, then the factorisation or solve); ver[nb^2 +
// j nb + r] those on block (j, r) of W (its r - j updates, then the solve;
// 1 once the diagonal block W_jj is written).
// CTAs take tasks by an atomic ticket in a fixed topological order (every
// task's inputs come earlier in the order), so a task only ever waits on
// tasks that running CTAs have already taken: the schedule cannot
// deadlock, whatever the number of co-resident CTAs.  Blocks written by
// other CTAs are read through L2 (ld.global.cg); every wait is bounded and
// reports through the error word.
template <int DB>
__global__ void __launch_bounds__(256) k_potrf_dag(Arena A, const ItemPotrf* __restrict__ items,
                                                   int count, const DagTask* __restrict__ tasks,
                                                   int ntasks, int* ticket, double* ldparts,
                                                   long long* info) {
  constexpr int DJ = DagShape<DB>::DJ, DTX = DagShape<DB>::DTX;
  __shared__ double S0[DB][DB + 1];
  __shared__ double S1[DB][DB + 1];
  __shared__ double S2[DB][DB + 1];
  __shared__ int s_t, s_ok, s_ok2;
  // lower triangle of a DB x DB block in row order: entry e -> (row, col)
  __shared__ uint16_t tri[DB * (DB + 1) / 2];
  const int b = A.b, nb = b / DB, tid = threadIdx.x;
  const int ty = tid / DTX, tx = tid % DTX;
  const int total = ntasks * count;
  for (int r = 0; r < DB; ++r)
    for (int c = tid; c <= r; c += blockDim.x) tri[r * (r + 1) / 2 + c] = (uint16_t)(r << 8 | c);
  for (;;) {
    if (tid == 0) s_t = atomicAdd(ticket, 1);
    __syncthreads();
    const int t = s_t;
    if (t >= total) break;
    const ItemPotrf it = items[t % count];
    const DagTask tk = tasks[t / count];
    const int r = tk.r, c = tk.c, k = tk.k;
    int* ver = it.ver;
    int* wv = ver + nb * nb;
    // chain trace (tracing on, chain task, thread 0 only)
    unsigned long long* tr = (A.trace && (tk.op == 0 || tk.op == 3) && tid == 0)
                                 ? A.trace + (int64_t)(it.ldslot + k) * TRACE_WORDS : nullptr;
    chain_stamp(tr, 0);
    if (tid == 0) {
      bool ok;
      if (tk.op == 0) ok = dag_wait(&ver[0], 0, A.err, A.wait_polls);
      else if (tk.op == 3)   // G(k): blocks (k, k-1) and (k, k) updated up to k-2 (F(k-1) below)
        ok = dag_wait(&ver[k * nb + k - 1], k - 1, A.err, A.wait_polls) && dag_wait(&ver[k * nb + k], k - 1, A.err, A.wait_polls);
      else if (tk.op == 1) ok = dag_wait(&ver[k * nb + k], k + 1, A.err, A.wait_polls) && dag_wait(&ver[r * nb + k], k, A.err, A.wait_polls);
      else if (tk.op == 2)
        ok = dag_wait(&ver[r * nb + k], k + 1, A.err, A.wait_polls) && dag_wait(&ver[c * nb + k], k + 1, A.err, A.wait_polls) &&
             dag_wait(&ver[r * nb + c], k, A.err, A.wait_polls);
      else if (tk.op == 4)   // V(r, j = c): F(r) done, W_jr has its r - j updates
        ok = dag_wait(&ver[r * nb + r], r + 1, A.err, A.wait_polls) && dag_wait(&wv[c * nb + r], r - c, A.err, A.wait_polls);
      else                   // E(r, k, j = c): L_rk, W_jk final; the previous update of W_jr
        ok = dag_wait(&ver[r * nb + k], k + 1, A.err, A.wait_polls) &&
             (k == c ? dag_wait(&wv[c * nb + c], 1, A.err, A.wait_polls) : dag_wait(&wv[c * nb + k], k - c + 1, A.err, A.wait_polls)) &&
             dag_wait(&wv[c * nb + r], k - c, A.err, A.wait_polls);
      if (!ok) atomicExch(A.err, 1);
      s_ok = ok;
      chain_stamp(tr, 1);
      if (tk.op == 0) chain_stamp(tr, 2);
    }
    __syncthreads();
    if (!s_ok) break;
    double* T = tile_ptr<double>(A, it.tile);
    if (tk.op == 0 || tk.op == 3) {
      double* Tk = T + (int64_t)k * DB * b + k * DB;
      for (int e = tid; e < DB * DB; e += blockDim.x) S2[e / DB][e % DB] = __ldcg(Tk + (int64_t)(e / DB) * b + e % DB);
      if (tk.op == 3) {
        // L_{k,k-1} = A_{k,k-1} Dinv_{k-1}^T, published before the rest; the
        // two blocks of A are final before F(k-1) ends, so they are read
        // first and only Dinv_{k-1} waits for it
        double* Tl = T + (int64_t)k * DB * b + (k - 1) * DB;
        const double* D = it.dinv + (int64_t)(k - 1) * DB * DB;
        for (int e = tid; e < DB * DB; e += blockDim.x) S0[e / DB][e % DB] = __ldcg(Tl + (int64_t)(e / DB) * b + e % DB);
        if (tid == 0) {
          s_ok2 = dag_wait(&ver[(k - 1) * nb + k - 1], k, A.err, A.wait_polls);
          if (!s_ok2) atomicExch(A.err, 1);
          chain_stamp(tr, 2);
        }
        __syncthreads();
        if (!s_ok2) break;
        for (int e = tid; e < DB * DB; e += blockDim.x) S1[e / DB][e % DB] = __ldcg(D + e);
        __syncthreads();
        double out[DJ];
        dag_solve<DB>(S0, S1, out);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < DJ; ++j) {
          int rr, cc;
          solve_rc<DB>(tid, j, rr, cc);
          S0[rr][cc] = out[j];
          Tl[(int64_t)rr * b + cc] = out[j];
        }
        __syncthreads();
        chain_stamp(tr, 3);
        // published by the last thread, which has no share of the update
        // below when DB = 16 (136 entries): the release overlaps the update
        if (tid == blockDim.x - 1) st_release(&ver[k * nb + k - 1], k);
        // A_kk -= X X^T on the lower triangle (DB (DB + 1) / 2 entries, table order)
        for (int e = tid; e < DB * (DB + 1) / 2; e += blockDim.x) {
          const int rr = tri[e] >> 8, cc = tri[e] & 0xff;
          double a0 = 0.0, a1 = 0.0;
#pragma unroll 8
          for (int q = 0; q < DB; q += 2) {
            a0 += S0[rr][q] * S0[cc][q];
            a1 += S0[rr][q + 1] * S0[cc][q + 1];
          }
          S2[rr][cc] -= a0 + a1;
        }
      }
      __syncthreads();
      if (tk.op == 0) chain_stamp(tr, 3);
      chain_stamp(tr, 4);
      dag_factor<DB>(S2, S1, Tk, b, it.dinv + (int64_t)k * DB * DB, info + it.mat,
                     it.row0 + (long long)k * DB, tri);
    } else if (tk.op == 1) {
      // L_rk = A_rk Dinv_k^T (Dinv_k lower triangular)
      double* Tr = T + (int64_t)r * DB * b + k * DB;
      const double* D = it.dinv + (int64_t)k * DB * DB;
      for (int e = tid; e < DB * DB; e += blockDim.x) {
        S0[e / DB][e % DB] = __ldcg(Tr + (int64_t)(e / DB) * b + e % DB);
        S1[e / DB][e % DB] = __ldcg(D + e);
      }
      __syncthreads();
      double out[DJ];
      dag_solve<DB>(S0, S1, out);
#pragma unroll
      for (int j = 0; j < DJ; ++j) {
        int rr, cc;
        solve_rc<DB>(tid, j, rr, cc);
        Tr[(int64_t)rr * b + cc] = out[j];
      }
    } else if (tk.op == 4) {
      // W_jr = W_jr Dinv_r^T
      double* Wb = it.w + (int64_t)c * DB * b + r * DB;
      const double* D = it.dinv + (int64_t)r * DB * DB;
      for (int e = tid; e < DB * DB; e += blockDim.x) {
        S0[e / DB][e % DB] = __ldcg(Wb + (int64_t)(e / DB) * b + e % DB);
        S1[e / DB][e % DB] = __ldcg(D + e);
      }
      __syncthreads();
      double out[DJ];
      dag_solve<DB>(S0, S1, out);
#pragma unroll
      for (int j = 0; j < DJ; ++j) {
        int rr, cc;
        solve_rc<DB>(tid, j, rr, cc);
        const int64_t o = (int64_t)c * DB * b + r * DB + (int64_t)rr * b + cc;
        Wb[(int64_t)rr * b + cc] = out[j];
        if (it.whi) {
          const float h = (float)out[j];
          it.whi[o] = h;
          it.wlo[o] = (float)(out[j] - (double)h);
        }
      }
    } else if (tk.op == 5) {
      // W_jr -= W_jk L_rk^T (the first update, k = j, starts from zero)
      const double* Wj = it.w + (int64_t)c * DB * b + k * DB;
      const double* Lr = T + (int64_t)r * DB * b + k * DB;
      double* Wb = it.w + (int64_t)c * DB * b + r * DB;
      for (int e = tid; e < DB * DB; e += blockDim.x) {
        S0[e / DB][e % DB] = __ldcg(Wj + (int64_t)(e / DB) * b + e % DB);
        S1[e / DB][e % DB] = __ldcg(Lr + (int64_t)(e / DB) * b + e % DB);
      }
      double cur[DJ];
#pragma unroll
      for (int j = 0; j < DJ; ++j) cur[j] = k == c ? 0.0 : __ldcg(Wb + (int64_t)ty * b + tx + DTX * j);
      __syncthreads();
      double acc[DJ] = {}, acc2[DJ] = {};
      for (int q = 0; q < DB; q += 2) {
        const double a = S0[ty][q], a2 = S0[ty][q + 1];
#pragma unroll
        for (int j = 0; j < DJ; ++j) {
          acc[j] += a * S1[tx + DTX * j][q];
          acc2[j] += a2 * S1[tx + DTX * j][q + 1];
        }
      }
#pragma unroll
      for (int j = 0; j < DJ; ++j) Wb[(int64_t)ty * b + tx + DTX * j] = cur[j] - (acc[j] + acc2[j]);
    } else {
      // A_rc -= L_rk L_ck^T
      const double* Lr = T + (int64_t)r * DB * b + k * DB;
      const double* Lc = T + (int64_t)c * DB * b + k * DB;
      double* Trc = T + (int64_t)r * DB * b + c * DB;
      for (int e = tid; e < DB * DB; e += blockDim.x) {
        S0[e / DB][e % DB] = __ldcg(Lr + (int64_t)(e / DB) * b + e % DB);
        S1[e / DB][e % DB] = __ldcg(Lc + (int64_t)(e / DB) * b + e % DB);
      }
      double cur[DJ];
#pragma unroll
      for (int j = 0; j < DJ; ++j) cur[j] = __ldcg(Trc + (int64_t)ty * b + tx + DTX * j);
      __syncthreads();
      double acc[DJ] = {}, acc2[DJ] = {};
      for (int q = 0; q < DB; q += 2) {
        const double a = S0[ty][q], a2 = S0[ty][q + 1];
#pragma unroll
        for (int j = 0; j < DJ; ++j) {
          acc[j] += a * S1[tx + DTX * j][q];
          acc2[j] += a2 * S1[tx + DTX * j][q + 1];
        }
      }
#pragma unroll
      for (int j = 0; j < DJ; ++j) Trc[(int64_t)ty * b + tx + DTX * j] = cur[j] - (acc[j] + acc2[j]);
    }
    __syncthreads();
    if (tid == 0) {
      chain_stamp(tr, 5);
      if (tk.op == 4) st_release(&wv[c * nb + r], r - c + 1);
      else if (tk.op == 5) st_release(&wv[c * nb + r], k - c + 1);
      else {
        const int blk = (tk.op == 0 || tk.op == 3) ? k * nb + k : tk.op == 1 ? r * nb + k : r * nb + c;
        st_release(&ver[blk], k + 1);
      }
      chain_stamp(tr, 6);
    }
    // off the critical chain, after publishing: W_kk = Dinv_k^T (published on
    // its own counter, read by the E(r, k, k)) and the log-determinant part
    // (the blocks of W left of W_kk are zero from the plan's creation:
    // nothing writes them)
    if (tk.op == 0 || tk.op == 3) {
      for (int e = tid; e < DB * DB; e += blockDim.x) {
        const int64_t o = (int64_t)k * DB * b + (int64_t)(e / DB) * b + k * DB + e % DB;
        const double v = S1[e % DB][e / DB];
        it.w[o] = v;
        if (it.whi) {
          const float h = (float)v;
          it.whi[o] = h;
          it.wlo[o] = (float)(v - (double)h);
        }
      }
      __syncthreads();
      if (tid == 0) st_release(&wv[k * nb + k], 1);
      dag_logdet<DB>(S2, ldparts + it.ldslot + k);
      chain_stamp(tr, 7);
    }
  }
}

constexpr int PK = 32;     // K chunk of L staged in shared memory

// Persistent over work units (panel tile, 16-row block): CTA u processes
// units u, u + gridDim.x, ...  The chunks of L_kk are double-buffered: the
// next chunk is fetched into registers while the current one is used.
template <int PR>
__global__ void __launch_bounds__(128) k_panel_trsm(Arena A, const ItemPanel* __restrict__ items,
                                                    int units) {
  constexpr int LPR = 128 / PR;                    // threads per row
  constexpr int NQ = NB / LPR;                     // columns of a 32-block per thread
  extern __shared__ double sm[];
  const int b = A.b, tid = threadIdx.x;
  double* X = sm;                                  // [PR][b]
  double* Ls = X + PR * b;                         // 2 x [NB][PK+1]
  double* Dv = Ls + 2 * NB * (PK + 1);             // [NB][NB+1]
  double* Ac = Dv + NB * (NB + 1);                 // [PR][NB+1]
  const int r = tid / LPR, cx = tid % LPR;
  const int per_tile = b / PR;
  __shared__ double red[4];
  for (int u = blockIdx.x; u < units; u += gridDim.x) {
    const ItemPanel it = items[u / per_tile];
    const int r0 = (u % per_tile) * PR;
    const TileRef ref = A.tiles[it.tile];
    const char* src = tile_bytes(A, it.tile);
    const double s_in = A.scale[it.tile];
    const double* L = tile_ptr<double>(A, it.diag);
    __syncthreads();                               // previous unit done with X
    for (int e = tid; e < PR * b; e += blockDim.x)
      X[e] = load_f64(src, ref.dt, (int64_t)r0 * b + e) * s_in;
    for (int cb = 0; cb < b / NB; ++cb) {
      // Dv[i][j] = Dinv_cb[i][j] = W[cb NB + j][cb NB + i]
      for (int e = tid; e < NB * NB; e += blockDim.x)
        Dv[(e % NB) * (NB + 1) + e / NB] = it.w[(int64_t)(cb * NB + e / NB) * b + cb * NB + e % NB];
      __syncthreads();
      double acc[NQ], acc2[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) { acc[q] = X[r * b + cb * NB + cx + LPR * q]; acc2[q] = 0.0; }
      const int ch0 = 0;
      const int nch = cb * NB / PK;
      double pre[NB * PK / 128];
      if (nch > 0) {
#pragma unroll
        for (int k = 0; k < NB * PK / 128; ++k) {
          const int e = tid + 128 * k, rr = e / PK, tt = e % PK;
          pre[k] = L[(int64_t)(cb * NB + rr) * b + ch0 * PK + tt];
        }
#pragma unroll
        for (int k = 0; k < NB * PK / 128; ++k) {
          const int e = tid + 128 * k, rr = e / PK, tt = e % PK;
          Ls[rr * (PK + 1) + tt] = pre[k];
        }
        __syncthreads();
      }
      for (int ch = 0; ch < nch; ++ch) {
        const double* Lc = Ls + (ch & 1) * NB * (PK + 1);
        if (ch + 1 < nch) {
#pragma unroll
          for (int k = 0; k < NB * PK / 128; ++k) {
            const int e = tid + 128 * k, rr = e / PK, tt = e % PK;
            pre[k] = L[(int64_t)(cb * NB + rr) * b + (ch0 + ch + 1) * PK + tt];
          }
        }
        const double* Xr = X + r * b + (ch0 + ch) * PK;
#pragma unroll 8
        for (int tt = 0; tt < PK; tt += 2) {
          const double x0 = Xr[tt], x1 = Xr[tt + 1];
#pragma unroll
          for (int q = 0; q < NQ; ++q) {
            acc[q] -= x0 * Lc[(cx + LPR * q) * (PK + 1) + tt];
            acc2[q] -= x1 * Lc[(cx + LPR * q) * (PK + 1) + tt + 1];
          }
        }
        if (ch + 1 < nch) {
          double* Ln = Ls + ((ch + 1) & 1) * NB * (PK + 1);
#pragma unroll
          for (int k = 0; k < NB * PK / 128; ++k) {
            const int e = tid + 128 * k, rr = e / PK, tt = e % PK;
            Ln[rr * (PK + 1) + tt] = pre[k];
          }
        }
        __syncthreads();
      }
#pragma unroll
      for (int q = 0; q < NQ; ++q) Ac[r * (NB + 1) + cx + LPR * q] = acc[q] + acc2[q];
      __syncthreads();
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int c = cx + LPR * q;
        double v0 = 0.0, v1 = 0.0;
        int t = 0;
        for (; t + 1 <= c; t += 2) {
          v0 += Ac[r * (NB + 1) + t] * Dv[c * (NB + 1) + t];
          v1 += Ac[r * (NB + 1) + t + 1] * Dv[c * (NB + 1) + t + 1];
        }
        if (t <= c) v0 += Ac[r * (NB + 1) + t] * Dv[c * (NB + 1) + t];
        X[r * b + cb * NB + c] = v0 + v1;
      }
      __syncthreads();
    }
    double mx = 0.0;
    for (int e = tid; e < PR * b; e += blockDim.x) {
      const double v = X[e];
      it.x[(int64_t)r0 * b + e] = v;
      mx = fmax(mx, fabs(v));
    }
    mx = warp_max(mx);
    if ((tid & 31) == 0) red[tid >> 5] = mx;
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < 4; ++w) mx = fmax(mx, red[w]);
      atomic_max_pos(&A.amax[it.amax], mx);
    }
  }
}

__global__ void __launch_bounds__(256) k_panel_round(Arena A, const ItemRound* __restrict__ items) {
  const ItemRound it = items[blockIdx.x];
  const int b = A.b;
  const int dt = A.tiles[it.tile].dt;
  const double amax = amax_value(&A.amax[it.amax]);
  const double s = dt == E4M3 ? e4m3_scale(amax) : 1.0;
  char* dst = tile_bytes(A, it.tile);
  // amax of the stored (rounded) tile = the rounded amax (rounding is monotone)
  double stored_amax = amax;
  if (dt == F32) stored_amax = (double)__double2float_rn(amax);
  else if (dt == BF16) stored_amax = (double)__bfloat162float(__double2bfloat16(amax));
  else if (dt == F16) stored_amax = (double)__half2float(__double2half(amax));
  int sdt[MAX_SHADOW];
  double ss[MAX_SHADOW];
  char* sdst[MAX_SHADOW];
#pragma unroll
  for (int q = 0; q < MAX_SHADOW; ++q) {
    sdt[q] = it.shadow[q] >= 0 ? A.tiles[it.shadow[q]].dt : -1;
    sdst[q] = it.shadow[q] >= 0 ? tile_bytes(A, it.shadow[q]) : nullptr;
    ss[q] = sdt[q] == E4M3 ? e4m3_scale(stored_amax) : 1.0;
  }
  float* hi = it.hi >= 0 ? tile_ptr<float>(A, it.hi) : nullptr;
  float* lo = it.lo >= 0 ? tile_ptr<float>(A, it.lo) : nullptr;
  const int64_t r0 = (int64_t)blockIdx.y * 16 * b;
  // one float64 rounding per entry; the shadow copies and the TF32 split
  // derive from the stored value, which is exact in FP32 (GB300 runs FP64
  // conversions on its narrow FP64 pipe)
  float sss[MAX_SHADOW];
#pragma unroll
  for (int q = 0; q < MAX_SHADOW; ++q) sss[q] = (float)(1.0 / ss[q]);   // powers of two
  const float fs = (float)s;
  if (dt == F64) {
    // FP64 tile: every copy is rounded once from the float64 value
    for (int e = threadIdx.x; e < 16 * b; e += blockDim.x) {
      const double v = it.x[r0 + e];
      reinterpret_cast<double*>(dst)[r0 + e] = v;
#pragma unroll
      for (int q = 0; q < MAX_SHADOW; ++q)
        if (sdst[q]) store_round(sdst[q], sdt[q], r0 + e, sdt[q] == E4M3 ? v / ss[q] : v);
      if (hi) {
        const float f = (float)v;
        uint32_t h;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(f));
        hi[r0 + e] = __uint_as_float(h);
        lo[r0 + e] = f - __uint_as_float(h);
      }
    }
  } else
  for (int e = threadIdx.x; e < 16 * b; e += blockDim.x) {
    const double v = it.x[r0 + e];
    float stored;
    if (dt == F32) {
      stored = __double2float_rn(v);
      reinterpret_cast<float*>(dst)[r0 + e] = stored;
    } else {
      store_round(dst, dt, r0 + e, dt == E4M3 ? v / s : v);
      stored = load_f32(dst, dt, r0 + e) * fs;
    }
#pragma unroll
    for (int q = 0; q < MAX_SHADOW; ++q)
      if (sdst[q]) store_round_f32(sdst[q], sdt[q], r0 + e, sdt[q] == E4M3 ? stored * sss[q] : stored);
    if (hi) {
      uint32_t h;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(stored));
      hi[r0 + e] = __uint_as_float(h);
      lo[r0 + e] = stored - __uint_as_float(h);
    }
  }
  if (blockIdx.y == 0 && threadIdx.x == 0) {
    A.scale[it.tile] = s;
#pragma unroll
    for (int q = 0; q < MAX_SHADOW; ++q)
      if (it.shadow[q] >= 0) A.scale[it.shadow[q]] = ss[q];
    if (it.hi >= 0) { A.scale[it.hi] = 1.0; A.scale[it.lo] = 1.0; }
  }
}

}  // namespace

std::vector<DagTask> potrf_dag_tasks(int nb) {
  // F(0), T(r, 0) for r >= 2, G(1); then per step k: the column-(k+1)
  // updates, the update of block (k+2, k+2) and at once G(k+2) (the
  // critical chain, one step ahead: the CTA that takes it loads its blocks
  // and waits for G(k+1) while the rest of step k is still being handed
  // out), T(r, k+1) for r >= k+3, the rest of step k's updates, then the
  // blocks of W.  Every task's inputs come earlier in this order.
  std::vector<DagTask> v;
  auto add = [&](int op, int r, int c, int k) {
    v.push_back(DagTask{(uint8_t)op, (uint8_t)r, (uint8_t)c, (uint8_t)k});
  };
  // W: per step k, the solves V(k, j) of row k of Y, then the updates
  // E(r, k, j) of the rows below with it
  auto wtasks = [&](int k) {
    for (int j = 0; j < k; ++j) add(4, k, j, 0);
    for (int r = k + 1; r < nb; ++r)
      for (int j = 0; j <= k; ++j) add(5, r, j, k);
  };
  add(0, 0, 0, 0);
  for (int r = 2; r < nb; ++r) add(1, r, 0, 0);
  if (nb > 1) add(3, 1, 1, 1);
  for (int k = 0; k + 1 < nb; ++k) {
    for (int r = k + 2; r < nb; ++r) add(2, r, k + 1, k);
    if (k + 2 < nb) {
      add(2, k + 2, k + 2, k);
      add(3, k + 2, k + 2, k + 2);
    }
    for (int r = k + 3; r < nb; ++r) add(1, r, k + 1, k + 1);
    for (int c = k + 2; c < nb; ++c)
      for (int r = c; r < nb; ++r)
        if (r != k + 2 || c != k + 2) add(2, r, c, k);
    wtasks(k);
  }
  for (int j = 0; j + 1 < nb; ++j) add(4, nb - 1, j, 0);
  return v;
}

void launch_potrf_dag(const Arena& A, const ItemPotrf* items, int count, const DagTask* tasks,
                      int ntasks, int* ticket, double* ldparts, long long* info, int db,
                      cudaStream_t s) {
  if (count <= 0) return;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const int64_t total = (int64_t)ntasks * count;
  // two CTAs per SM: a block task spends about half its time in round trips
  // (its counter polls, the loads of its blocks, the release, the next
  // ticket), which the other CTA's arithmetic fills.  With one CTA per SM
  // the blocks the critical chain reads arrived 5-15k cycles after the
  // block before it was factored (the bulk tasks are handed out too slowly),
  // with two they arrive before it: b = 512, n = 16384: 0.42 -> 0.32 ms per
  // diagonal tile, 25.2 -> 24.3 ms per factorisation, measured
  const int per_sm = 2;
  const int grid =
      (int)std::min<int64_t>(total, std::max<int64_t>(16, std::min<int64_t>(per_sm * sms, total / 8)));
  if (db == 16) k_potrf_dag<16><<<grid, 256, 0, s>>>(A, items, count, tasks, ntasks, ticket, ldparts, info);
  else k_potrf_dag<32><<<grid, 256, 0, s>>>(A, items, count, tasks, ntasks, ticket, ldparts, info);
}

namespace {

template <int PR>
void panel_launch(const Arena& A, const ItemPanel* items, int count, int reserve_sms, cudaStream_t s) {
  const size_t smem =
      sizeof(double) * ((size_t)PR * A.b + 2 * NB * (PK + 1) + NB * (NB + 1) + PR * (NB + 1));
  static int slots = 0;
  if (!slots) {
    cudaFuncSetAttribute(k_panel_trsm<PR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    slots = sms;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_panel_trsm<PR>, 128, smem);
  const int units = count * (A.b / PR);
  const int grid = std::min(units, std::max(1, slots - reserve_sms) * std::max(per_sm, 1));
  k_panel_trsm<PR><<<grid, 128, smem, s>>>(A, items, units);
}

}  // namespace

// 16 rows per work unit keep L_kk's chunks reused across rows; a launch
// with fewer 16-row units than SMs (one panel tile on the critical chain,
// the identity solve for L_kk^{-T}) takes 4-row units instead, so that its
// latency, set by the slowest unit, drops about fourfold.
void launch_panel_trsm(const Arena& A, const ItemPanel* items, int count, int reserve_sms,
                       cudaStream_t s) {
  if (count <= 0) return;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  if ((int64_t)count * (A.b / 16) < sms) panel_launch<4>(A, items, count, reserve_sms, s);
  else panel_launch<16>(A, items, count, reserve_sms, s);
}

void launch_panel_round(const Arena& A, const ItemRound* items, int count, cudaStream_t s) {
  if (count <= 0) return;
  k_panel_round<<<dim3(count, A.b / 16), 256, 0, s>>>(A, items);
}

}  // namespace mp
