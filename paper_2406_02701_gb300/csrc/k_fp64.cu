// FP64 kernels of the factorisation: the diagonal tile's Cholesky and the
// panel triangular solve (the `chol` / `forwardsolve` steps of Sec. 6.2 done
// tile by tile, as in the tiled extension of Sec. 7).
//
// The FP64 diagonal tile (b x b, b a multiple of 64) is factored by a
// blocked right-looking Cholesky over 32 x 32 blocks:
//   potrf_block  one CTA factors block (kb, kb) in shared memory, adds
//                2 sum log L_tt to the log-determinant partials, flags the
//                first pivot that is not > 0, and forms the block's inverse;
//   inner_trsm   the blocks below: X = A L_kb^{-T} = A Dinv^T;
//   inner_syrk   the trailing blocks of the tile: A -= X X^T.
// The panel solve X = A_ik L_kk^{-T} keeps 16 rows of the panel tile in
// shared memory in float64 and sweeps L_kk's 32-column blocks left to right:
// acc = A[:, c] - X[:, <c] L[c, <c]^T, then X[:, c] = acc Dinv_c^T.  The
// float64 result goes to a scratch slot; `panel_round` then rounds it once
// into the tile's format (E4M3: scale from the tile's amax) and into the
// tile's shadow copy, the operand form that lower-precision updates read.
//
// GB300 has little FP64 throughput (about 1.2 TFLOP/s of DFMA), so these
// kernels are bound by the FP64 pipe, not by memory.
#include <algorithm>

#include "mp_device.cuh"

namespace mp {

namespace {

constexpr int NB = 32;   // inner block of the diagonal tile

__global__ void __launch_bounds__(256) k_potrf_block(Arena A, const ItemDiag* __restrict__ items,
                                                     double* __restrict__ ldparts,
                                                     long long* __restrict__ info) {
  __shared__ double S[NB][NB + 1];
  const ItemDiag it = items[blockIdx.x];
  const int b = A.b, tid = threadIdx.x;
  double* T = tile_ptr<double>(A, it.tile) + (int64_t)it.kb * NB * b + it.kb * NB;
  for (int e = tid; e < NB * NB; e += blockDim.x) S[e / NB][e % NB] = T[(int64_t)(e / NB) * b + e % NB];
  __syncthreads();
  __shared__ double rpiv;
  for (int c = 0; c < NB; ++c) {
    if (tid == 0) {
      const double d = S[c][c];
      const double piv = sqrt(d);
      if (!(d > 0.0)) atomicMin(&info[it.mat], (long long)(it.row0 + it.kb * NB + c + 1));
      S[c][c] = piv;
      rpiv = 1.0 / piv;
    }
    __syncthreads();
    for (int r = c + 1 + tid; r < NB; r += blockDim.x) S[r][c] *= rpiv;
    __syncthreads();
    const int m = NB - 1 - c;
    for (int e = tid; e < m * m; e += blockDim.x) {
      int rr = e / m, cc = e - rr * m;
      if (cc <= rr) S[c + 1 + rr][c + 1 + cc] -= S[c + 1 + rr][c] * S[c + 1 + cc][c];
    }
    __syncthreads();
  }
  // 2 sum log L_tt: one log per lane of warp 0, fixed-order butterfly sum
  if (tid < 32) {
    double lg = log(S[tid][tid]);
    for (int o = 16; o > 0; o >>= 1) lg += __shfl_xor_sync(0xffffffffu, lg, o);
    if (tid == 0) ldparts[it.ldslot] = 2.0 * lg;
  }
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    int r = e / NB, c = e % NB;
    if (c <= r) T[(int64_t)r * b + c] = S[r][c];
  }
  // inverse of the lower triangular block by recursive doubling: with
  // L = [A 0; C D], L^{-1} = [A^{-1} 0; -D^{-1} C A^{-1}  D^{-1}]; blocks of
  // size 1, 2, 4, 8, 16 are combined pairwise (dependency depth 2 * 31)
  __shared__ double Di[NB][NB + 1];
  __shared__ double Tm[NB][NB + 1];
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    int r = e / NB, c = e % NB;
    Di[r][c] = r == c ? 1.0 / S[r][r] : 0.0;
  }
  __syncthreads();
  for (int sz = 1; sz < NB; sz <<= 1) {
    const int per = sz * sz, pairs = NB / (2 * sz);
    // T = C A^{-1}: C = S[d0 + r][a0 + t], A^{-1} = Di[a0 + t][a0 + c]
    for (int e = tid; e < pairs * per; e += blockDim.x) {
      const int pr = e / per, r = (e % per) / sz, c = e % sz;
      const int a0 = pr * 2 * sz, d0 = a0 + sz;
      double acc = 0.0;
      for (int t = c; t < sz; ++t) acc += S[d0 + r][a0 + t] * Di[a0 + t][a0 + c];
      Tm[d0 + r][a0 + c] = acc;
    }
    __syncthreads();
    // W = -D^{-1} T: D^{-1} = Di[d0 + r][d0 + t] (t <= r)
    for (int e = tid; e < pairs * per; e += blockDim.x) {
      const int pr = e / per, r = (e % per) / sz, c = e % sz;
      const int a0 = pr * 2 * sz, d0 = a0 + sz;
      double acc = 0.0;
      for (int t = 0; t <= r; ++t) acc += Di[d0 + r][d0 + t] * Tm[d0 + t][a0 + c];
      Di[d0 + r][a0 + c] = -acc;
    }
    __syncthreads();
  }
  for (int e = tid; e < NB * NB; e += blockDim.x) it.dinv[e] = Di[e / NB][e % NB];
}

// Rows below block kb inside the diagonal tile: X = A Dinv^T.
__global__ void __launch_bounds__(256) k_inner_trsm(Arena A, const ItemDiag* __restrict__ items, int kb) {
  __shared__ double X[NB][NB + 1];
  __shared__ double D[NB][NB + 1];
  const ItemDiag it = items[blockIdx.x];
  const int b = A.b, tid = threadIdx.x;
  const int r0 = (kb + 1 + blockIdx.y) * NB;
  double* T = tile_ptr<double>(A, it.tile);
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    int r = e / NB, c = e % NB;
    X[r][c] = T[(int64_t)(r0 + r) * b + kb * NB + c];
    D[r][c] = it.dinv[e];
  }
  __syncthreads();
  const int ty = tid / 8, tx = tid % 8;
  double out[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    int c = tx + 8 * j;
    double a0 = 0.0, a1 = 0.0;
    int t = 0;
    for (; t + 1 <= c; t += 2) {
      a0 += X[ty][t] * D[c][t];
      a1 += X[ty][t + 1] * D[c][t + 1];
    }
    if (t <= c) a0 += X[ty][t] * D[c][t];
    out[j] = a0 + a1;
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) T[(int64_t)(r0 + ty) * b + kb * NB + tx + 8 * j] = out[j];
}

// Trailing blocks (rb, cb), kb < cb <= rb, of the diagonal tile: A -= X_r X_c^T.
__global__ void __launch_bounds__(256) k_inner_syrk(Arena A, const ItemDiag* __restrict__ items, int kb) {
  __shared__ double Xr[NB][NB + 1];
  __shared__ double Xc[NB][NB + 1];
  const ItemDiag it = items[blockIdx.x];
  const int b = A.b, tid = threadIdx.x;
  // blockIdx.y -> (rb, cb) over the lower triangle of the m x m trailing blocks
  int p = blockIdx.y, rb = 0;
  while (p > rb) { p -= rb + 1; ++rb; }
  const int cb = p;
  const int R0 = (kb + 1 + rb) * NB, C0 = (kb + 1 + cb) * NB;
  double* T = tile_ptr<double>(A, it.tile);
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    int r = e / NB, c = e % NB;
    Xr[r][c] = T[(int64_t)(R0 + r) * b + kb * NB + c];
    Xc[r][c] = T[(int64_t)(C0 + r) * b + kb * NB + c];
  }
  __syncthreads();
  const int ty = tid / 8, tx = tid % 8;
  double acc[4] = {}, acc2[4] = {};
  for (int t = 0; t < NB; t += 2) {
    double a = Xr[ty][t], a2 = Xr[ty][t + 1];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      acc[j] += a * Xc[tx + 8 * j][t];
      acc2[j] += a2 * Xc[tx + 8 * j][t + 1];
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    int64_t o = (int64_t)(R0 + ty) * b + C0 + tx + 8 * j;
    T[o] -= acc[j] + acc2[j];
  }
}

constexpr int PR = 16;     // panel rows per work unit
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
    // rows r0.. of I L^{-T} vanish left of column r0: skip those blocks
    const int cb0 = it.identity ? r0 / NB : 0;
    for (int cb = cb0; cb < b / NB; ++cb) {
      for (int e = tid; e < NB * NB; e += blockDim.x)
        Dv[(e / NB) * (NB + 1) + e % NB] = it.dinv[(int64_t)cb * NB * NB + e];
      __syncthreads();
      double acc[NQ], acc2[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) { acc[q] = X[r * b + cb * NB + cx + LPR * q]; acc2[q] = 0.0; }
      const int ch0 = cb0 * NB / PK;
      const int nch = cb * NB / PK - ch0;
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
  for (int e = threadIdx.x; e < 16 * b; e += blockDim.x) {
    double v = it.x[r0 + e];
    store_round(dst, dt, r0 + e, dt == E4M3 ? v / s : v);
    if (sdst[0] || hi) {
      double stored = load_f64(dst, dt, r0 + e) * s;
#pragma unroll
      for (int q = 0; q < MAX_SHADOW; ++q)
        if (sdst[q]) store_round(sdst[q], sdt[q], r0 + e, sdt[q] == E4M3 ? stored / ss[q] : stored);
      if (hi) {
        // the stored value is exact in FP32 (formats up to FP32)
        const float f = (float)stored;
        uint32_t h;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(f));
        hi[r0 + e] = __uint_as_float(h);
        lo[r0 + e] = f - __uint_as_float(h);
      }
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

void launch_potrf_block(const Arena& A, const ItemDiag* items, int count, double* ldparts,
                        long long* info, cudaStream_t s) {
  if (count <= 0) return;
  k_potrf_block<<<count, 256, 0, s>>>(A, items, ldparts, info);
}

void launch_inner_trsm(const Arena& A, const ItemDiag* items, int count, int kb, cudaStream_t s) {
  int m = A.b / NB - kb - 1;
  if (count <= 0 || m <= 0) return;
  k_inner_trsm<<<dim3(count, m), 256, 0, s>>>(A, items, kb);
}

void launch_inner_syrk(const Arena& A, const ItemDiag* items, int count, int kb, cudaStream_t s) {
  int m = A.b / NB - kb - 1;
  if (count <= 0 || m <= 0) return;
  k_inner_syrk<<<dim3(count, m * (m + 1) / 2), 256, 0, s>>>(A, items, kb);
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
