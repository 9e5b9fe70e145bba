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
  if (tid == 0) {
    double s = 0.0;
    for (int c = 0; c < NB; ++c) s += log(S[c][c]);
    ldparts[it.ldslot] = 2.0 * s;
  }
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    int r = e / NB, c = e % NB;
    if (c <= r) T[(int64_t)r * b + c] = S[r][c];
  }
  // inverse of the lower triangular block: row sweep, Di[r][t] for t <= r
  __shared__ double Di[NB][NB + 1];
  __shared__ double rdiag[NB];
  for (int e = tid; e < NB * NB; e += blockDim.x) Di[e / NB][e % NB] = 0.0;
  if (tid < NB) rdiag[tid] = 1.0 / S[tid][tid];
  __syncthreads();
  for (int r = 0; r < NB; ++r) {
    for (int t = tid; t <= r; t += blockDim.x) {
      double acc = (t == r) ? 1.0 : 0.0;
      for (int s = t; s < r; ++s) acc -= S[r][s] * Di[s][t];
      Di[r][t] = acc * rdiag[r];
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
    double acc = 0.0;
    for (int t = 0; t <= c; ++t) acc += X[ty][t] * D[c][t];
    out[j] = acc;
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
  double acc[4] = {};
  for (int t = 0; t < NB; ++t) {
    double a = Xr[ty][t];
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] += a * Xc[tx + 8 * j][t];
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    int64_t o = (int64_t)(R0 + ty) * b + C0 + tx + 8 * j;
    T[o] -= acc[j];
  }
}

constexpr int PR = 16;     // panel rows per CTA
constexpr int PK = 32;     // K chunk of L staged in shared memory

__global__ void __launch_bounds__(128) k_panel_trsm(Arena A, const ItemPanel* __restrict__ items) {
  extern __shared__ double sm[];
  const ItemPanel it = items[blockIdx.x];
  const int b = A.b, tid = threadIdx.x;
  const int r0 = blockIdx.y * PR;
  double* X = sm;                                  // [PR][b]
  double* Ls = X + PR * b;                         // [NB][PK+1]
  double* Dv = Ls + NB * (PK + 1);                 // [NB][NB+1]
  double* Ac = Dv + NB * (NB + 1);                 // [PR][NB+1]
  const TileRef ref = A.tiles[it.tile];
  const char* src = tile_bytes(A, it.tile);
  const double s_in = A.scale[it.tile];
  for (int e = tid; e < PR * b; e += blockDim.x)
    X[e] = load_f64(src, ref.dt, (int64_t)r0 * b + e) * s_in;
  const double* L = tile_ptr<double>(A, it.diag);
  const int r = tid / 8, cx = tid % 8;
  __syncthreads();
  for (int cb = 0; cb < b / NB; ++cb) {
    for (int e = tid; e < NB * NB; e += blockDim.x) Dv[(e / NB) * (NB + 1) + e % NB] = it.dinv[(int64_t)cb * NB * NB + e];
    double acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = X[r * b + cb * NB + cx + 8 * q];
    for (int t0 = 0; t0 < cb * NB; t0 += PK) {
      __syncthreads();
      for (int e = tid; e < NB * PK; e += blockDim.x) {
        int rr = e / PK, tt = e % PK;
        Ls[rr * (PK + 1) + tt] = L[(int64_t)(cb * NB + rr) * b + t0 + tt];
      }
      __syncthreads();
#pragma unroll 8
      for (int tt = 0; tt < PK; ++tt) {
        double xv = X[r * b + t0 + tt];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] -= xv * Ls[(cx + 8 * q) * (PK + 1) + tt];
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) Ac[r * (NB + 1) + cx + 8 * q] = acc[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int c = cx + 8 * q;
      double v = 0.0;
      for (int t = 0; t <= c; ++t) v += Ac[r * (NB + 1) + t] * Dv[c * (NB + 1) + t];
      X[r * b + cb * NB + c] = v;
    }
    __syncthreads();
  }
  double mx = 0.0;
  for (int e = tid; e < PR * b; e += blockDim.x) {
    double v = X[e];
    it.x[(int64_t)r0 * b + e] = v;
    mx = fmax(mx, fabs(v));
  }
  __shared__ double red[4];
  mx = warp_max(mx);
  if ((tid & 31) == 0) red[tid >> 5] = mx;
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < 4; ++w) mx = fmax(mx, red[w]);
    atomic_max_pos(&A.amax[it.tile], mx);
  }
}

__global__ void __launch_bounds__(256) k_panel_round(Arena A, const ItemRound* __restrict__ items) {
  const ItemRound it = items[blockIdx.x];
  const int b = A.b;
  const int dt = A.tiles[it.tile].dt;
  const double amax = amax_value(&A.amax[it.tile]);
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

void launch_panel_trsm(const Arena& A, const ItemPanel* items, int count, cudaStream_t s) {
  if (count <= 0) return;
  size_t smem = sizeof(double) * ((size_t)PR * A.b + NB * (PK + 1) + NB * (NB + 1) + PR * (NB + 1));
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_panel_trsm, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  k_panel_trsm<<<dim3(count, A.b / PR), 128, smem, s>>>(A, items);
}

void launch_panel_round(const Arena& A, const ItemRound* items, int count, cudaStream_t s) {
  if (count <= 0) return;
  k_panel_round<<<dim3(count, A.b / 16), 256, 0, s>>>(A, items);
}

}  // namespace mp
