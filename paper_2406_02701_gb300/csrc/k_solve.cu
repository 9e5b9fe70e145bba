// Triangular solves with the tiled factor, the FP64 refinement residual and
// the log-likelihood reductions (Sec. 6.2: `forwardsolve`, the sum of
// squares, the log-determinant from the factor's diagonal; Sec. 1: float64
// refinement).
//
// Solves run on the identity-padded system of order N = NT b with float64
// arithmetic on the exactly upcast tiles.  Per tile column i (forward) the
// diagonal solve uses the 32 x 32 block inverses kept by the factorisation,
// and every tile below it updates its own segment in one launch; the
// backward solve mirrors this with transposed tiles.  The residual
// r = z - Sigma x reads the float64 copy of Sigma's lower tiles, using a
// tile transposed for the upper part.
//
// Every kernel that a refinement iteration may skip takes a `gate`: when
// the pointed-to flag is 0 (all columns converged) it returns at once.
#include "mp_device.cuh"

namespace mp {

namespace {

constexpr int NB = 32;
constexpr int RCMAX = 8;   // right-hand sides per pass (1 when there is one)

__device__ __forceinline__ bool gated(const int* gate) { return gate && *gate == 0; }

// Diagonal step with the explicit inverse X = L_ii^{-T} (upper triangular,
// row-major, computed by the factorisation): forward out_i = X^T in_i,
// backward out_i = X in_i.  32 output rows per CTA.
template <int TRANS, int RCT>
__global__ void __launch_bounds__(256) k_diag_gemv(Arena A, const ItemSolve* __restrict__ items,
                                                   const int* gate) {
  if (gated(gate)) return;
  extern __shared__ double vs[];          // [b][RCT]
  __shared__ double part[8][32][RCT];
  const ItemSolve it = items[blockIdx.x];
  const int b = A.b, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double* X = tile_ptr<double>(A, it.tile);
  const int r0 = blockIdx.y * 32;
  for (int c0 = 0; c0 < it.nrhs; c0 += RCT) {
    const int nc = min(RCT, it.nrhs - c0);
    __syncthreads();
    for (int e = tid; e < b * RCT; e += blockDim.x) {
      int t = e / RCT, c = e % RCT;
      vs[e] = c < nc ? it.xi[(int64_t)(c0 + c) * it.ld + t] : 0.0;
    }
    __syncthreads();
    if (!TRANS) {
      // out[r0 + lane] = sum_{t <= r} X[t][r] v[t]; warps split t
      double acc[4][RCT];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < RCT; ++c) acc[u][c] = 0.0;
      const int r = r0 + lane;
      const int tend = r0 + 32;
      int t = warp;
      for (; t + 24 < tend; t += 32) {        // four independent chains
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int tu = t + 8 * u;
          const double x = tu > r ? 0.0 : X[(int64_t)tu * b + r];
#pragma unroll
          for (int c = 0; c < RCT; ++c) acc[u][c] += x * vs[tu * RCT + c];
        }
      }
      for (; t < tend; t += 8) {
        const double x = t > r ? 0.0 : X[(int64_t)t * b + r];
#pragma unroll
        for (int c = 0; c < RCT; ++c) acc[0][c] += x * vs[t * RCT + c];
      }
#pragma unroll
      for (int c = 0; c < RCT; ++c) part[warp][lane][c] = (acc[0][c] + acc[1][c]) + (acc[2][c] + acc[3][c]);
      __syncthreads();
      if (warp == 0) {
#pragma unroll
        for (int c = 0; c < RCT; ++c) {
          double v = 0.0;
          for (int w = 0; w < 8; ++w) v += part[w][lane][c];
          if (c < nc) it.xj[(int64_t)(c0 + c) * it.ld + r] = v;
        }
      }
    } else {
      // out[r] = sum_{t >= r} X[r][t] v[t]; a warp per 4 rows, lanes over t
      for (int rr = 0; rr < 4; ++rr) {
        const int r = r0 + warp * 4 + rr;
        double acc[RCT];
#pragma unroll
        for (int c = 0; c < RCT; ++c) acc[c] = 0.0;
        const double* Xr = X + (int64_t)r * b;
        double acc2[RCT];
#pragma unroll
        for (int c = 0; c < RCT; ++c) acc2[c] = 0.0;
        int t = (r & ~31) + lane;
        for (; t + 32 < b; t += 64) {
          const double x0 = t >= r ? Xr[t] : 0.0, x1 = Xr[t + 32];
#pragma unroll
          for (int c = 0; c < RCT; ++c) {
            acc[c] += x0 * vs[t * RCT + c];
            acc2[c] += x1 * vs[(t + 32) * RCT + c];
          }
        }
        for (; t < b; t += 32) {
          const double x = t >= r ? Xr[t] : 0.0;
#pragma unroll
          for (int c = 0; c < RCT; ++c) acc[c] += x * vs[t * RCT + c];
        }
#pragma unroll
        for (int c = 0; c < RCT; ++c) acc[c] += acc2[c];
#pragma unroll
        for (int c = 0; c < RCT; ++c) {
          double v = warp_sum(acc[c]);
          if (lane == 0 && c < nc) it.xj[(int64_t)(c0 + c) * it.ld + r] = v;
        }
      }
    }
  }
}

// Forward: in_j -= L_ji out_i (tile rows).  One CTA: 32 rows, a warp per 4 rows.
template <int RCT>
__global__ void __launch_bounds__(256) k_offdiag_fwd(Arena A, const ItemSolve* __restrict__ items,
                                                     const int* gate) {
  if (gated(gate)) return;
  extern __shared__ double xs[];         // [b][RCT]
  const ItemSolve it = items[blockIdx.x];
  const int b = A.b, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const TileRef ref = A.tiles[it.tile];
  const char* L = tile_bytes(A, it.tile);
  const double sc = A.scale[it.tile];
  const int r0 = blockIdx.y * 32;
  for (int c0 = 0; c0 < it.nrhs; c0 += RCT) {
    const int nc = min(RCT, it.nrhs - c0);
    __syncthreads();
    for (int e = tid; e < b * RCT; e += blockDim.x) {
      int t = e / RCT, c = e % RCT;
      xs[e] = c < nc ? it.xi[(int64_t)(c0 + c) * it.ld + t] : 0.0;
    }
    __syncthreads();
    for (int rr = 0; rr < 4; ++rr) {
      const int r = r0 + warp * 4 + rr;
      double acc[RCT];
#pragma unroll
      for (int c = 0; c < RCT; ++c) acc[c] = 0.0;
      double acc2[RCT];
#pragma unroll
      for (int c = 0; c < RCT; ++c) acc2[c] = 0.0;
#pragma unroll 4
      for (int t = lane; t < b; t += 64) {        // b is a multiple of 64
        const double l0 = load_f64(L, ref.dt, (int64_t)r * b + t) * sc;
        const double l1 = load_f64(L, ref.dt, (int64_t)r * b + t + 32) * sc;
#pragma unroll
        for (int c = 0; c < RCT; ++c) {
          acc[c] += l0 * xs[t * RCT + c];
          acc2[c] += l1 * xs[(t + 32) * RCT + c];
        }
      }
#pragma unroll
      for (int c = 0; c < RCT; ++c) acc[c] += acc2[c];
#pragma unroll
      for (int c = 0; c < RCT; ++c) {
        double v = warp_sum(acc[c]);
        if (lane == 0 && c < nc) it.xj[(int64_t)(c0 + c) * it.ld + r] -= v;
      }
    }
  }
}

// Backward: in_j -= L_ij^T out_i (tile columns).  One CTA: 32 columns (one
// per lane, so a warp reads 256 contiguous bytes of a row), eight warps
// splitting the rows with two accumulator chains each, partial sums added
// in a fixed order.
template <int RCT>
__global__ void __launch_bounds__(256) k_offdiag_bwd(Arena A, const ItemSolve* __restrict__ items,
                                                     const int* gate) {
  if (gated(gate)) return;
  extern __shared__ double xs[];         // [b][RCT]
  __shared__ double part[8][32][RCT];
  const ItemSolve it = items[blockIdx.x];
  const int b = A.b, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const TileRef ref = A.tiles[it.tile];
  const char* L = tile_bytes(A, it.tile);
  const double sc = A.scale[it.tile];
  const int col = blockIdx.y * 32 + lane;
  for (int c0 = 0; c0 < it.nrhs; c0 += RCT) {
    const int nc = min(RCT, it.nrhs - c0);
    __syncthreads();
    for (int e = tid; e < b * RCT; e += blockDim.x) {
      int t = e / RCT, c = e % RCT;
      xs[e] = c < nc ? it.xi[(int64_t)(c0 + c) * it.ld + t] : 0.0;
    }
    __syncthreads();
    double a0[RCT], a1[RCT];
#pragma unroll
    for (int c = 0; c < RCT; ++c) { a0[c] = 0.0; a1[c] = 0.0; }
#pragma unroll 4
    for (int r = warp; r < b; r += 16) {
      const double l0 = load_f64(L, ref.dt, (int64_t)r * b + col) * sc;
      const double l1 = load_f64(L, ref.dt, (int64_t)(r + 8) * b + col) * sc;
#pragma unroll
      for (int c = 0; c < RCT; ++c) {
        a0[c] += l0 * xs[r * RCT + c];
        a1[c] += l1 * xs[(r + 8) * RCT + c];
      }
    }
#pragma unroll
    for (int c = 0; c < RCT; ++c) part[warp][lane][c] = a0[c] + a1[c];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int c = 0; c < RCT; ++c) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += part[w][lane][c];
        if (c < nc) it.xj[(int64_t)(c0 + c) * it.ld + col] -= v;
      }
    }
  }
}

// r_i = z_i - sum_j Sigma_ij x_j for 32 rows of block row ti, in chunks of
// 32 rows x 128 columns of Sigma staged through shared memory.
constexpr int RW = 128;
template <int RC>
__global__ void __launch_bounds__(256) k_residual(Arena A, const ItemResid* __restrict__ items,
                                                  int want_rowabs, const int* gate) {
  if (gated(gate)) return;
  __shared__ double blk[32][RW + 1];
  __shared__ double xs[RW][RC];
  const ItemResid it = items[blockIdx.x];
  const int b = A.b, tid = threadIdx.x;
  const int lr0 = blockIdx.y * 32;                // local row offset in block row ti
  const int64_t g0 = (int64_t)it.ti * b + lr0;    // global row
  const int row = tid / 8, part = tid % 8;        // 8 threads per row, 16 columns each
  for (int c0 = 0; c0 < it.nrhs; c0 += RC) {
    const int nc = min(RC, it.nrhs - c0);
    double acc[RC], acc2[RC];
#pragma unroll
    for (int c = 0; c < RC; ++c) { acc[c] = 0.0; acc2[c] = 0.0; }
    double rabs = 0.0;
    for (int tj = 0; tj < it.nt; ++tj) {
      const bool lower = tj <= it.ti;
      const int tile = lower ? it.sig[it.ti * it.nt + tj] : it.sig[tj * it.nt + it.ti];
      const double* S = tile_ptr<double>(A, tile);
      for (int cc0 = 0; cc0 < b; cc0 += RW) {
        __syncthreads();
        for (int e = tid; e < 32 * RW; e += blockDim.x) {
          if (tj > it.ti) {
            // upper part: Sigma_ij = Sigma_ji^T; consecutive threads read a row of S
            int cc = e / 32, rr = e % 32;
            blk[rr][cc] = S[(int64_t)(cc0 + cc) * b + lr0 + rr];
          } else {
            int rr = e / RW, cc = e % RW;
            int gr = lr0 + rr, gc = cc0 + cc;
            blk[rr][cc] = (tj < it.ti || gc <= gr) ? S[(int64_t)gr * b + gc] : S[(int64_t)gc * b + gr];
          }
        }
        for (int e = tid; e < RW * RC; e += blockDim.x) {
          int t = e / RC, c = e % RC;
          xs[t][c] = c < nc ? it.x[(int64_t)(c0 + c) * it.ld + (int64_t)tj * b + cc0 + t] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int q = 0; q < RW / 8; q += 2) {
          const int cc = part + 8 * q, cc2 = cc + 8;
          const double v = blk[row][cc], v2 = blk[row][cc2];
          if (want_rowabs && c0 == 0) rabs += fabs(v) + fabs(v2);
#pragma unroll
          for (int c = 0; c < RC; ++c) {
            acc[c] += v * xs[cc][c];
            acc2[c] += v2 * xs[cc2][c];
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < RC; ++c) acc[c] += acc2[c];
    for (int o = 4; o > 0; o >>= 1) {
#pragma unroll
      for (int c = 0; c < RC; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
      rabs += __shfl_xor_sync(0xffffffffu, rabs, o);
    }
    if (part == 0) {
      const int64_t g = g0 + row;
      for (int c = 0; c < nc; ++c)
        it.r[(int64_t)(c0 + c) * it.ld + g] = it.z[(int64_t)(c0 + c) * it.ld + g] - acc[c];
      if (want_rowabs && c0 == 0) it.rowabs[g] = rabs;
    }
  }
}

__global__ void k_logdet(const double* ldparts, const int32_t* ldoff, const int32_t* ldcnt,
                         int nmat, double* logdet) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nmat) return;
  double s = 0.0;
  for (int i = 0; i < ldcnt[m]; ++i) s += ldparts[ldoff[m] + i];
  logdet[m] = s;
}

__global__ void k_colmax(const double* v, int64_t n, int64_t ld, double* out, const int* gate) {
  if (gated(gate)) return;
  __shared__ double red[8];
  const double* col = v + (int64_t)blockIdx.x * ld;
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(col[i]));
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) m = fmax(m, red[w]);
    out[blockIdx.x] = m;
  }
}

__global__ void k_refine_check(const double* rmax, const double* xmax, const double* zmax,
                               const double* snorm, int64_t n, int nrhs, int* active, int* iters,
                               int* any, const int* gate) {
  if (gated(gate)) return;
  if (threadIdx.x != 0) return;
  int a = 0;
  for (int c = 0; c < nrhs; ++c) {
    if (active[c]) {
      double tol = (double)n * 0x1p-53 * (snorm[0] * xmax[c] + zmax[c]);
      if (rmax[c] <= tol) active[c] = 0;
      else iters[c] += 1;
    }
    a |= active[c];
  }
  *any = a;
}

__global__ void k_axpy_active(double* x, const double* d, int64_t n, int64_t ld,
                              const int* active, const int* gate) {
  if (gated(gate)) return;
  const int c = blockIdx.y;
  if (!active[c]) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[(int64_t)c * ld + i] += d[(int64_t)c * ld + i];
}

__global__ void k_copy_pad(const double* src, int64_t lds, double* dst, int64_t ldd, int64_t n,
                           int64_t N, const int* gate) {
  if (gated(gate)) return;
  const int c = blockIdx.y;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[(int64_t)c * ldd + i] = i < n ? src[(int64_t)c * lds + i] : 0.0;
}

__global__ void k_dot(const double* a, const double* b, int64_t n, int64_t ld, double* out) {
  __shared__ double red[8];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += a[(int64_t)c * ld + i] * b[(int64_t)c * ld + i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) s += red[w];
    out[c] = s;
  }
}

__global__ void k_loglik(const double* logdet, const double* quad, int64_t n, int nrhs,
                         double* ll) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nrhs) return;
  const double log2pi = 1.8378770664093454836;   // log(2 pi)
  ll[c] = -0.5 * (double)n * log2pi - 0.5 * logdet[0] - 0.5 * quad[c];
}

}  // namespace

void launch_diag_solve(const Arena& A, const ItemSolve* items, int count, int nrhs, int trans,
                       const int* gate, cudaStream_t s) {
  if (count <= 0) return;
  dim3 grid(count, A.b / 32);
  static bool attr = false;
  if (!attr) {
    for (auto f : {(const void*)k_diag_gemv<0, 1>, (const void*)k_diag_gemv<1, 1>,
                   (const void*)k_diag_gemv<0, RCMAX>, (const void*)k_diag_gemv<1, RCMAX>})
      cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    attr = true;
  }
  if (nrhs == 1) {
    size_t smem = sizeof(double) * A.b;
    if (trans) k_diag_gemv<1, 1><<<grid, 256, smem, s>>>(A, items, gate);
    else k_diag_gemv<0, 1><<<grid, 256, smem, s>>>(A, items, gate);
  } else {
    size_t smem = sizeof(double) * A.b * RCMAX;
    if (trans) k_diag_gemv<1, RCMAX><<<grid, 256, smem, s>>>(A, items, gate);
    else k_diag_gemv<0, RCMAX><<<grid, 256, smem, s>>>(A, items, gate);
  }
}

void launch_offdiag_solve(const Arena& A, const ItemSolve* items, int count, int nrhs, int trans,
                          const int* gate, cudaStream_t s) {
  if (count <= 0) return;
  static bool attr = false;
  if (!attr) {
    for (auto f : {(const void*)k_offdiag_fwd<1>, (const void*)k_offdiag_fwd<RCMAX>,
                   (const void*)k_offdiag_bwd<1>, (const void*)k_offdiag_bwd<RCMAX>})
      cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    attr = true;
  }
  const int rc = nrhs == 1 ? 1 : RCMAX;
  size_t smem = sizeof(double) * A.b * rc;
  if (trans) {
    dim3 grid(count, A.b / 32);
    if (rc == 1) k_offdiag_bwd<1><<<grid, 256, smem, s>>>(A, items, gate);
    else k_offdiag_bwd<RCMAX><<<grid, 256, smem, s>>>(A, items, gate);
  } else {
    dim3 grid(count, A.b / 32);
    if (rc == 1) k_offdiag_fwd<1><<<grid, 256, smem, s>>>(A, items, gate);
    else k_offdiag_fwd<RCMAX><<<grid, 256, smem, s>>>(A, items, gate);
  }
}

void launch_residual(const Arena& A, const ItemResid* items, int count, int nrhs,
                     int want_rowabs, const int* gate, cudaStream_t s) {
  if (count <= 0) return;
  dim3 grid(count, A.b / 32);
  if (nrhs == 1) k_residual<1><<<grid, 256, 0, s>>>(A, items, want_rowabs, gate);
  else k_residual<RCMAX><<<grid, 256, 0, s>>>(A, items, want_rowabs, gate);
}

void launch_logdet(const double* ldparts, const int32_t* ldoff, const int32_t* ldcnt, int nmat,
                   double* logdet, cudaStream_t s) {
  if (nmat <= 0) return;
  k_logdet<<<(nmat + 127) / 128, 128, 0, s>>>(ldparts, ldoff, ldcnt, nmat, logdet);
}

void launch_colmax(const double* v, int64_t n, int64_t ld, int nrhs, double* out,
                   const int* gate, cudaStream_t s) {
  k_colmax<<<nrhs, 256, 0, s>>>(v, n, ld, out, gate);
}

void launch_refine_check(const double* rmax, const double* xmax, const double* zmax,
                         const double* snorm, int64_t n, int nrhs, int* active, int* iters,
                         int* any, const int* gate, cudaStream_t s) {
  k_refine_check<<<1, 32, 0, s>>>(rmax, xmax, zmax, snorm, n, nrhs, active, iters, any, gate);
}

void launch_axpy_active(double* x, const double* d, int64_t n, int64_t ld, int nrhs,
                        const int* active, const int* gate, cudaStream_t s) {
  k_axpy_active<<<dim3(64, nrhs), 256, 0, s>>>(x, d, n, ld, active, gate);
}

void launch_copy_pad(const double* src, int64_t lds, double* dst, int64_t ldd, int64_t n,
                     int64_t N, int nrhs, const int* gate, cudaStream_t s) {
  k_copy_pad<<<dim3(64, nrhs), 256, 0, s>>>(src, lds, dst, ldd, n, N, gate);
}

void launch_dot(const double* a, const double* b, int64_t n, int64_t ld, int nrhs, double* out,
                cudaStream_t s) {
  k_dot<<<nrhs, 256, 0, s>>>(a, b, n, ld, out);
}

void launch_loglik(const double* logdet, const double* quad, int64_t n, int nrhs, double* ll,
                   cudaStream_t s) {
  k_loglik<<<(nrhs + 127) / 128, 128, 0, s>>>(logdet, quad, n, nrhs, ll);
}

}  // namespace mp
