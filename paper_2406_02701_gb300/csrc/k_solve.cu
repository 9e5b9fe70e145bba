// Triangular solves with the tiled factor, the FP64 refinement residual and
// the log-likelihood reductions (Sec. 6.2: `forwardsolve`, the sum of
// squares, the log-determinant from the factor's diagonal; Sec. 1: float64
// refinement).
//
// Solves run on the identity-padded system of order N = NT b as one task
// graph per solve (below): the diagonal steps use the explicit inverses
// L_ii^{-T} kept by the factorisation (float64), the off-diagonal tiles
// update the right-hand side block by block.  The residual r = z - Sigma x
// reads the float64 copy of Sigma's lower tiles, using a tile transposed
// for the upper part.
//
// Every kernel that a refinement iteration may skip takes a `gate`: when
// the pointed-to flag is 0 (all columns converged) it returns at once.
#include <algorithm>
#include <vector>

#include "mp_device.cuh"

namespace mp {

namespace {

constexpr int RCMAX = 8;   // right-hand sides per pass (1 when there is one)

__device__ __forceinline__ bool gated(const int* gate) { return gate && *gate == 0; }

// ------------------------------------------------------------ solve graph
//
// One persistent launch runs a whole tiled triangular solve as tasks over
// 32-row blocks (P = b / 32 per tile row), tile rows taken in solve order
// s_0, s_1, ... (forward 0, 1, ...; backward nt-1, nt-2, ...):
//   D(i, p)     diagonal block: out_i[p] from in_i - chain_i with the
//               explicit inverse X = L_ii^{-T};
//   O(i, j, p)  off-diagonal block applied in place: in_i[p] -= L_ij out_j
//               (forward) or L_ji^T out_j (backward), for every j but the
//               row solved just before i;
//   C(i, j, p)  the same product with that last row j, stored in chain_i[p]
//               (the critical chain: it does not wait for the in-place
//               updates, so it can be handed out right after D(j)).
// Counters (zero at launch) per tile row i: updates applied in place to
// each block of in_i, finished blocks of out_i, and the chain product of
// each block.  D(i, p) waits until the blocks of in_i it reads have all
// their in-place updates and chain products; O and C wait for the whole of
// out_j, O also for the in-place update before it on the same block
// (updates to one block are applied in a fixed order and the chain
// product is subtracted last, so the result is deterministic and equals
// in-place accumulation in solve order).  Tasks are taken by an atomic
// ticket in a topological order, so the graph cannot deadlock whatever the
// number of co-resident CTAs.
//
// Off-diagonal tiles stored in FP32 or below hold values exact in FP32, so
// their products run on the FP32 pipe in float-float arithmetic: out_j is
// split as h + l (two floats), a tile value a gives a h exactly as p + e
// (one product and one FMA), a l to 2^-24 of a term already 2^-24 small,
// and the row sums accumulate as compensated pairs; the result carries
// about 2^-46 relative error against a float64 sum.  FP64 tiles use float64.

// Value i of a tile stored in format DT (exact in FP32).
template <int DT>
__device__ __forceinline__ float tval(const char* base, int64_t i) {
  if (DT == F32) return reinterpret_cast<const float*>(base)[i];
  if (DT == BF16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(base)[i]);
  if (DT == F16) return __half2float(reinterpret_cast<const __half*>(base)[i]);
  __nv_fp8_e4m3 v;
  v.__x = reinterpret_cast<const __nv_fp8_storage_t*>(base)[i];
  return (float)v;
}

// (hi, lo) += a (h + l) with a exact in FP32.
__device__ __forceinline__ void ff_madd(float& hi, float& lo, float a, float h, float l) {
  const float p = a * h;
  const float e = fmaf(a, h, -p);               // a h = p + e exactly
  const float s = hi + p;                       // two-sum of hi and p
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (p - bb);
  hi = s;
  lo += err + e + a * l;
}

constexpr int MLP = 32;   // loads a thread issues before using them

// Diagonal block: out_i[p] from in_i with X = L_ii^{-T} (float64).
// in_i - chain_i (the chain product is the row's last update; none for the
// first row solved)
__device__ __forceinline__ double solve_in(const double* v, const double* ch, int64_t o) {
  return ch ? __ldcg(v + o) - __ldcg(ch + o) : __ldcg(v + o);
}

template <int RCT>
__device__ void solve_diag(const Arena& A, const ItemSolveDag& it, int i, int p, int trans,
                           double* vs, double* part, bool first) {
  const int b = A.b, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double* X = tile_ptr<double>(A, it.linv[i]);
  const double* v = it.in + (int64_t)i * b;
  const double* ch = first ? nullptr : it.chain + (int64_t)i * b;
  double* o = it.out + (int64_t)i * b;
  const int t0 = trans ? p * 32 : 0, t1 = trans ? b : (p + 1) * 32;
  for (int c0 = 0; c0 < it.nrhs; c0 += RCT) {
    const int nc = min(RCT, it.nrhs - c0);
    __syncthreads();
    for (int e = tid; e < (t1 - t0) * RCT; e += blockDim.x) {
      const int t = t0 + e / RCT, c = e % RCT;
      vs[t * RCT + c] = c < nc ? solve_in(v, ch, (int64_t)(c0 + c) * it.ld + t) : 0.0;
    }
    __syncthreads();
    double acc[RCT];
#pragma unroll
    for (int c = 0; c < RCT; ++c) acc[c] = 0.0;
    if (!trans) {
      // out[r] = sum_{t <= r} X[t][r] v[t], r = 32 p + lane; warp w takes t = w + 8 k
      const int r = p * 32 + lane;
      const int nk = t1 / 8;
      for (int k0 = 0; k0 < nk; k0 += MLP) {
        double x[MLP];
#pragma unroll
        for (int u = 0; u < MLP; ++u) {
          const int t = warp + 8 * (k0 + u);
          x[u] = (k0 + u < nk && t <= r) ? X[(int64_t)t * b + r] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < MLP; ++u) {
          if (k0 + u >= nk) break;                 // uniform: nk is the same for all threads
          const int t = warp + 8 * (k0 + u);
#pragma unroll
          for (int c = 0; c < RCT; ++c) acc[c] += x[u] * vs[t * RCT + c];
        }
      }
#pragma unroll
      for (int c = 0; c < RCT; ++c) part[(warp * 32 + lane) * RCT + c] = acc[c];
      __syncthreads();
      if (warp == 0) {
        for (int c = 0; c < nc; ++c) {
          double sum = 0.0;
          for (int w = 0; w < 8; ++w) sum += part[(w * 32 + lane) * RCT + c];
          o[(int64_t)(c0 + c) * it.ld + r] = sum;
        }
      }
    } else {
      // out[r] = sum_{t >= r} X[r][t] v[t]: thread (row r = 32 p + tid / 8,
      // s = tid % 8) takes t = 32 p + s + 8 k
      const int r = p * 32 + (tid >> 3), sg = tid & 7;
      const double* Xr = X + (int64_t)r * b;
      const int nk = (b - p * 32) / 8;
      for (int k0 = 0; k0 < nk; k0 += MLP) {
        double x[MLP];
#pragma unroll
        for (int u = 0; u < MLP; ++u) {
          const int t = p * 32 + sg + 8 * (k0 + u);
          x[u] = (k0 + u < nk && t >= r) ? Xr[t] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < MLP; ++u) {
          if (k0 + u >= nk) break;
          const int t = p * 32 + sg + 8 * (k0 + u);
#pragma unroll
          for (int c = 0; c < RCT; ++c) acc[c] += x[u] * vs[t * RCT + c];
        }
      }
      for (int c = 0; c < nc; ++c) {
        double sum = acc[c];
        for (int o2 = 4; o2 > 0; o2 >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o2);
        if (sg == 0) o[(int64_t)(c0 + c) * it.ld + r] = sum;
      }
    }
  }
}

// (hi, lo) += (xh + xl)(vh + vl) to about 2^-46: xh vh exactly as p + e,
// the cross terms once rounded, xl vl dropped.
__device__ __forceinline__ void ff_madd2(float& hi, float& lo, float xh, float xl, float vh, float vl) {
  const float p = xh * vh;
  const float e = fmaf(xh, vh, -p);
  const float cross = fmaf(xh, vl, xl * vh);
  const float s = hi + p;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (p - bb);
  hi = s;
  lo += err + e + cross;
}

// Four consecutive values (exact in FP32) of a tile stored in format DT,
// from element i, a multiple of 4: one 16-, 8- or 4-byte load.
template <int DT>
__device__ __forceinline__ float4 tval4(const char* base, int64_t i) {
  if (DT == F32) return __ldcg(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(base) + i));
  if (DT == BF16 || DT == F16) {
    const uint2 u = __ldcg(reinterpret_cast<const uint2*>(reinterpret_cast<const uint16_t*>(base) + i));
    const uint32_t w[4] = {u.x & 0xffffu, u.x >> 16, u.y & 0xffffu, u.y >> 16};
    float f[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
      f[j] = DT == BF16 ? __uint_as_float(w[j] << 16) : __half2float(__ushort_as_half((unsigned short)w[j]));
    return make_float4(f[0], f[1], f[2], f[3]);
  }
  const uint32_t u = __ldcg(reinterpret_cast<const unsigned int*>(reinterpret_cast<const uint8_t*>(base) + i));
  float f[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    __nv_fp8_e4m3 v;
    v.__x = (__nv_fp8_storage_t)((u >> (8 * j)) & 0xffu);
    f[j] = (float)v;
  }
  return make_float4(f[0], f[1], f[2], f[3]);
}

__device__ __forceinline__ float f4(const float4& v, int j) {
  return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}

// The 32 columns of block p: thread (row group rg = tid / 8, column quad
// cq = tid % 8) has the float-float sums of columns 32 p + 4 cq + j over its
// rows; sums over the four row groups of a warp, then over the warps in
// order, give column 32 p + lane to warp 0 (returned there, 0 elsewhere).
__device__ __forceinline__ double ff_column_sums(const float* hi, const float* lo, double* part) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    double s = (double)hi[j] + (double)lo[j];
    s += __shfl_xor_sync(0xffffffffu, s, 8);
    s += __shfl_xor_sync(0xffffffffu, s, 16);
    if (lane < 8) part[warp * 32 + 4 * lane + j] = s;
  }
  __syncthreads();
  double sum = 0.0;
  if (warp == 0)
    for (int w = 0; w < 8; ++w) sum += part[w * 32 + lane];
  return sum;
}

// One right-hand side, off-diagonal block of a tile stored in FP32 or below,
// with 16-byte loads: a thread keeps all of its share of the 32 x b block
// (or b x 32 for the backward solve) in flight at once, issued before the
// vector it multiplies is staged.  Items with one right-hand side take this
// code in every launch, so a request's bits do not depend on the other
// requests of its batch.
constexpr int VB = 16;     // vector loads a thread issues before using them
template <int DT>
__device__ void solve_off_ff1(const char* L, float scf, int b, int p, int trans, const double* y,
                              float2* ys, double* part, double* r, bool store) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nk = b / 32;
  // y (the solved block the task waits for) is staged as float pairs while
  // the block's first loads are in flight
  auto stage = [&]() {
    for (int t = tid; t < b; t += blockDim.x) {
      const double v = __ldcg(y + t);
      const float h = (float)v;
      ys[t] = make_float2(h, (float)(v - (double)h));
    }
    __syncthreads();
  };
  const int ys_stride = 1;
  if (!trans) {
    // in_i[q] -= sum_t L_ij[q][t] y[t]: thread (row q = 32 p + tid / 8,
    // sg = tid % 8), t = 4 sg + 32 k + j
    const int q = p * 32 + (tid >> 3), sg = tid & 7;
    const int64_t row = (int64_t)q * b + 4 * sg;
    float hi = 0.f, lo = 0.f;
    for (int k0 = 0; k0 < nk; k0 += VB) {
      float4 a[VB];
#pragma unroll
      for (int u = 0; u < VB; ++u)
        a[u] = k0 + u < nk ? tval4<DT>(L, row + 32 * (k0 + u)) : make_float4(0.f, 0.f, 0.f, 0.f);
      if (k0 == 0) stage();
#pragma unroll
      for (int u = 0; u < VB; ++u) {
        if (k0 + u >= nk) break;                   // uniform
        const int t = 4 * sg + 32 * (k0 + u);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float2 h = ys[(t + j) * ys_stride];
          ff_madd(hi, lo, f4(a[u], j) * scf, h.x, h.y);
        }
      }
    }
    double sum = (double)hi + (double)lo;
    for (int o2 = 4; o2 > 0; o2 >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o2);
    if (sg == 0) {
      double* rp = r + q;
      *rp = store ? sum : __ldcg(rp) - sum;
    }
  } else {
    // in_i[q] -= sum_t L_ji[t][q] y[t], q = 32 p + 4 cq + j: thread (row
    // group rg = tid / 8, cq = tid % 8) takes rows t = rg + 32 k
    const int rg = tid >> 3, cq = tid & 7;
    float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < nk; k0 += VB) {
      float4 a[VB];
#pragma unroll
      for (int u = 0; u < VB; ++u)
        a[u] = k0 + u < nk ? tval4<DT>(L, (int64_t)(rg + 32 * (k0 + u)) * b + p * 32 + 4 * cq)
                           : make_float4(0.f, 0.f, 0.f, 0.f);
      if (k0 == 0) stage();
#pragma unroll
      for (int u = 0; u < VB; ++u) {
        if (k0 + u >= nk) break;
        const float2 h = ys[(rg + 32 * (k0 + u)) * ys_stride];
#pragma unroll
        for (int j = 0; j < 4; ++j) ff_madd(hi[j], lo[j], f4(a[u], j) * scf, h.x, h.y);
      }
    }
    const double sum = ff_column_sums(hi, lo, part);
    if (warp == 0) {
      double* rp = r + p * 32 + lane;
      *rp = store ? sum : __ldcg(rp) - sum;
    }
  }
}

// One right-hand side, diagonal block p in float-float from W's FP32 hi/lo
// parts, with 16-byte loads issued before in_i - chain_i is staged.
// X = L_ii^{-T} is upper triangular: the products outside it are masked
// (only the triangle is guaranteed to be written).
constexpr int VBD = 8;     // vector loads of each of hi and lo in flight
__device__ void solve_diag_ff1(const float* Xh, const float* Xl, int b, int p, int trans,
                               const double* v, const double* ch, float2* vsf, double* part,
                               double* o) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // in_i - chain_i over the rows the block reads, staged as float pairs
  // while the first loads of X are in flight
  const int t0 = trans ? p * 32 : 0, t1 = trans ? b : (p + 1) * 32;
  auto stage = [&]() {
    for (int t = t0 + tid; t < t1; t += blockDim.x) {
      const double x = solve_in(v, ch, t);
      const float h = (float)x;
      vsf[t] = make_float2(h, (float)(x - (double)h));
    }
    __syncthreads();
  };
  const int v_stride = 1;
  if (!trans) {
    // out[r] = sum_{t <= r} X[t][r] v[t], r = 32 p + 4 cq + j: thread (row
    // group rg = tid / 8, cq = tid % 8) takes rows t = rg + 32 k, k <= p
    const int rg = tid >> 3, cq = tid & 7, r0 = p * 32 + 4 * cq;
    const int nk = p + 1;
    float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < nk; k0 += VBD) {
      float4 xh[VBD], xl[VBD];
#pragma unroll
      for (int u = 0; u < VBD; ++u) {
        const int64_t o4 = (int64_t)(rg + 32 * (k0 + u)) * b + r0;
        const bool ok = k0 + u < nk;
        xh[u] = ok ? __ldcg(reinterpret_cast<const float4*>(Xh + o4)) : make_float4(0.f, 0.f, 0.f, 0.f);
        xl[u] = ok ? __ldcg(reinterpret_cast<const float4*>(Xl + o4)) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      if (k0 == 0) stage();
#pragma unroll
      for (int u = 0; u < VBD; ++u) {
        if (k0 + u >= nk) break;                   // uniform
        const int t = rg + 32 * (k0 + u);
        const float2 w = vsf[t * v_stride];
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (t <= r0 + j) ff_madd2(hi[j], lo[j], f4(xh[u], j), f4(xl[u], j), w.x, w.y);
      }
    }
    const double sum = ff_column_sums(hi, lo, part);
    if (warp == 0) o[p * 32 + lane] = sum;
  } else {
    // out[r] = sum_{t >= r} X[r][t] v[t], r = 32 p + tid / 8: thread (r,
    // sg = tid % 8) takes t = 32 p + 4 sg + 32 k + j
    const int r = p * 32 + (tid >> 3), sg = tid & 7;
    const int nk = (b - p * 32) / 32;
    const int64_t row = (int64_t)r * b + p * 32 + 4 * sg;
    float hi = 0.f, lo = 0.f;
    for (int k0 = 0; k0 < nk; k0 += VBD) {
      float4 xh[VBD], xl[VBD];
#pragma unroll
      for (int u = 0; u < VBD; ++u) {
        const bool ok = k0 + u < nk;
        xh[u] = ok ? __ldcg(reinterpret_cast<const float4*>(Xh + row + 32 * (k0 + u))) : make_float4(0.f, 0.f, 0.f, 0.f);
        xl[u] = ok ? __ldcg(reinterpret_cast<const float4*>(Xl + row + 32 * (k0 + u))) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      if (k0 == 0) stage();
#pragma unroll
      for (int u = 0; u < VBD; ++u) {
        if (k0 + u >= nk) break;
        const int t = p * 32 + 4 * sg + 32 * (k0 + u);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float2 w = vsf[(t + j) * v_stride];
          if (t + j >= r) ff_madd2(hi, lo, f4(xh[u], j), f4(xl[u], j), w.x, w.y);
        }
      }
    }
    double sum = (double)hi + (double)lo;
    for (int o2 = 4; o2 > 0; o2 >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o2);
    if (sg == 0) o[r] = sum;
  }
}

// Diagonal block in float-float from W's FP32 hi/lo parts (mixed factors):
// same data flow as solve_diag, the products on the FP32 pipe.
template <int RCT>
__device__ void solve_diag_ff(const Arena& A, const ItemSolveDag& it, int i, int p, int trans,
                              double* vs, double* part, bool first) {
  const int b = A.b, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = it.nt;
  const float* Xh = tile_ptr<float>(A, it.linv[nt + i]);
  const float* Xl = tile_ptr<float>(A, it.linv[2 * nt + i]);
  const double* v = it.in + (int64_t)i * b;
  const double* ch = first ? nullptr : it.chain + (int64_t)i * b;
  double* o = it.out + (int64_t)i * b;
  float2* vsf = reinterpret_cast<float2*>(vs);
  if (it.nrhs == 1) {   // one right-hand side: the same code whatever RCT
    solve_diag_ff1(Xh, Xl, b, p, trans, v, ch, vsf, part, o);
    return;
  }
  const int t0 = trans ? p * 32 : 0, t1 = trans ? b : (p + 1) * 32;
  for (int c0 = 0; c0 < it.nrhs; c0 += RCT) {
    const int nc = min(RCT, it.nrhs - c0);
    __syncthreads();
    for (int e = tid; e < (t1 - t0) * RCT; e += blockDim.x) {
      const int t = t0 + e / RCT, c = e % RCT;
      const double x = c < nc ? solve_in(v, ch, (int64_t)(c0 + c) * it.ld + t) : 0.0;
      const float h = (float)x;
      vsf[t * RCT + c] = make_float2(h, (float)(x - (double)h));
    }
    __syncthreads();
    float hi[RCT], lo[RCT];
#pragma unroll
    for (int c = 0; c < RCT; ++c) { hi[c] = 0.f; lo[c] = 0.f; }
    if (!trans) {
      const int r = p * 32 + lane;
      const int nk = t1 / 8;
      for (int k0 = 0; k0 < nk; k0 += MLP) {
        float xh[MLP], xl[MLP];
#pragma unroll
        for (int u = 0; u < MLP; ++u) {
          const int t = warp + 8 * (k0 + u);
          const bool ok = k0 + u < nk && t <= r;
          xh[u] = ok ? Xh[(int64_t)t * b + r] : 0.f;
          xl[u] = ok ? Xl[(int64_t)t * b + r] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < MLP; ++u) {
          if (k0 + u >= nk) break;
          const int t = warp + 8 * (k0 + u);
#pragma unroll
          for (int c = 0; c < RCT; ++c) {
            const float2 w = vsf[t * RCT + c];
            ff_madd2(hi[c], lo[c], xh[u], xl[u], w.x, w.y);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < RCT; ++c) part[(warp * 32 + lane) * RCT + c] = (double)hi[c] + (double)lo[c];
      __syncthreads();
      if (warp == 0) {
        for (int c = 0; c < nc; ++c) {
          double sum = 0.0;
          for (int w = 0; w < 8; ++w) sum += part[(w * 32 + lane) * RCT + c];
          o[(int64_t)(c0 + c) * it.ld + r] = sum;
        }
      }
    } else {
      const int r = p * 32 + (tid >> 3), sg = tid & 7;
      const int nk = (b - p * 32) / 8;
      for (int k0 = 0; k0 < nk; k0 += MLP) {
        float xh[MLP], xl[MLP];
#pragma unroll
        for (int u = 0; u < MLP; ++u) {
          const int t = p * 32 + sg + 8 * (k0 + u);
          const bool ok = k0 + u < nk && t >= r;
          xh[u] = ok ? Xh[(int64_t)r * b + t] : 0.f;
          xl[u] = ok ? Xl[(int64_t)r * b + t] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < MLP; ++u) {
          if (k0 + u >= nk) break;
          const int t = p * 32 + sg + 8 * (k0 + u);
#pragma unroll
          for (int c = 0; c < RCT; ++c) {
            const float2 w = vsf[t * RCT + c];
            ff_madd2(hi[c], lo[c], xh[u], xl[u], w.x, w.y);
          }
        }
      }
      for (int c = 0; c < nc; ++c) {
        double sum = (double)hi[c] + (double)lo[c];
        for (int o2 = 4; o2 > 0; o2 >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o2);
        if (sg == 0) o[(int64_t)(c0 + c) * it.ld + r] = sum;
      }
    }
  }
}

// Off-diagonal block, tiles stored in FP32 or below (DT), float-float sums.
template <int RCT, int DT>
__device__ void solve_off_ff(const char* L, float scf, const ItemSolveDag& it, int b, int p,
                             int trans, const float2* ys, double* part, double* r, int c0, int nc,
                             bool store) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float hi[RCT], lo[RCT];
#pragma unroll
  for (int c = 0; c < RCT; ++c) { hi[c] = 0.f; lo[c] = 0.f; }
  if (!trans) {
    // in_i[q] -= sum_t L_ij[q][t] y[t]: thread (row q = 32 p + tid / 8, s = tid % 8), t = s + 8 k
    const int q = p * 32 + (tid >> 3), sg = tid & 7;
    const int64_t row = (int64_t)q * b;
    const int nk = b / 8;
    for (int k0 = 0; k0 < nk; k0 += MLP) {
      float a[MLP];
#pragma unroll
      for (int u = 0; u < MLP; ++u) a[u] = k0 + u < nk ? tval<DT>(L, row + sg + 8 * (k0 + u)) * scf : 0.f;
#pragma unroll
      for (int u = 0; u < MLP; ++u) {
        if (k0 + u >= nk) break;                   // uniform: nk = b / 8 for every thread
        const int t = sg + 8 * (k0 + u);
#pragma unroll
        for (int c = 0; c < RCT; ++c) {
          const float2 h = ys[t * RCT + c];
          ff_madd(hi[c], lo[c], a[u], h.x, h.y);
        }
      }
    }
    for (int c = 0; c < nc; ++c) {
      double sum = (double)hi[c] + (double)lo[c];
      for (int o2 = 4; o2 > 0; o2 >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o2);
      if (sg == 0) {
        double* rp = r + (int64_t)(c0 + c) * it.ld + q;
        *rp = store ? sum : __ldcg(rp) - sum;
      }
    }
  } else {
    // in_i[q] -= sum_t L_ji[t][q] y[t]: q = 32 p + lane, warp w takes t = w + 8 k
    const int q = p * 32 + lane;
    const int nk = b / 8;
    for (int k0 = 0; k0 < nk; k0 += MLP) {
      float a[MLP];
#pragma unroll
      for (int u = 0; u < MLP; ++u)
        a[u] = k0 + u < nk ? tval<DT>(L, (int64_t)(warp + 8 * (k0 + u)) * b + q) * scf : 0.f;
#pragma unroll
      for (int u = 0; u < MLP; ++u) {
        if (k0 + u >= nk) break;
        const int t = warp + 8 * (k0 + u);
#pragma unroll
        for (int c = 0; c < RCT; ++c) {
          const float2 h = ys[t * RCT + c];
          ff_madd(hi[c], lo[c], a[u], h.x, h.y);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < RCT; ++c) part[(warp * 32 + lane) * RCT + c] = (double)hi[c] + (double)lo[c];
    __syncthreads();
    if (warp == 0) {
      for (int c = 0; c < nc; ++c) {
        double sum = 0.0;
        for (int w = 0; w < 8; ++w) sum += part[(w * 32 + lane) * RCT + c];
        double* rp = r + (int64_t)(c0 + c) * it.ld + q;
        *rp = store ? sum : __ldcg(rp) - sum;
      }
    }
  }
}

// Off-diagonal block of an FP64 tile, float64 sums.
template <int RCT>
__device__ void solve_off_f64(const double* L, const ItemSolveDag& it, int b, int p, int trans,
                              const double* vs, double* part, double* r, int c0, int nc, bool store) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double acc[RCT];
#pragma unroll
  for (int c = 0; c < RCT; ++c) acc[c] = 0.0;
  if (!trans) {
    const int q = p * 32 + (tid >> 3), sg = tid & 7;
    const int64_t row = (int64_t)q * b;
    const int nk = b / 8;
    for (int k0 = 0; k0 < nk; k0 += MLP) {
      double a[MLP];
#pragma unroll
      for (int u = 0; u < MLP; ++u) a[u] = k0 + u < nk ? L[row + sg + 8 * (k0 + u)] : 0.0;
#pragma unroll
      for (int u = 0; u < MLP; ++u) {
        if (k0 + u >= nk) break;
#pragma unroll
        for (int c = 0; c < RCT; ++c) acc[c] += a[u] * vs[(sg + 8 * (k0 + u)) * RCT + c];
      }
    }
    for (int c = 0; c < nc; ++c) {
      double sum = acc[c];
      for (int o2 = 4; o2 > 0; o2 >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o2);
      if (sg == 0) {
        double* rp = r + (int64_t)(c0 + c) * it.ld + q;
        *rp = store ? sum : __ldcg(rp) - sum;
      }
    }
  } else {
    const int q = p * 32 + lane;
    const int nk = b / 8;
    for (int k0 = 0; k0 < nk; k0 += MLP) {
      double a[MLP];
#pragma unroll
      for (int u = 0; u < MLP; ++u) a[u] = k0 + u < nk ? L[(int64_t)(warp + 8 * (k0 + u)) * b + q] : 0.0;
#pragma unroll
      for (int u = 0; u < MLP; ++u) {
        if (k0 + u >= nk) break;
#pragma unroll
        for (int c = 0; c < RCT; ++c) acc[c] += a[u] * vs[(warp + 8 * (k0 + u)) * RCT + c];
      }
    }
#pragma unroll
    for (int c = 0; c < RCT; ++c) part[(warp * 32 + lane) * RCT + c] = acc[c];
    __syncthreads();
    if (warp == 0) {
      for (int c = 0; c < nc; ++c) {
        double sum = 0.0;
        for (int w = 0; w < 8; ++w) sum += part[(w * 32 + lane) * RCT + c];
        double* rp = r + (int64_t)(c0 + c) * it.ld + q;
        *rp = store ? sum : __ldcg(rp) - sum;
      }
    }
  }
}

template <int RCT>
__device__ void solve_off(const Arena& A, const ItemSolveDag& it, int i, int j, int p, int trans,
                          double* vs, double* part, bool store) {
  const int b = A.b, tid = threadIdx.x, nt = it.nt;
  const int tile = trans ? it.tiles[j * nt + i] : it.tiles[i * nt + j];
  const TileRef ref = A.tiles[tile];
  const char* L = tile_bytes(A, tile);
  const float scf = (float)A.scale[tile];       // a power of two (1 except E4M3)
  const bool f64 = ref.dt == F64;
  const double* y = it.out + (int64_t)j * b;
  double* r = (store ? it.chain : it.in) + (int64_t)i * b;
  float2* ys = reinterpret_cast<float2*>(vs);
  if (it.nrhs == 1 && !f64) {
    switch (ref.dt) {
      case F32: solve_off_ff1<F32>(L, scf, b, p, trans, y, ys, part, r, store); break;
      case BF16: solve_off_ff1<BF16>(L, scf, b, p, trans, y, ys, part, r, store); break;
      case F16: solve_off_ff1<F16>(L, scf, b, p, trans, y, ys, part, r, store); break;
      default: solve_off_ff1<E4M3>(L, scf, b, p, trans, y, ys, part, r, store); break;
    }
    return;
  }
  for (int c0 = 0; c0 < it.nrhs; c0 += RCT) {
    const int nc = min(RCT, it.nrhs - c0);
    __syncthreads();
    for (int e = tid; e < b * RCT; e += blockDim.x) {
      const int t = e / RCT, c = e % RCT;
      const double v = c < nc ? __ldcg(y + (int64_t)(c0 + c) * it.ld + t) : 0.0;
      if (f64) {
        vs[e] = v;
      } else {
        const float h = (float)v;
        ys[e] = make_float2(h, (float)(v - (double)h));
      }
    }
    __syncthreads();
    switch (ref.dt) {
      case F64: solve_off_f64<RCT>(reinterpret_cast<const double*>(L), it, b, p, trans, vs, part, r, c0, nc, store); break;
      case F32:
        solve_off_ff<RCT, F32>(L, scf, it, b, p, trans, ys, part, r, c0, nc, store);
        break;
      case BF16:
        solve_off_ff<RCT, BF16>(L, scf, it, b, p, trans, ys, part, r, c0, nc, store);
        break;
      case F16:
        solve_off_ff<RCT, F16>(L, scf, it, b, p, trans, ys, part, r, c0, nc, store);
        break;
      default:
        solve_off_ff<RCT, E4M3>(L, scf, it, b, p, trans, ys, part, r, c0, nc, store);
        break;
    }
  }
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Before a task waits: pull the factor data it will read (final before the
// solve starts) from HBM into L2, one 128-byte line per request, so that
// the reads after the wait hit L2.  A rows x (cols elements of esz bytes)
// block with row stride b.
__device__ __forceinline__ void prefetch_block(const char* base, int b, int esz, int r0, int rows,
                                               int c0, int cols) {
  const int lpr = (cols * esz + 127) / 128;          // lines per row (segments start 128-byte aligned)
  for (int e = threadIdx.x; e < rows * lpr; e += blockDim.x) {
    const int r = r0 + e / lpr, l = e % lpr;
    prefetch_l2(base + ((int64_t)r * b + c0) * esz + 128 * l);
  }
}

__device__ void solve_prefetch(const Arena& A, const ItemSolveDag& it, int op, int i, int j, int p,
                               int trans) {
  const int b = A.b, nt = it.nt;
  if (op == 0) {
    // X = L_ii^{-T}: forward rows t < 32 (p + 1), columns of block p;
    // backward rows of block p, columns t >= 32 p
    const int r0 = trans ? 32 * p : 0, rows = trans ? 32 : 32 * (p + 1);
    const int c0 = trans ? 32 * p : 32 * p, cols = trans ? b - 32 * p : 32;
    if (it.ffdiag) {
      prefetch_block(tile_bytes(A, it.linv[nt + i]), b, 4, r0, rows, c0, cols);
      prefetch_block(tile_bytes(A, it.linv[2 * nt + i]), b, 4, r0, rows, c0, cols);
    } else {
      prefetch_block(tile_bytes(A, it.linv[i]), b, 8, r0, rows, c0, cols);
    }
  } else {
    // L_ij rows of block p (forward), or L_ji's columns of block p (backward)
    const int tile = trans ? it.tiles[j * nt + i] : it.tiles[i * nt + j];
    const int esz = esize(A.tiles[tile].dt);
    if (trans) prefetch_block(tile_bytes(A, tile), b, esz, 0, b, 32 * p, 32);
    else prefetch_block(tile_bytes(A, tile), b, esz, 32 * p, 32, 0, b);
  }
}

template <int RCT>
__global__ void __launch_bounds__(256, RCT == 1 ? 2 : 1)
    k_solve_dag(Arena A, const ItemSolveDag* __restrict__ items, const SolveTask* __restrict__ tasks,
                int ntasks, int* ticket, int trans, const int* gate) {
  if (gated(gate)) return;
  extern __shared__ double sm[];
  double* vs = sm;                               // b x RCT (doubles or float pairs)
  double* part = sm + A.b * RCT;                 // 8 warps x 32 lanes x RCT
  __shared__ int s_t, s_ok;
  const int b = A.b, P = b / 32, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (;;) {
    if (tid == 0) s_t = atomicAdd(ticket, 1);
    __syncthreads();
    const int t = s_t;
    if (t >= ntasks) break;
    const SolveTask tk = tasks[t];
    const int m = (int)(tk & 0xffffff), op = (int)((tk >> 24) & 0xf);
    const int i = (int)((tk >> 28) & 0xfff), j = (int)((tk >> 40) & 0xfff), p = (int)((tk >> 52) & 0xff);
    const ItemSolveDag it = items[m];
    int* cnt = it.cnt;
    const int nt = it.nt;
    solve_prefetch(A, it, op, i, j, p, trans);
    const int CS = 2 * P + 1;                      // counters per tile row
    const int sti = trans ? nt - 1 - i : i;        // i's place in solve order
    if (warp == 0) {
      bool ok = true;
      if (op == 0) {
        // the blocks of in_i this block reads: p' <= p (forward), p' >= p
        // (backward), with their sti - 1 in-place updates and chain product
        if (lane < P && (trans ? lane >= p : lane <= p) && sti >= 1)
          ok = dag_wait(&cnt[i * CS + lane], sti - 1, A.err, A.wait_polls) &&
               dag_wait(&cnt[i * CS + P + 1 + lane], 1, A.err, A.wait_polls);
      } else if (lane == 0) {
        ok = dag_wait(&cnt[j * CS + P], P, A.err, A.wait_polls);
        if (op == 1) ok = ok && dag_wait(&cnt[i * CS + p], trans ? nt - 1 - j : j, A.err, A.wait_polls);
      }
      ok = __all_sync(0xffffffffu, ok);
      if (lane == 0) {
        if (!ok) atomicExch(A.err, 1);
        s_ok = ok;
      }
    }
    __syncthreads();
    if (!s_ok) break;
    if (op == 0) {
      if (it.ffdiag) solve_diag_ff<RCT>(A, it, i, p, trans, vs, part, sti == 0);
      else solve_diag<RCT>(A, it, i, p, trans, vs, part, sti == 0);
    }
    else solve_off<RCT>(A, it, i, j, p, trans, vs, part, op == 2);
    __syncthreads();
    if (tid == 0) {
      if (op == 0) red_release_add(&cnt[i * CS + P], 1);
      else if (op == 1) st_release(&cnt[i * CS + p], trans ? nt - j : j + 1);
      else st_release(&cnt[i * CS + P + 1 + p], 1);
    }
  }
}

// Residual pass 1: one CTA per lower tile of the fixed-point copy of Sigma:
// entries M = Sigma 2^(62 - E) (unsigned, below 2^62), E set by the
// matrix's generation (every entry, the identity padding included, is
// below 2^E).  The CTA scales the two segments of x it reads to integers
// X = x 2^(54 - e), 2^e above the segment's largest magnitude (per
// right-hand side), so each product M X is exact in 128 bits and so is
// every sum of them: a tile's row and column partials are rounded to
// float64 once.  The integer pipe carries the multiply-adds (GB300's FP64
// pipe runs at 1/64 of its FP32 rate).
//
// Columns are split into the fewest groups of at most 32 NCOL (NCOL = 8 for
// one right-hand side per pass, 4 for two: two CTAs fit an SM); the warps
// of a group take rows round-robin.
// For a row, a lane loads its NCOL entries (the next row's loads issued
// before the current row's arithmetic), adds their products with X_j into
// the row's sum (reduced across the warp) and their products with
// X_i[row] into per-column sums (the transposed product).  Group and warp
// sums meet in shared memory through 64-bit atomic adds with the carry
// passed on explicitly: exact integers, so the order does not matter and
// the result is deterministic.  Absolute sums (first iteration only) add
// M >> 42: they only scale the stopping tolerance.
struct s128 {
  uint64_t lo;
  int64_t hi;   // value hi 2^64 + lo
};

// a += m x (m < 2^62, read as signed): the low product with carry out,
// the high product with carry in
__device__ __forceinline__ void mac128(s128& a, uint64_t m, int64_t x) {
  asm("mad.lo.cc.u64 %0, %2, %3, %0;\n\tmadc.hi.s64 %1, %2, %3, %1;"
      : "+l"(a.lo), "+l"(a.hi)
      : "l"(m), "l"(x));
}

__device__ __forceinline__ s128 warp_sum128(s128 a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t ol = __shfl_xor_sync(0xffffffffu, (unsigned long long)a.lo, o);
    const int64_t oh = __shfl_xor_sync(0xffffffffu, (long long)a.hi, o);
    const uint64_t lo = a.lo + ol;
    a.hi += oh + (int64_t)(lo < ol);
    a.lo = lo;
  }
  return a;
}

__device__ __forceinline__ void atomic_add128(unsigned long long* lo, unsigned long long* hi, s128 v) {
  const unsigned long long old = atomicAdd(lo, (unsigned long long)v.lo);
  atomicAdd(hi, (unsigned long long)v.hi + (unsigned long long)(old + v.lo < old));
}

__device__ __forceinline__ double s128_double(unsigned long long lo, unsigned long long hi) {
  return fma((double)(long long)hi, 0x1p64, (double)lo);
}

template <int RC>
__global__ void __launch_bounds__(256, 2) k_residual_tile(Arena A, const ItemResTile* __restrict__ items,
                                                       int want_abs, const int* gate) {
  if (gated(gate)) return;
  constexpr int NCOL = RC == 1 ? 8 : 4;
  extern __shared__ unsigned long long rsm[];
  __shared__ double s_mx[2 * RC][8];
  __shared__ int s_e[2 * RC];
  const ItemResTile it = items[blockIdx.x];
  const int b = A.b, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // column groups: the fewest (1, 2, 4 or 8) with at most 32 NCOL columns
  // each; lane l holds the group's columns l + 32 m below gw
  int G = 1;
  while (b > G * 32 * NCOL) G <<= 1;
  const int W = 8 / G;                                  // warps per group
  const int g = warp / W, wl = warp % W;
  const int gw = b / G;                                 // columns per group
  const int cbase = g * gw;
  const bool diag = it.ti == it.tj;
  const bool full = !diag && gw == 32 * NCOL;
  const int E = *it.sig_e;
  long long* Xj = reinterpret_cast<long long*>(rsm);   // [b][RC]
  long long* Xi = Xj + (size_t)b * RC;                  // [b][RC]
  unsigned long long* yl = rsm + (size_t)2 * b * RC;    // row sums [b][RC], low / high words
  unsigned long long* yh = yl + (size_t)b * RC;
  unsigned long long* cl = yh + (size_t)b * RC;         // column sums [b][RC]
  unsigned long long* ch = cl + (size_t)b * RC;
  unsigned* arow = reinterpret_cast<unsigned*>(ch + (size_t)b * RC);   // [b]
  unsigned* acol = arow + b;                                            // [b]
  const uint64_t* S = tile_ptr<uint64_t>(A, it.tile);
  const double* xjg = it.x + (int64_t)it.tj * b;
  const double* xig = it.x + (int64_t)it.ti * b;
  for (int c0 = 0; c0 < it.nrhs; c0 += RC) {
    const int nc = min(RC, it.nrhs - c0);
    const bool abs_now = want_abs && c0 == 0;
    __syncthreads();
    // the segments' largest magnitudes (a NaN or infinity makes the
    // partials NaN, as float64 arithmetic would)
    double mx[2 * RC];
    bool bad = false;
#pragma unroll
    for (int q = 0; q < 2 * RC; ++q) mx[q] = 0.0;
    for (int t = tid; t < b; t += blockDim.x) {
#pragma unroll
      for (int c = 0; c < RC; ++c) {
        if (c >= nc) break;
        const double vj = xjg[(int64_t)(c0 + c) * it.ld + t], vi = xig[(int64_t)(c0 + c) * it.ld + t];
        bad |= !isfinite(vj) || !isfinite(vi);
        mx[c] = fmax(mx[c], fabs(vj));
        mx[RC + c] = fmax(mx[RC + c], fabs(vi));
      }
    }
#pragma unroll
    for (int q = 0; q < 2 * RC; ++q) {
      mx[q] = warp_max(mx[q]);
      if (lane == 0) s_mx[q][warp] = mx[q];
    }
    bad = __syncthreads_or(bad);
    if (tid < 2 * RC) {
      double m = 0.0;
      for (int w = 0; w < 8; ++w) m = fmax(m, s_mx[tid][w]);
      s_e[tid] = m > 0.0 ? ilogb(m) + 1 : 0;   // |x| < 2^e on the segment
    }
    __syncthreads();
    if (bad) {
      double* pr = it.part + ((size_t)(it.ti * it.nt + it.tj) * it.nrhs) * b;
      double* pc = it.part + ((size_t)(it.tj * it.nt + it.ti) * it.nrhs) * b;
      for (int e = tid; e < b * nc; e += blockDim.x) {
        pr[(size_t)c0 * b + e] = __longlong_as_double(0x7ff8000000000000ll);
        if (!diag) pc[(size_t)c0 * b + e] = __longlong_as_double(0x7ff8000000000000ll);
      }
      continue;
    }
    for (int e = tid; e < b * RC; e += blockDim.x) {
      const int t = e / RC, c = e % RC;
      Xj[e] = c < nc ? __double2ll_rn(ldexp(xjg[(int64_t)(c0 + c) * it.ld + t], 54 - s_e[c])) : 0;
      Xi[e] = c < nc ? __double2ll_rn(ldexp(xig[(int64_t)(c0 + c) * it.ld + t], 54 - s_e[RC + c])) : 0;
      yl[e] = yh[e] = cl[e] = ch[e] = 0ull;
    }
    if (abs_now)
      for (int e = tid; e < b; e += blockDim.x) arow[e] = acol[e] = 0u;
    __syncthreads();
    s128 cacc[NCOL][RC];
    unsigned cabs[NCOL];
#pragma unroll
    for (int m = 0; m < NCOL; ++m) {
      cabs[m] = 0u;
#pragma unroll
      for (int c = 0; c < RC; ++c) cacc[m][c] = s128{0ull, 0ll};
    }
    uint64_t cur[NCOL], nxt[NCOL];
    int r = wl;
#pragma unroll
    for (int m = 0; m < NCOL; ++m)
      cur[m] = (lane + 32 * m < gw && r < b) ? S[(int64_t)r * b + cbase + lane + 32 * m] : 0ull;
    for (; r < b; r += W) {
      const int rn = r + W;
#pragma unroll
      for (int m = 0; m < NCOL; ++m)
        nxt[m] = (lane + 32 * m < gw && rn < b) ? S[(int64_t)rn * b + cbase + lane + 32 * m] : 0ull;
      // a diagonal tile holds its lower half: row r uses columns <= r, and
      // the transposed product takes the columns < r
      s128 dot[RC];
#pragma unroll
      for (int c = 0; c < RC; ++c) dot[c] = s128{0ull, 0ll};
      unsigned ra = 0u;
      if (full && !abs_now) {   // an off-diagonal tile, every lane's NCOL columns in it
#pragma unroll
        for (int m = 0; m < NCOL; ++m) {
          const int col = cbase + lane + 32 * m;
#pragma unroll
          for (int c = 0; c < RC; ++c) {
            mac128(dot[c], cur[m], Xj[col * RC + c]);
            mac128(cacc[m][c], cur[m], Xi[r * RC + c]);
          }
        }
      } else {
#pragma unroll
        for (int m = 0; m < NCOL; ++m) {
          const int col = cbase + lane + 32 * m;
          const bool in = lane + 32 * m < gw;
          const uint64_t sv = (in && (!diag || col <= r)) ? cur[m] : 0ull;
          const uint64_t tv = (!diag || col < r) ? sv : 0ull;
#pragma unroll
          for (int c = 0; c < RC; ++c) {
            mac128(dot[c], sv, Xj[(in ? col : 0) * RC + c]);
            mac128(cacc[m][c], tv, Xi[r * RC + c]);
          }
          if (abs_now) {
            ra += (unsigned)(sv >> 42);
            cabs[m] += (unsigned)(tv >> 42);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < RC; ++c) dot[c] = warp_sum128(dot[c]);
      if (abs_now)
        for (int o = 16; o > 0; o >>= 1) ra += __shfl_xor_sync(0xffffffffu, ra, o);
      if (lane == 0) {
#pragma unroll
        for (int c = 0; c < RC; ++c) atomic_add128(&yl[r * RC + c], &yh[r * RC + c], dot[c]);
        if (abs_now) atomicAdd(&arow[r], ra);
      }
#pragma unroll
      for (int m = 0; m < NCOL; ++m) cur[m] = nxt[m];
    }
#pragma unroll
    for (int m = 0; m < NCOL; ++m) {
      if (lane + 32 * m >= gw) break;
      const int col = cbase + lane + 32 * m;
#pragma unroll
      for (int c = 0; c < RC; ++c) atomic_add128(&cl[col * RC + c], &ch[col * RC + c], cacc[m][c]);
      if (abs_now) atomicAdd(&acol[col], cabs[m]);
    }
    __syncthreads();
    // the partials: float64, each rounded once from its exact sum
    double* pr = it.part + ((size_t)(it.ti * it.nt + it.tj) * it.nrhs) * b;
    double* pc = it.part + ((size_t)(it.tj * it.nt + it.ti) * it.nrhs) * b;
    for (int e = tid; e < b * nc; e += blockDim.x) {
      const int c = e / b, t = e % b, k = t * RC + c;
      if (diag) {   // x_i = x_j: one scale; the two sums added exactly first
        const unsigned long long lo = yl[k] + cl[k];
        const unsigned long long hi = yh[k] + ch[k] + (lo < yl[k]);
        pr[(size_t)(c0 + c) * b + t] = ldexp(s128_double(lo, hi), E - 62 + s_e[c] - 54);
      } else {
        pr[(size_t)(c0 + c) * b + t] = ldexp(s128_double(yl[k], yh[k]), E - 62 + s_e[c] - 54);
        pc[(size_t)(c0 + c) * b + t] = ldexp(s128_double(cl[k], ch[k]), E - 62 + s_e[RC + c] - 54);
      }
    }
    if (abs_now) {
      float* ar = it.pabs + (size_t)(it.ti * it.nt + it.tj) * b;
      float* ac = it.pabs + (size_t)(it.tj * it.nt + it.ti) * b;
      for (int t = tid; t < b; t += blockDim.x) {
        if (diag) ar[t] = ldexpf((float)(arow[t] + acol[t]), E - 62 + 42);
        else {
          ar[t] = ldexpf((float)arow[t], E - 62 + 42);
          ac[t] = ldexpf((float)acol[t], E - 62 + 42);
        }
      }
    }
  }
}

// Residual pass 2: r_i = z_i - sum_j part(i, j), j in increasing order.
__global__ void __launch_bounds__(256) k_residual_rows(int b, const ItemResRow* __restrict__ items,
                                                       int want_abs, const int* gate) {
  if (gated(gate)) return;
  const ItemResRow it = items[blockIdx.x];
  const int t = blockIdx.y * blockDim.x + threadIdx.x;
  if (t >= b) return;
  const int64_t g = (int64_t)it.ti * b + t;
  for (int c = 0; c < it.nrhs; ++c) {
    double acc = 0.0;
    for (int j = 0; j < it.nt; ++j) acc += it.part[((size_t)(it.ti * it.nt + j) * it.nrhs + c) * b + t];
    it.r[(int64_t)c * it.ld + g] = it.z[(int64_t)c * it.ld + g] - acc;
  }
  if (want_abs && it.rowabs) {
    double a = 0.0;
    for (int j = 0; j < it.nt; ++j) a += (double)it.pabs[(size_t)(it.ti * it.nt + j) * b + t];
    it.rowabs[g] = a;
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

// A bounded wait that ran out in the factorisation or the solves leaves the
// error word set: the log-likelihood is then NaN, not a number computed
// from an unfinished solve.
__global__ void k_loglik(const double* logdet, const double* quad, int64_t n, int nrhs,
                         double* ll, const int* err) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nrhs) return;
  const double log2pi = 1.8378770664093454836;   // log(2 pi)
  ll[c] = *err ? __longlong_as_double(0x7ff8000000000000LL)
               : -0.5 * (double)n * log2pi - 0.5 * logdet[0] - 0.5 * quad[c];
}

}  // namespace

std::vector<SolveTask> solve_dag_tasks(const std::vector<int>& nts, int P, int trans) {
  // per matrix, rows in solve order s_0, s_1, ...: D(s_0), then per step t
  // the chain products of s_{t+1} with out_{s_t} and at once the diagonal
  // blocks of s_{t+1} (the critical chain, handed out together), then the
  // in-place updates of the rows s_{t+2}.. with out_{s_t}, which run while
  // the chain waits; the in-place updates of a row come in solve order of
  // their columns.  Matrices are interleaved round-robin, which keeps each
  // matrix's order.
  std::vector<std::vector<SolveTask>> per(nts.size());
  auto pack = [](int m, int op, int i, int j, int p) {
    return (SolveTask)m | ((SolveTask)op << 24) | ((SolveTask)i << 28) | ((SolveTask)j << 40) |
           ((SolveTask)p << 52);
  };
  size_t total = 0;
  for (size_t m = 0; m < nts.size(); ++m) {
    const int nt = nts[m];
    auto& v = per[m];
    auto row = [&](int st) { return trans ? nt - 1 - st : st; };
    auto blk = [&](int q) { return trans ? P - 1 - q : q; };
    for (int q = 0; q < P; ++q) v.push_back(pack((int)m, 0, row(0), 0, blk(q)));
    for (int st = 0; st + 1 < nt; ++st) {
      for (int q = 0; q < P; ++q) v.push_back(pack((int)m, 2, row(st + 1), row(st), blk(q)));
      for (int q = 0; q < P; ++q) v.push_back(pack((int)m, 0, row(st + 1), 0, blk(q)));
      for (int u = st + 2; u < nt; ++u)
        for (int q = 0; q < P; ++q) v.push_back(pack((int)m, 1, row(u), row(st), q));
    }
    total += v.size();
  }
  std::vector<SolveTask> out;
  out.reserve(total);
  for (size_t k = 0; out.size() < total; ++k)
    for (auto& v : per)
      if (k < v.size()) out.push_back(v[k]);
  return out;
}

void launch_solve_dag(const Arena& A, const ItemSolveDag* items, const SolveTask* tasks, int ntasks,
                      int* ticket, int trans, int nrhs_max, const int* gate, cudaStream_t s) {
  if (ntasks <= 0) return;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_solve_dag<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    cudaFuncSetAttribute(k_solve_dag<RCMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  }
  const int rc = nrhs_max == 1 ? 1 : RCMAX;
  const size_t smem = sizeof(double) * ((size_t)A.b * rc + 8 * 32 * rc);
  const int grid = std::min(ntasks, 2 * sms);
  if (rc == 1) k_solve_dag<1><<<grid, 256, smem, s>>>(A, items, tasks, ntasks, ticket, trans, gate);
  else k_solve_dag<RCMAX><<<grid, 256, smem, s>>>(A, items, tasks, ntasks, ticket, trans, gate);
}

void launch_residual(const Arena& A, const ItemResTile* tiles, int ntiles, const ItemResRow* rows,
                     int nrows, int nrhs, int want_rowabs, const int* gate, cudaStream_t s) {
  if (ntiles <= 0) return;
  const int b = A.b;
  const int rc = nrhs == 1 ? 1 : 2;
  // X_j, X_i, row and column sums (two words each), absolute sums
  const size_t smem = sizeof(unsigned long long) * (size_t)b * rc * 6 + sizeof(unsigned) * (size_t)b * 2;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_residual_tile<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_residual_tile<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  if (rc == 1) k_residual_tile<1><<<ntiles, 256, smem, s>>>(A, tiles, want_rowabs, gate);
  else k_residual_tile<2><<<ntiles, 256, smem, s>>>(A, tiles, want_rowabs, gate);
  k_residual_rows<<<dim3(nrows, (b + 255) / 256), 256, 0, s>>>(b, rows, want_rowabs, gate);
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
                   const int* err, cudaStream_t s) {
  k_loglik<<<(nrhs + 127) / 128, 128, 0, s>>>(logdet, quad, n, nrhs, ll, err);
}

}  // namespace mp
