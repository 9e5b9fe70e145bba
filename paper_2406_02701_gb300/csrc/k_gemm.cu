// Standalone per-precision matrix product C = alpha op(A) op(B) + beta C
// (the paper's `%*%` / `crossprod`, Sec. 5, run in the operands' precision).
// Column-major operands of one storage format; products accumulate in FP32
// (FP64 for FP64 operands); the epilogue is float64 for FP64/FP32 targets and
// FP32 for 16-/8-bit ones, and rounds once into the format.  CUDA-core
// kernel with 64 x 64 output tiles and bounds checks for ragged edges.
#include "mp_device.cuh"

namespace mp {

namespace {

constexpr int GM = 64, GK = 16;

template <typename Acc>
__global__ void __launch_bounds__(256) k_gemm(int dt, int ta, int tb, int64_t m, int64_t n,
                                              int64_t k, double alpha, const char* A, int64_t lda,
                                              const char* B, int64_t ldb, double beta, char* C,
                                              int64_t ldc) {
  __shared__ Acc As[GK][GM + 1];
  __shared__ Acc Bs[GK][GM + 1];
  const int tid = threadIdx.x;
  const int64_t i0 = (int64_t)blockIdx.x * GM, j0 = (int64_t)blockIdx.y * GM;
  const int ty = tid / 16, tx = tid % 16;
  Acc acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = Acc(0);
  for (int64_t t0 = 0; t0 < k; t0 += GK) {
    for (int e = tid; e < GK * GM; e += blockDim.x) {
      const int kk = e / GM, rr = e % GM;
      const int64_t i = i0 + rr, j = j0 + rr, t = t0 + kk;
      Acc av = Acc(0), bv = Acc(0);
      if (i < m && t < k) {
        int64_t o = ta ? t + i * lda : i + t * lda;
        av = sizeof(Acc) == 8 ? (Acc)load_f64(A, dt, o) : (Acc)load_f32(A, dt, o);
      }
      if (j < n && t < k) {
        int64_t o = tb ? j + t * ldb : t + j * ldb;
        bv = sizeof(Acc) == 8 ? (Acc)load_f64(B, dt, o) : (Acc)load_f32(B, dt, o);
      }
      As[kk][rr] = av;
      Bs[kk][rr] = bv;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      Acc a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t r = i0 + ty + 16 * i, c = j0 + tx + 16 * j;
      if (r >= m || c >= n) continue;
      const int64_t o = r + c * ldc;
      if (dt == F64 || dt == F32) {
        double v = alpha * (double)acc[i][j];
        if (beta != 0.0) v += beta * load_f64(C, dt, o);
        store_round(C, dt, o, v);
      } else {
        float v = (float)alpha * (float)acc[i][j];
        if (beta != 0.0) v += (float)beta * load_f32(C, dt, o);
        store_round_f32(C, dt, o, v);
      }
    }
}

}  // namespace

void launch_gemm(int dt, int ta, int tb, int64_t m, int64_t n, int64_t k, double alpha,
                 const void* A, int64_t lda, const void* B, int64_t ldb, double beta, void* C,
                 int64_t ldc, cudaStream_t s) {
  dim3 grid((unsigned)((m + GM - 1) / GM), (unsigned)((n + GM - 1) / GM));
  if (dt == F64)
    k_gemm<double><<<grid, 256, 0, s>>>(dt, ta, tb, m, n, k, alpha, (const char*)A, lda,
                                         (const char*)B, ldb, beta, (char*)C, ldc);
  else
    k_gemm<float><<<grid, 256, 0, s>>>(dt, ta, tb, m, n, k, alpha, (const char*)A, lda,
                                        (const char*)B, ldb, beta, (char*)C, ldc);
}

}  // namespace mp
