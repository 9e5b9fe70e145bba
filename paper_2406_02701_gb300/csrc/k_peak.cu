// FP64 FMA throughput probe: the roofline denominator of the FP64 kernels
// (panel TRSM, diagonal POTRF), whose bound is the DFMA pipe.  Eight
// independent FMA chains per thread, 8 resident CTAs of 256 threads per SM.
#include <vector>

#include "../../include/mpchol.h"
#include "mp_internal.h"

namespace {

__global__ void k_dfma_loop(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  double x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

}  // namespace

extern "C" mp_status mp_probe_fp64_peak(int device, double* h_tflops) {
  if (!h_tflops) return MP_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return MP_ERR_ARG;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int blocks = sms * 8, threads = 256, iters = 200;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) return MP_ERR_OOM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_dfma_loop<<<blocks, threads>>>(out, 10, 0.999, 0.001);
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0);
    k_dfma_loop<<<blocks, threads>>>(out, iters, 0.999, 0.001);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return MP_ERR_CUDA;
  *h_tflops = 2.0 * 8 * 16 * (double)iters * blocks * threads / (best * 1e-3) / 1e12;
  return MP_OK;
}
