// Trailing updates of the tiled Cholesky, A_ij -= A_ik A_jk^T (SYRK when
// i == j), on CUDA cores.
//
// k_update_f32 serves every product whose precision (the update rule
// min(p(target), max(p(A), p(B))), after Sec. 4.3's "highest input
// precision wins" capped by the target) is below FP64: FP32, BF16, FP16 or
// E4M3.  Operands arrive already in the product's format (the planner
// substitutes a tile's rounded shadow copy where the tile is stored in a
// wider format), so every operand value is exact in FP32; products of two
// 16-bit or 8-bit values are exact in FP32 and the sum accumulates in FP32.
// E4M3 operands use their codes; the FP32 sum is multiplied by the two
// power-of-two scales.  The epilogue subtracts from the target:
//   FP64 target  in float64,
//   FP32 target  one FP32 subtraction (correctly rounded, so the exact
//                difference of the two FP32 values rounded once),
//   16-bit       in FP32, rounded to the target format,
//   E4M3         in FP32 into a scratch slot plus the slot's amax; the
//                target is rounded with its new scale by k_fp8_round.
// k_update_f64 is the FP64 product (all-FP64 maps).
#include "mp_device.cuh"

namespace mp {

namespace {

constexpr int BM = 128, BK = 16;

__global__ void __launch_bounds__(256) k_update_f32(Arena A, const ItemUpd* __restrict__ items) {
  __shared__ __align__(16) float As[BK][BM + 4];
  __shared__ __align__(16) float Bs[BK][BM + 4];
  const ItemUpd it = items[blockIdx.x];
  const int b = A.b, tid = threadIdx.x;
  const int nsub = b / BM;
  const int rb = blockIdx.y / nsub, cb = blockIdx.y % nsub;
  if (it.syrk && cb > rb) return;
  const TileRef ra = A.tiles[it.a], rbt = A.tiles[it.b];
  const char* pa = tile_bytes(A, it.a);
  const char* pb = tile_bytes(A, it.b);
  const float sab = (float)(A.scale[it.a] * A.scale[it.b]);
  const int lr = tid >> 1, lh = (tid & 1) * 8;
  const int64_t arow = (int64_t)(rb * BM + lr) * b, brow = (int64_t)(cb * BM + lr) * b;
  const int ty = tid / 16, tx = tid % 16;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  for (int t0 = 0; t0 < b; t0 += BK) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      As[lh + q][lr] = load_f32(pa, ra.dt, arow + t0 + lh + q);
      Bs[lh + q][lr] = load_f32(pb, rbt.dt, brow + t0 + lh + q);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float av[8], bv[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) av[i] = As[kk][ty * 8 + i];
#pragma unroll
      for (int j = 0; j < 8; ++j) bv[j] = Bs[kk][tx * 8 + j];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
  const TileRef rc = A.tiles[it.c];
  char* pc = tile_bytes(A, it.c);
  const double sc = A.scale[it.c];
  float mx = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t row = (int64_t)(rb * BM + ty * 8 + i) * b + cb * BM + tx * 8;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t o = row + j;
      const float p = acc[i][j] * sab;
      switch (rc.dt) {
        case F64: reinterpret_cast<double*>(pc)[o] -= (double)p; break;
        case F32: {
          float* c = reinterpret_cast<float*>(pc);
          c[o] = __fsub_rn(c[o], p);        // correctly rounded: the exact difference rounded once
          break;
        }
        case E4M3: {
          float v = load_f32(pc, E4M3, o) * (float)sc - p;
          it.v[o] = v;
          mx = fmaxf(mx, fabsf(v));
          break;
        }
        default: store_round_f32(pc, rc.dt, o, load_f32(pc, rc.dt, o) - p);
      }
    }
  }
  if (rc.dt == E4M3) {
    __shared__ float red[8];
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((tid & 31) == 0) red[tid >> 5] = mx;
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < 8; ++w) mx = fmaxf(mx, red[w]);
      atomic_max_pos(&A.amax[it.vslot], (double)mx);
    }
  }
}

constexpr int DM = 64, DK = 16;

__global__ void __launch_bounds__(256) k_update_f64(Arena A, const ItemUpd* __restrict__ items) {
  __shared__ double As[DK][DM + 1];
  __shared__ double Bs[DK][DM + 1];
  const ItemUpd it = items[blockIdx.x];
  const int b = A.b, tid = threadIdx.x;
  const int nsub = b / DM;
  const int rb = blockIdx.y / nsub, cb = blockIdx.y % nsub;
  if (it.syrk && cb > rb) return;
  const double* pa = tile_ptr<double>(A, it.a);
  const double* pb = tile_ptr<double>(A, it.b);
  double* pc = tile_ptr<double>(A, it.c);
  const int lr = tid >> 2, lq = (tid & 3) * 4;
  const int ty = tid / 16, tx = tid % 16;
  double acc[4][4] = {};
  for (int t0 = 0; t0 < b; t0 += DK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      As[lq + q][lr] = pa[(int64_t)(rb * DM + lr) * b + t0 + lq + q];
      Bs[lq + q][lr] = pb[(int64_t)(cb * DM + lr) * b + t0 + lq + q];
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < DK; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
      pc[(int64_t)(rb * DM + ty + 16 * i) * b + cb * DM + tx + 16 * j] -= acc[i][j];
}

__global__ void __launch_bounds__(256) k_fp8_round(Arena A, const ItemFp8* __restrict__ items) {
  const ItemFp8 it = items[blockIdx.x];
  const int b = A.b;
  const double s = e4m3_scale(amax_value(&A.amax[it.vslot]));
  char* dst = tile_bytes(A, it.tile);
  const int64_t r0 = (int64_t)blockIdx.y * 16 * b;
  for (int e = threadIdx.x; e < 16 * b; e += blockDim.x)
    store_round(dst, E4M3, r0 + e, (double)it.v[r0 + e] / s);
  if (blockIdx.y == 0 && threadIdx.x == 0) A.scale[it.tile] = s;
}

}  // namespace

void launch_update_f32(const Arena& A, const ItemUpd* items, int count, cudaStream_t s) {
  if (count <= 0) return;
  int nsub = A.b / BM;
  k_update_f32<<<dim3(count, nsub * nsub), 256, 0, s>>>(A, items);
}

void launch_update_f64(const Arena& A, const ItemUpd* items, int count, cudaStream_t s) {
  if (count <= 0) return;
  int nsub = A.b / DM;
  k_update_f64<<<dim3(count, nsub * nsub), 256, 0, s>>>(A, items);
}

void launch_fp8_round(const Arena& A, const ItemFp8* items, int count, cudaStream_t s) {
  if (count <= 0) return;
  k_fp8_round<<<dim3(count, A.b / 16), 256, 0, s>>>(A, items);
}

}  // namespace mp
