// Standalone per-precision matrix product on the tcgen05 tensor cores:
// C = alpha op(A) op(B) + beta C (the paper's `%*%` / `crossprod`, Sec. 5,
// run in the operands' precision) for BF16, FP16, E4M3 (codes, scale 1)
// and FP32 (three TF32 products of hi/lo splits).
//
// The product reuses the persistent tensor-core update kernel of the
// factorisation (k_update_tc_p: TMA-fed operands, FP32 accumulators in
// tensor memory, one warp issuing the MMAs) on a workspace arena of
// gb x gb tiles:
//   pack     op(A) into row tiles A(i, kk) and op(B)^T into B(j, kk), each
//            row-major with the contraction index contiguous (K-major, the
//            layout of the MMA descriptors), zero beyond the matrix; the
//            values keep their storage format (FP32: split into a TF32 hi
//            part and the FP32 remainder lo).  Column-major sources are
//            transposed through shared memory in 32 x 32 blocks.
//   update   for kk = 0 .. kt-1 one launch over all (i, j): the FP32 tile
//            C(i, j) -= A(i, kk) B(j, kk)^T (within a tile the accumulation
//            is the tensor cores' FP32; across tiles one IEEE FP32
//            subtraction each).  Tiles of one target are never in one
//            launch together, so no two CTAs write the same tile.
//   finish   C = alpha (-acc) + beta C, in float64 for an FP32 target and
//            FP32 for 16-/8-bit ones, rounded once into the format.
// The workspace is allocated and freed on the stream (stream-ordered).
#include <cuda.h>

#include <algorithm>
#include <vector>

#include "mp_device.cuh"

namespace mp {

namespace {

// op(X) rows r0.. of a tile: tile (ti, tk) of a (rows x K) operand holds
// element (r, c) = op(X)[ti gb + r][tk gb + c]; op(X)[r][t] = X[r + t ld]
// when `rowcol` (X stored rows x K) else X[t + r ld] (X stored K x rows).
// F32 sources write hi (TF32, round to nearest, ties away) and lo.
__global__ void __launch_bounds__(256) k_pack(const char* __restrict__ X, int dt, int64_t ld,
                                              int rowcol, int64_t rows, int64_t K, int gb, int mt,
                                              char* __restrict__ dst, float* __restrict__ dst_lo) {
  __shared__ float s[32][33];
  __shared__ uint8_t raw[32][33 * 2];
  const int64_t tile = blockIdx.z;                 // ti * kt + tk
  const int kt = (int)((K + gb - 1) / gb);
  const int ti = (int)(tile / kt), tk = (int)(tile % kt);
  (void)mt;
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;   // column block (K), row block
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  const int es = (int)esize(dt);
  const int64_t R0 = (int64_t)ti * gb + by, C0 = (int64_t)tk * gb + bx;
  // read a 32 x 32 block with the source's contiguous index along tx
  for (int q = ty; q < 32; q += 8) {
    int64_t r, c;
    if (rowcol) { r = R0 + tx; c = C0 + q; }     // X[r + c ld]: r contiguous
    else        { r = R0 + q;  c = C0 + tx; }    // X[c + r ld]: c contiguous
    const bool in = r < rows && c < K;
    const int64_t o = rowcol ? r + c * ld : c + r * ld;
    const int lr = rowcol ? tx : q, lc = rowcol ? q : tx;
    if (dt == F32) {
      s[lr][lc] = in ? reinterpret_cast<const float*>(X)[o] : 0.f;
    } else {
      for (int e = 0; e < es; ++e) raw[lr][lc * es + e] = in ? (uint8_t)X[o * es + e] : 0;
    }
  }
  __syncthreads();
  // write row-major: element (by + q, bx + tx) of the tile
  for (int q = ty; q < 32; q += 8) {
    const int64_t off = (tile * gb + by + q) * gb + bx + tx;
    if (dt == F32) {
      const float v = s[q][tx];
      uint32_t hb;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(v));
      reinterpret_cast<float*>(dst)[off] = __uint_as_float(hb);
      dst_lo[off] = v - __uint_as_float(hb);
    } else {
      for (int e = 0; e < es; ++e) dst[off * es + e] = (char)raw[q][tx * es + e];
    }
  }
}

// C = alpha (-acc) + beta C, rounded once into the format.
__global__ void k_finish(const float* __restrict__ acc, int gb, int nt, int dt, int64_t m, int64_t n,
                         double alpha, double beta, char* __restrict__ C, int64_t ldc) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * n) return;
  const int64_t r = idx % m, c = idx / m;               // column-major: consecutive threads, one column
  const int64_t tile = (r / gb) * nt + c / gb;
  const float p = -acc[(tile * gb + r % gb) * gb + c % gb];
  const int64_t o = r + c * ldc;
  if (dt == F32) {
    double v = alpha * (double)p;
    if (beta != 0.0) v += beta * load_f64(C, dt, o);
    store_round(C, dt, o, v);
  } else {
    float v = (float)alpha * p;
    if (beta != 0.0) v += (float)beta * load_f32(C, dt, o);
    store_round_f32(C, dt, o, v);
  }
}

typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                             const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                             CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                             CUtensorMapFloatOOBfill);

EncodeFn encoder() {
  static EncodeFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<EncodeFn>(f);
  }();
  return fn;
}

}  // namespace

int gemm_tc_tile(int64_t m, int64_t n, int64_t k) {
  const int64_t s = std::min(std::min(m, n), k);
  return s >= 4096 ? 512 : s >= 1024 ? 256 : 128;
}

// Returns 0 on success, 1 for an allocation failure, 2 for another CUDA or
// driver failure (the caller reports it), 3 when the sizes exceed the tile
// layout's limits (nothing was enqueued).
int launch_gemm_tc(int dt, int ta, int tb, int64_t m, int64_t n, int64_t k, double alpha,
                   const void* A, int64_t lda, const void* B, int64_t ldb, double beta, void* C,
                   int64_t ldc, cudaStream_t s) {
  EncodeFn encode = encoder();
  if (!encode) return 2;
  const int gb = gemm_tc_tile(m, n, k);
  const int64_t mt = (m + gb - 1) / gb, nt = (n + gb - 1) / gb, kt = (k + gb - 1) / gb;
  // launch-grid and 32-bit row limits of the tile layout (the caller falls
  // back to the CUDA-core kernel beyond them)
  if (mt * kt > 65535 || nt * kt > 65535 || (2 * (mt + nt) * kt + mt * nt) * gb >= (int64_t)1 << 31) return 3;
  const int es = (int)esize(dt);
  const int64_t tsz = (int64_t)gb * gb;
  const bool f32 = dt == F32;
  // pools: the operand format (A tiles, then B tiles; F32: hi tiles, then lo
  // tiles) and the FP32 accumulators (after the operand tiles in the F32 pool)
  const int64_t na = mt * kt, nb = nt * kt, nc = mt * nt;
  const int64_t op_tiles = f32 ? 2 * (na + nb) : na + nb;
  const size_t op_bytes = (size_t)op_tiles * tsz * es;
  const size_t acc_bytes = (size_t)nc * tsz * 4;
  const int64_t ntiles = op_tiles + nc;
  std::vector<TileRef> refs(ntiles);
  for (int64_t t = 0; t < op_tiles; ++t) refs[t] = TileRef{dt, (int32_t)t};
  for (int64_t t = 0; t < nc; ++t) refs[op_tiles + t] = TileRef{F32, (int32_t)((f32 ? op_tiles : 0) + t)};
  const size_t meta = sizeof(TileRef) * ntiles + sizeof(double) * ntiles + sizeof(unsigned long long) + 256;
  char* ws = nullptr;
  const size_t total = op_bytes + acc_bytes + meta + 2048;
  if (cudaMallocAsync((void**)&ws, total, s) != cudaSuccess) return 1;
  char* pool_op = ws;
  float* acc = reinterpret_cast<float*>(ws + ((op_bytes + 1023) & ~size_t(1023)));
  char* mbase = reinterpret_cast<char*>(acc) + acc_bytes;
  TileRef* d_refs = reinterpret_cast<TileRef*>(mbase);
  double* d_scale = reinterpret_cast<double*>(mbase + sizeof(TileRef) * ntiles);
  int* d_err = reinterpret_cast<int*>(d_scale + ntiles);
  std::vector<double> ones(ntiles, 1.0);
  int rc = 0;
  if (cudaMemcpyAsync(d_refs, refs.data(), sizeof(TileRef) * ntiles, cudaMemcpyHostToDevice, s) ||
      cudaMemcpyAsync(d_scale, ones.data(), sizeof(double) * ntiles, cudaMemcpyHostToDevice, s) ||
      cudaMemsetAsync(d_err, 0, sizeof(int), s) || cudaMemsetAsync(acc, 0, acc_bytes, s))
    rc = 2;
  Arena Ar{};
  for (int d = 0; d < NDT; ++d) Ar.pool[d] = nullptr;
  Ar.pool[dt] = pool_op;
  if (!f32) Ar.pool[F32] = reinterpret_cast<char*>(acc);
  else Ar.pool[F32] = pool_op;      // accumulators follow the splits in the same pool
  Ar.tiles = d_refs;
  Ar.scale = d_scale;
  Ar.amax = reinterpret_cast<unsigned long long*>(d_err + 2);
  Ar.err = d_err;
  Ar.b = gb;
  // pack: A rows = m (op(A) = A when ta = 0, stored m x k), B rows = n
  // (op(B)^T: element (j, t) = B[t + j ldb] when tb = 0 (B stored k x n,
  // t contiguous), B[j + t ldb] when tb = 1)
  if (!rc) {
    const dim3 blk(256);
    char* a_dst = pool_op;
    char* b_dst = pool_op + (size_t)na * tsz * es;
    float* a_lo = f32 ? reinterpret_cast<float*>(pool_op) + (na + nb) * tsz : nullptr;
    float* b_lo = f32 ? a_lo + na * tsz : nullptr;
    k_pack<<<dim3(gb / 32, gb / 32, (unsigned)na), blk, 0, s>>>((const char*)A, dt, lda, ta ? 0 : 1, m, k, gb,
                                                                (int)mt, a_dst, a_lo);
    k_pack<<<dim3(gb / 32, gb / 32, (unsigned)nb), blk, 0, s>>>((const char*)B, dt, ldb, tb ? 1 : 0, n, k, gb,
                                                                (int)nt, b_dst, b_lo);
  }
  // the operand pool as one (tiles * gb) x gb row-major matrix
  CUtensorMap map{};
  if (!rc) {
    const CUtensorMapDataType ty = dt == F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : dt == BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                   : dt == F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                               : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    cuuint64_t dims[2] = {(cuuint64_t)gb, (cuuint64_t)op_tiles * gb};
    cuuint64_t strides[1] = {(cuuint64_t)gb * es};
    cuuint32_t box[2] = {(cuuint32_t)(128 / es), 128};
    cuuint32_t estr[2] = {1, 1};
    if (encode(&map, ty, 2, pool_op, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      rc = 2;
  }
  // items: a unit contracts over up to `span` tiles (K <= 4096) in tensor
  // memory; one launch per group of contraction tiles, so the accumulator
  // tiles are read and written once per group
  const int64_t span = std::max<int64_t>(1, std::min<int64_t>(kt, 4096 / gb));
  const int64_t groups = (kt + span - 1) / span;
  ItemTC* d_items = nullptr;
  if (!rc && cudaMallocAsync((void**)&d_items, sizeof(ItemTC) * nc * groups, s) != cudaSuccess) rc = 1;
  if (!rc) {
    std::vector<ItemTC> all((size_t)(nc * groups));
    for (int64_t g = 0; g < groups; ++g)
      for (int64_t i = 0; i < mt; ++i)
        for (int64_t j = 0; j < nt; ++j) {
          const int64_t kk = g * span;
          ItemTC u{};
          u.c = (int32_t)(op_tiles + i * nt + j);
          u.a = (int32_t)(i * kt + kk);
          u.b = (int32_t)(na + j * kt + kk);
          u.a2 = f32 ? (int32_t)(na + nb + i * kt + kk) : -1;
          u.b2 = f32 ? (int32_t)(na + nb + na + j * kt + kk) : -1;
          u.syrk = 0;
          u.vslot = -1;
          u.kspan = (int32_t)std::min<int64_t>(span, kt - kk);
          u.v = nullptr;
          all[(size_t)(g * nc + i * nt + j)] = u;
        }
    if (cudaMemcpyAsync(d_items, all.data(), sizeof(ItemTC) * all.size(), cudaMemcpyHostToDevice, s)) rc = 2;
    for (int64_t g = 0; g < groups && !rc; ++g) launch_update_tc(Ar, dt, d_items + g * nc, (int)nc, map, s);
  }
  if (!rc) {
    const int64_t total_mn = m * n;
    k_finish<<<(unsigned)((total_mn + 255) / 256), 256, 0, s>>>(acc, gb, (int)nt, dt, m, n, alpha, beta,
                                                                (char*)C, ldc);
  }
  if (d_items) cudaFreeAsync(d_items, s);
  cudaFreeAsync(ws, s);
  if (!rc && cudaPeekAtLastError() != cudaSuccess) rc = 2;
  return rc;
}

}  // namespace mp
