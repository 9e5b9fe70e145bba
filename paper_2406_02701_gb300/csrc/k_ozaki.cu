// Panel triangular solve X = A L_kk^{-T} = A W on the tensor cores, with
// float64-class accuracy, by exact integer-slice arithmetic (the Ozaki
// scheme: error-free splitting of both operands into short integer digits
// whose products and sums are exact in FP32).
//
//   rows of A:    a = sigma_r sum_p d_p 2^(-6(p+1)),  p < S
//   columns of W: w = tau_c   sum_q e_q 2^(-6(q+1)),  q < S
// with sigma_r, tau_c powers of two bounding the row / column; the digits
// represent the entry rounded to the nearest multiple of 2^(-6S) (ties to
// even) with |d_0| <= 64 and every later digit <= 32, so a digit is an
// integer of at most 7 bits, exact in BF16 (A: S steps d = rint(64 r) on
// the FP32 pipe; W: the balanced base-64 digits of rint(w 2^(6S) / tau_c)
// in integer arithmetic -- the same represented value).  For one
// level l = p + q the products d_p e_q summed over K = b are integers of
// magnitude at most K 2^12 (l = 0) or K (l + 3) 2^10 (l >= 1); for S = 8 and
// K <= 1024 that is below 2^24, so every level accumulates exactly in an
// FP32 tensor-memory accumulator of a kind::f16 BF16 MMA (the S = 8 levels
// of a 128 x 64 output block fill the 512 TMEM columns).  Levels l >= S are
// dropped:
//   X = sigma_r tau_c sum_{l < S} 2^(-6(l+2)) sum_{p+q=l} (D_p E_q^T)
// which, with the digits' own remainders, leaves an error of at most
// K (1 + (S + 3) / 3) 2^(-6S) sigma_r tau_c (about 8.5e-12 sigma_r tau_c
// for K = 512 and S = 8).  The levels are added from the smallest to the
// largest in float-float (pairs of FP32 numbers: about S^2 2^-48 relative
// error), scaled by the power of two sigma_r tau_c, and written in float64.
// The splits hold S = 8 digits; a unit uses the first s of them (dropping a
// digit only moves more of the operand into the dropped levels, so the bound
// holds with s in place of S), s = ozaki_digits of the panel tile's format:
// the smallest s whose bound at K = 1024 sits 2^11 below half a unit in the
// last place of that format (FP32 8, BF16 and FP16 6, E4M3 5), so a 16-bit
// tile takes 8 MMAs per K slice instead of 12 and an E4M3 tile 6.
//
// Data movement of the product (one work unit = 128 rows x 64 columns of
// X; persistent CTAs walk the units): per K chunk of 64, the S digit chunks
// of W^T (S x 8 KB, adjacent in shared memory) are loaded once into a
// two-slot ring and the S digit chunks of A (16 KB each) stream through a
// three-slot ring; A_p meets the W digits 0 .. S-1-p it pairs with in one
// MMA per 256 columns, whose output columns are exactly levels p .. S-1.
#include <cuda.h>

#include <algorithm>

#include "mp_device.cuh"

namespace mp {

namespace {

constexpr int OZ_S_MAX_ORDER = 8;          // digits per operand (the kernels' S)
constexpr uint32_t OZ_WAIT_LIMIT = 1u << 22;

__device__ __forceinline__ uint32_t su32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mb_init(uint64_t* b, uint32_t c) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(c) : "memory");
}
__device__ __forceinline__ void mb_expect(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mb_try(uint64_t* b, uint32_t par) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(b)), "r"(par)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mb_wait(uint64_t* b, uint32_t par, int* err) {
  for (uint32_t i = 0; i < OZ_WAIT_LIMIT; ++i)
    if (mb_try(b, par)) return true;
  if (err) atomicExch(err, 1);
  return false;
}
__device__ __forceinline__ void tma2d(void* dst, const CUtensorMap* m, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(su32(bar))
      : "memory");
}
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// kind::f16, D = FP32, A = B = BF16, K-major, M = 128, N = n (a multiple of
// 16, at most 256)
__device__ __forceinline__ uint32_t oz_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc,
                                         uint32_t idesc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   su32(bar))
               : "memory");
}
__device__ __forceinline__ void ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Smallest power of two >= x (1 for x = 0).
__device__ __forceinline__ double pow2_above_d(double x) {
  if (!(x > 0.0)) return 1.0;
  int e;
  double m = frexp(x, &e);
  return m == 0.5 ? ldexp(1.0, e - 1) : ldexp(1.0, e);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const uint32_t a = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
  const uint32_t c = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
  return a | (c << 16);
}

// Rows of A (tile in any storage format; values exact in FP32) into S BF16
// digit tiles and the row bounds sigma.  One warp per row, four consecutive
// entries per lane (8-byte stores of four digits).
template <int S>
__global__ void __launch_bounds__(256) k_oz_split_rows(Arena A, const ItemOzA* __restrict__ items) {
  const ItemOzA it = items[blockIdx.x];
  const int b = A.b, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int row = blockIdx.y * 8 + warp;
  const TileRef ref = A.tiles[it.tile];
  const char* src = tile_bytes(A, it.tile);
  const float sc = (float)A.scale[it.tile];
  uint2* dst[S];
#pragma unroll
  for (int p = 0; p < S; ++p)
    dst[p] = reinterpret_cast<uint2*>(tile_ptr<__nv_bfloat16>(A, it.slices[p]) + (int64_t)row * b);
  const int64_t r0 = (int64_t)row * b;
  float mx = 0.f;
  for (int k = lane * 4; k < b; k += 128)
#pragma unroll
    for (int e = 0; e < 4; ++e) mx = fmaxf(mx, fabsf(load_f32(src, ref.dt, r0 + k + e) * sc));
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  // sigma = 2^es >= mx; a row whose largest entry is below 2^-126 (an
  // FP32 subnormal, far from the diagonal of a long-range field) has an
  // inverse bound beyond the float range, so it is scaled by the exponent
  // (exact both ways)
  int es = 0;
  if (mx > 0.f) {
    const float m = frexpf(mx, &es);          // mx = m 2^es, m in [0.5, 1)
    if (m == 0.5f) es -= 1;
  }
  const float sig = ldexpf(1.f, es);
  if (lane == 0) it.sigma[row] = sig;
  const bool wide = es < -126;
  const float inv = wide ? 0.f : ldexpf(1.f, -es);
  for (int k = lane * 4; k < b; k += 128) {
    float v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float x = load_f32(src, ref.dt, r0 + k + e) * sc;
      v[e] = wide ? ldexpf(x, -es) : x * inv;
    }
#pragma unroll
    for (int p = 0; p < S; ++p) {
      float d[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float t = v[e] * 64.f;
        d[e] = rintf(t);
        v[e] = t - d[e];                      // exact
      }
      dst[p][k / 4] = make_uint2(pack_bf16x2(d[0], d[1]), pack_bf16x2(d[2], d[3]));
    }
  }
}

// Columns of W (FP64 tile, row-major) into S BF16 digit tiles of W^T (the
// MMA's K-major B operand: row n of a digit tile is column n of W) and the
// column bounds tau.  One CTA: 32 columns x 64 rows; the column bound is
// taken over all b rows by every CTA of the column block (same value).
// The digits of v = W / tau come from the integer N = rint(v 2^(6S)) (round
// half to even): its balanced base-64 digits, least significant first, in
// [-32, 31], the leading one in [-64, 64].  They represent exactly the value
// that S successive steps d = rint(64 r), r = 64 r - d represent (both are
// the nearest multiple of 2^(-6S), ties to even), with integer arithmetic in
// place of 4 FP64 operations per digit.
template <int S>
__global__ void __launch_bounds__(256) k_oz_split_cols(Arena A, const ItemOzW* __restrict__ items) {
  static_assert(S <= 8, "N = v 2^(6S) must fit in 63 bits");
  __shared__ double tr[32][65];
  __shared__ unsigned long long cmax[8][32];
  __shared__ double cscale[32];
  const ItemOzW it = items[blockIdx.x];
  const int b = A.b, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n0 = blockIdx.y * 32, k0 = blockIdx.z * 64;
  const double* W = tile_ptr<double>(A, it.wtile);
  // largest |W| of the column: the bit patterns of magnitudes order like the
  // values (finite doubles), so an integer maximum does
  unsigned long long mx = 0;
  for (int k = warp; k < b; k += 8)
    mx = max(mx, (unsigned long long)__double_as_longlong(W[(int64_t)k * b + n0 + lane]) & 0x7fffffffffffffffull);
  cmax[warp][lane] = mx;
  __syncthreads();
  if (warp == 0) {
    for (int w = 1; w < 8; ++w) mx = max(mx, cmax[w][lane]);
    const double t = pow2_above_d(__longlong_as_double((long long)mx));
    if (blockIdx.z == 0) it.tau[n0 + lane] = (float)t;
    cscale[lane] = ldexp(1.0, 6 * S) / t;     // exact: powers of two
  }
  __syncthreads();
  // tr[n][k] = W[k0 + k][n0 + n] 2^(6S) / tau_n
  for (int e = threadIdx.x; e < 64 * 32; e += blockDim.x) {
    const int k = e / 32, n = e % 32;
    tr[n][k] = W[(int64_t)(k0 + k) * b + n0 + n] * cscale[n];
  }
  __syncthreads();
  // thread: row n = e / 16 of W^T, four consecutive k (8-byte stores)
  for (int e = threadIdx.x; e < 32 * 16; e += blockDim.x) {
    const int n = e / 16, kq = (e % 16) * 4;
    int dg[S][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      long long m = __double2ll_rn(tr[n][kq + j]);
#pragma unroll
      for (int q = S - 1; q > 0; --q) {
        const long long d = ((m + 32) & 63) - 32;
        dg[q][j] = (int)d;
        m = (m - d) >> 6;                     // exact: m - d is a multiple of 64
      }
      dg[0][j] = (int)m;
    }
#pragma unroll
    for (int q = 0; q < S; ++q) {
      uint2* dst = reinterpret_cast<uint2*>(tile_ptr<__nv_bfloat16>(A, it.slices[q]) +
                                            (int64_t)(n0 + n) * b + k0 + kq);
      *dst = make_uint2(pack_bf16x2((float)dg[q][0], (float)dg[q][1]),
                        pack_bf16x2((float)dg[q][2], (float)dg[q][3]));
    }
  }
}

constexpr int OZ_ACH = 128 * 128;          // A digit chunk: 128 rows x 128 bytes

// Order in which a K chunk's A digits are consumed when a unit uses s
// digits: digit p pairs with the s - p digits of W, so large and small
// amounts of MMA work alternate (0, s-1, 1, s-2, ...) and the ring never
// waits on several short chunks in a row.  Digit 0 comes first: it opens
// every level's accumulator.
__device__ __forceinline__ int oz_digit_order(int pi, int s) {
  return (pi & 1) ? s - 1 - (pi >> 1) : (pi >> 1);
}
constexpr int OZ_ASTG = 3;                 // A ring slots
constexpr int OZ_BSTG = 2;                 // W ring slots (S chunks each)
constexpr int OZ_STAGE = 32 * 33 * 8;      // epilogue staging per warp (32 x 33 float2 / double)

// Persistent: a work unit is (tile z, 128-row block y, BN-column block x),
// x fastest, so that the CTAs working on one row strip of A's digits run
// side by side; CTA i takes units i, i + gridDim.x, ...  Warp 0 (lane 0)
// streams the K chunks of W's and A's digits through two rings that run on
// across units, warp 1 (lane 0) issues the MMAs of a unit once the epilogue
// has read the previous unit's levels out of tensor memory, and warps 2-5
// (lane quarter warp % 4) read the levels into float-float registers, hand
// tensor memory back, then round and store, so one unit's stores overlap
// the next unit's MMAs.  Barriers: afull/aempty, bfull/bempty per ring slot,
// accf (a unit's MMAs complete), tfree (levels read, 4 arrivals), fin.
// Every wait is bounded (on expiry: error word, the roles stop; copies in
// flight land and issued MMAs complete before tensor memory is freed).
template <int S, int BN>
__global__ void __launch_bounds__(192, 1)
    k_oz_gemm(Arena A, const ItemOz* __restrict__ items, int count,
              const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB) {
  static_assert(S * BN <= 512 && (S * BN) % 32 == 0, "levels exceed tensor memory");
  constexpr int BCH = BN * 128;            // W digit chunk: BN rows x 128 bytes
  constexpr uint32_t TCOLS = S * BN;       // tensor-memory columns (a power of two)
  static_assert(S <= OZ_S_MAX_ORDER, "at most 8 digits per operand");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* bring = smem;                                   // OZ_BSTG x S x BCH
  uint8_t* aring = bring + OZ_BSTG * S * BCH;           // OZ_ASTG x OZ_ACH
  uint8_t* stage = aring + OZ_ASTG * OZ_ACH;               // 4 x OZ_STAGE
  uint64_t* afull = reinterpret_cast<uint64_t*>(stage + 4 * OZ_STAGE);
  uint64_t* aempty = afull + OZ_ASTG;
  uint64_t* bfull = aempty + OZ_ASTG;
  uint64_t* bempty = bfull + OZ_BSTG;
  uint64_t* accf = bempty + OZ_BSTG;
  uint64_t* tfree = accf + 1;
  uint64_t* fin = tfree + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(fin + 1);
  const int b = A.b;
  const int nnb = b / BN, nmb = b / 128;
  const int units = count * nnb * nmb;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_ASTG; ++s) { mb_init(&afull[s], 1); mb_init(&aempty[s], 1); }
    for (int s = 0; s < OZ_BSTG; ++s) { mb_init(&bfull[s], 1); mb_init(&bempty[s], 1); }
    mb_init(accf, 1);
    mb_init(tfree, 4);
    mb_init(fin, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapB)) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "r"(TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const int KT = b / 64;
  if (warp == 0) {
    if (lane == 0) {
      // producer: per K chunk, the S chunks of W^T, then the S chunks of A
      bool ok = true;
      int na = 0, nb = 0;
      for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
        const ItemOz& it = items[u / (nnb * nmb)];
        const int m0 = ((u / nnb) % nmb) * 128, n0 = (u % nnb) * BN;
        const int su = it.s;                // digits this unit uses (<= S)
        int32_t aidx[S], widx[S];
#pragma unroll
        for (int p = 0; p < S; ++p) { aidx[p] = A.tiles[it.a[p]].idx; widx[p] = A.tiles[it.w[p]].idx; }
        for (int kt = 0; kt < KT && ok; ++kt) {
          const int sb = nb % OZ_BSTG;
          if (nb >= OZ_BSTG && !(ok = mb_wait(&bempty[sb], ((nb / OZ_BSTG) - 1) & 1, A.err))) break;
          mb_expect(&bfull[sb], su * BCH);
#pragma unroll
          for (int q = 0; q < S; ++q)
            if (q < su) tma2d(bring + (sb * S + q) * BCH, &mapB, kt * 64, widx[q] * b + n0, &bfull[sb]);
          ++nb;
#pragma unroll 1
          for (int pi = 0; pi < su; ++pi) {
            const int p = oz_digit_order(pi, su);
            const int sa = na % OZ_ASTG;
            if (na >= OZ_ASTG && !(ok = mb_wait(&aempty[sa], ((na / OZ_ASTG) - 1) & 1, A.err))) break;
            mb_expect(&afull[sa], OZ_ACH);
            tma2d(aring + sa * OZ_ACH, &mapA, kt * 64, aidx[p] * b + m0, &afull[sa]);
            ++na;
          }
        }
      }
      if (!ok) {
        // let the copies in flight land before the CTA exits
        for (int i = (na > OZ_ASTG ? na - OZ_ASTG : 0); i < na; ++i)
          mb_wait(&afull[i % OZ_ASTG], (i / OZ_ASTG) & 1, nullptr);
        for (int k = (nb > OZ_BSTG ? nb - OZ_BSTG : 0); k < nb; ++k)
          mb_wait(&bfull[k % OZ_BSTG], (k / OZ_BSTG) & 1, nullptr);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      int na = 0, nb = 0, t = 0;
      for (int u = blockIdx.x; u < units && ok; u += gridDim.x, ++t) {
        // the epilogue has read the previous unit's levels
        if (t >= 1 && !(ok = mb_wait(tfree, (t - 1) & 1, A.err))) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int su = items[u / (nnb * nmb)].s;
        for (int kt = 0; kt < KT && ok; ++kt) {
          const int sb = nb % OZ_BSTG;
          if (!(ok = mb_wait(&bfull[sb], (nb / OZ_BSTG) & 1, A.err))) break;
          const uint32_t b0 = su32(bring + sb * S * BCH);
#pragma unroll 1
          for (int pi = 0; pi < su; ++pi) {
            const int p = oz_digit_order(pi, su);
            const int sa = na % OZ_ASTG;
            if (!(ok = mb_wait(&afull[sa], (na / OZ_ASTG) & 1, A.err))) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = su32(aring + sa * OZ_ACH);
            // A_p against W digits q = 0 .. S-1-p in one product per 256
            // columns: the digits lie one after another in the ring (BN
            // rows each) and level l sits at tensor-memory column l * BN,
            // so the product of A_p with digits q0 .. q0+nq-1 lands on levels
            // p+q0 .. p+q0+nq-1 (A_p is read once per 256 columns)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint32_t acc = !(kt == 0 && p == 0 && kk == 0);   // level p+q first touched at p = 0
#pragma unroll 1
              for (int q0 = 0; q0 < su - p; q0 += 256 / BN) {
                const int nq = min(256 / BN, su - p - q0);
                mma_bf16(tmem + (uint32_t)(p + q0) * BN, sdesc(a0 + kk * 32),
                         sdesc(b0 + q0 * BCH + kk * 32), acc, oz_idesc(nq * BN));
              }
            }
            commit(&aempty[sa]);
            ++na;
          }
          if (!ok) break;
          commit(&bempty[sb]);
          ++nb;
        }
        if (!ok) break;
        commit(accf);
      }
      // every MMA issued has completed before tensor memory is freed
      commit(fin);
      mb_wait(fin, 0, A.err);
    }
  } else {
    // epilogue warps 2-5: lane quarter qr = warp % 4 of the accumulator
    const int qr = warp & 3;
    double (*Sx)[33] = reinterpret_cast<double (*)[33]>(stage + (warp - 2) * OZ_STAGE);
    float2 (*Sf)[33] = reinterpret_cast<float2 (*)[33]>(stage + (warp - 2) * OZ_STAGE);
    int t = 0;
    for (int u = blockIdx.x; u < units; u += gridDim.x, ++t) {
      const ItemOz it = items[u / (nnb * nmb)];
      const int m0 = ((u / nnb) % nmb) * 128, n0 = (u % nnb) * BN;
      if (!mb_wait(accf, t & 1, A.err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // levels from the smallest (l = s-1) to the largest, in float-float
      float hi[BN], lo[BN];
#pragma unroll
      for (int j = 0; j < BN; ++j) { hi[j] = 0.f; lo[j] = 0.f; }
#pragma unroll 1
      for (int l = it.s - 1; l >= 0; --l) {
        const float scl = ldexpf(1.f, -6 * (l + 2));
#pragma unroll
        for (int h = 0; h < BN / 32; ++h) {
          float v[32];
          ld32(tmem + ((uint32_t)(qr * 32) << 16) + (uint32_t)(l * BN + h * 32), v);
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float x = v[j] * scl;           // exact: the level sum is an integer < 2^24
            const float s = hi[h * 32 + j] + x;   // two-sum
            const float bb = s - hi[h * 32 + j];
            const float e = (hi[h * 32 + j] - (s - bb)) + (x - bb);
            hi[h * 32 + j] = s;
            lo[h * 32 + j] += e;
          }
        }
      }
      // tensor memory read: the next unit's MMAs may start
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(tfree)) : "memory");
      const int row = m0 + qr * 32 + lane;
      const float sg = it.sigma[row];
      float mx = 0.f;
      // fused rounding (no E4M3 target or shadow): the tile, its shadow
      // copies and its TF32 split come straight from the float-float value
      int tdt = -1, sdt[MAX_SHADOW];
      char* tdst = nullptr;
      char* sdst[MAX_SHADOW];
      float* thi = nullptr;
      float* tlo = nullptr;
      if (it.fuse) {
        tdt = A.tiles[it.tile].dt;
        tdst = tile_bytes(A, it.tile);
#pragma unroll
        for (int q = 0; q < MAX_SHADOW; ++q) {
          sdt[q] = it.shadow[q] >= 0 ? A.tiles[it.shadow[q]].dt : -1;
          sdst[q] = it.shadow[q] >= 0 ? tile_bytes(A, it.shadow[q]) : nullptr;
        }
        if (it.hi >= 0) { thi = tile_ptr<float>(A, it.hi); tlo = tile_ptr<float>(A, it.lo); }
      }
#pragma unroll
      for (int h = 0; h < BN / 32; ++h) {
        if (it.fuse) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float st = sg * it.tau[n0 + h * 32 + j];   // power of two: scaling is exact
            Sf[lane][j] = make_float2(hi[h * 32 + j] * st, lo[h * 32 + j] * st);
          }
          __syncwarp();
#pragma unroll 4
          for (int rr = 0; rr < 32; ++rr) {
            const float2 p = Sf[rr][lane];
            const int64_t o = (int64_t)(m0 + qr * 32 + rr) * b + n0 + h * 32 + lane;
            float stored;
            if (tdt == F32) {
              stored = __fadd_rn(p.x, p.y);              // the float-float value rounded once
              reinterpret_cast<float*>(tdst)[o] = stored;
            } else {
              store_round(tdst, tdt, o, (double)p.x + (double)p.y);
              stored = load_f32(tdst, tdt, o);
            }
#pragma unroll
            for (int q = 0; q < MAX_SHADOW; ++q)
              if (sdst[q]) store_round_f32(sdst[q], sdt[q], o, stored);
            if (thi) {
              uint32_t hb;
              asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(stored));
              thi[o] = __uint_as_float(hb);
              tlo[o] = stored - __uint_as_float(hb);
            }
          }
          __syncwarp();
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float st = sg * it.tau[n0 + h * 32 + j];
            Sx[lane][j] = (double)(hi[h * 32 + j] * st) + (double)(lo[h * 32 + j] * st);
          }
          __syncwarp();
#pragma unroll 4
          for (int rr = 0; rr < 32; ++rr) {
            const double xv = Sx[rr][lane];
            it.x[(int64_t)(m0 + qr * 32 + rr) * b + n0 + h * 32 + lane] = xv;
            mx = fmaxf(mx, fabsf((float)xv));
          }
          __syncwarp();
        }
      }
      if (!it.fuse) {
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) atomic_max_pos(&A.amax[it.amax], (double)mx);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
}

template <int S, int BN>
constexpr size_t oz_smem() {
  return (size_t)OZ_BSTG * S * BN * 128 + (size_t)OZ_ASTG * OZ_ACH + 4 * (size_t)OZ_STAGE +
         8 * (2 * OZ_ASTG + 2 * OZ_BSTG + 3) + 16 + 1024;
}

}  // namespace

constexpr int OZ_S = 8;

int oz_slices(int) { return OZ_S; }

void launch_oz_split_rows(const Arena& A, const ItemOzA* items, int count, cudaStream_t s) {
  if (count <= 0) return;
  k_oz_split_rows<OZ_S><<<dim3(count, A.b / 8), 256, 0, s>>>(A, items);
}

void launch_oz_split_cols(const Arena& A, const ItemOzW* items, int count, cudaStream_t s) {
  if (count <= 0) return;
  k_oz_split_cols<OZ_S><<<dim3(count, A.b / 32, A.b / 64), 256, 0, s>>>(A, items);
}

template <int BN>
void oz_gemm_launch(const Arena& A, const ItemOz* items, int count, const CUtensorMap& mapA,
                    const CUtensorMap& mapB, cudaStream_t s) {
  constexpr size_t smem = oz_smem<OZ_S, BN>();
  static bool attr = false;
  static int sms = 0;
  if (!attr) {
    cudaFuncSetAttribute(k_oz_gemm<OZ_S, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    attr = true;
  }
  const int64_t units = (int64_t)count * (A.b / BN) * (A.b / 128);
  const int grid = (int)std::min<int64_t>(units, sms);
  k_oz_gemm<OZ_S, BN><<<grid, 192, smem, s>>>(A, items, count, mapA, mapB);
}

// One tile (the critical chain's first panel tile): 128 x 32 units, twice as
// many CTAs as 128 x 64 units; several tiles: 128 x 64 units (fewer, wider
// MMAs per output column).
void launch_oz_gemm(const Arena& A, const ItemOz* items, int count, const CUtensorMap& mapA,
                    const CUtensorMap& mapB64, const CUtensorMap& mapB32, cudaStream_t s) {
  if (count <= 0) return;
  if (count == 1) oz_gemm_launch<32>(A, items, count, mapA, mapB32, s);
  else oz_gemm_launch<64>(A, items, count, mapA, mapB64, s);
}

}  // namespace mp
