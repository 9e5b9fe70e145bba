// Trailing updates on the 5th-generation tensor cores (tcgen05), for the
// products whose precision (min(p(target), max(p(A), p(B))), Sec. 4.3's
// promotion rule capped by the target tile) is below FP64:
//   BF16 / FP16  kind::f16     A, B in the 16-bit format, FP32 accumulate
//   E4M3         kind::f8f6f4  scaled codes; FP32 sum times s_a s_b
//   FP32         kind::tf32    three products of hi/lo splits,
//                              A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T,
//                              where hi = A rounded to TF32 and lo = A - hi,
//                              in two MMAs per K step (A_hi against
//                              [B_hi | B_lo] with N = 256, A_lo against B_hi)
//                              into a 256-column accumulator whose halves
//                              the epilogue adds
// A work unit is a 128 x 128 sub-tile of a target with the full contraction
// K = b; one persistent CTA per SM runs units back to back.  Warp 0 (one
// lane) streams 128-byte-wide K slices of the operand tiles into shared
// memory with TMA (128-byte swizzle, one tensor map per format pool; no
// multicast), warp 1 (one lane) issues the MMAs into one of two FP32
// accumulators in tensor memory, and warps 2-5 read the other one back
// (each its lane quarter) and apply the update to the target tile in global
// memory:
//   FP64 target (SYRK into the diagonal)  C -= acc            (float64)
//   FP32 target                           C = C - acc         (one FP32 sub,
//                                         correctly rounded)
//   16-bit target                         C = round(C - acc)  (FP32 sub)
//   E4M3 target                           FP32 scratch + amax (rounded by
//                                         k_fp8_round with the new scale)
// Every mbarrier wait is bounded: when it runs out the CTA records the
// failure in the arena's error word, lets the copies and MMAs it issued
// complete, frees its tensor memory and returns.
#include <cuda.h>

#include <algorithm>

#include "mp_device.cuh"

namespace mp {

namespace {

constexpr int TC_BM = 128, TC_BN = 128;
constexpr int TC_BUF = 128 * 128;          // one 128-row x 128-byte operand slice
constexpr uint32_t TC_WAIT_LIMIT = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait; on time-out records the failure and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
  for (uint32_t i = 0; i < TC_WAIT_LIMIT; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  if (err) atomicExch(err, 1);
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand slice, 128-byte swizzle,
// rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);          // start address
  d |= (uint64_t)1 << 16;                           // leading byte offset (unused: 16 B)
  d |= (uint64_t)(1024 >> 4) << 32;                 // stride byte offset
  d |= (uint64_t)1 << 46;                           // descriptor version
  d |= (uint64_t)2 << 61;                           // 128-byte swizzle
  return d;
}

// Instruction descriptor: D = FP32, A/B format code `fmt`, both K-major,
// M = 128, N = n.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt, int n = TC_BN) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(TC_BM >> 4) << 24);
}

template <int KIND, int N = TC_BN>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  constexpr uint32_t idesc = instr_desc(KIND == 0 ? 1u : KIND == 1 ? 0u : KIND == 2 ? 0u : 2u, N);
  if constexpr (KIND == 0 || KIND == 1) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else if constexpr (KIND == 2) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
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

// KIND: 0 BF16, 1 FP16, 2 E4M3, 3 FP32 as three TF32 products.  The FP32
// kind's accumulator is 256 columns wide: per K step one MMA of A_hi
// against [B_hi | B_lo] (N = 256: hi*hi into the first 128 columns, hi*lo
// into the second) and one of A_lo against B_hi into the second; the
// epilogue adds the two halves.
// Persistent variant: one CTA per SM walks the work units (target tile,
// 128 x 128 sub-block; the sub-blocks of one target next to each other) in
// a fixed round-robin order.  Warp 0 streams K slices through a STAGES-deep
// ring that runs on across units, warp 1 issues the MMAs into one of two
// 128-column tensor-memory accumulators, and warps 2-5 drain the other one
// (each its lane quarter) and update the target, so a unit's epilogue
// overlaps the next unit's MMAs.  Barriers: full/empty per ring slot,
// accf (accumulator complete) and acce (accumulator read back, 4 arrivals)
// per accumulator.  Every wait is bounded (on expiry: error word, then the
// roles stop; issued MMAs are waited for before tensor memory is freed).
template <int KIND, int STAGES, int MINB>
__global__ void __launch_bounds__(192, MINB)
    k_update_tc_p(Arena A, const ItemTC* __restrict__ items, const __grid_constant__ CUtensorMap tmap,
                  int count) {
  extern __shared__ uint8_t smem_raw[];
  constexpr int NA = KIND == 3 ? 2 : 1;
  constexpr int STAGE_BYTES = 2 * NA * TC_BUF;
  constexpr int KCH = KIND == 2 ? 128 : KIND == 3 ? 32 : 64;
  constexpr int ACC_COLS = KIND == 3 ? 2 * TC_BN : TC_BN;   // tensor-memory columns per accumulator
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* stage_c = reinterpret_cast<float*>(smem + STAGES * STAGE_BYTES);     // 4 x [32][33]
  uint64_t* full = reinterpret_cast<uint64_t*>(stage_c + 4 * 32 * 33);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;        // [2]
  uint64_t* acce = accf + 2;              // [2]
  uint64_t* fin = acce + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(fin + 1);
  const int b = A.b, nsub = b / TC_BM, nsub2 = nsub * nsub;
  const int KT = b / KCH;
  const int units = count * nsub2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int q = 0; q < STAGES; ++q) { mbar_init(&full[q], 1); mbar_init(&empty[q], 1); }
    for (int q = 0; q < 2; ++q) { mbar_init(&accf[q], 1); mbar_init(&acce[q], 4); }
    mbar_init(fin, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(2 * ACC_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  // unit u -> (item, rb, cb); SYRK units strictly above the diagonal are skipped
  auto unit = [&](int u, ItemTC& it, int& rb, int& cb) {
    it = items[u / nsub2];
    const int sb = u % nsub2;
    rb = sb / nsub;
    cb = sb % nsub;
    return !(it.syrk && cb > rb);
  };
  if (warp == 0) {
    if (lane == 0) {
      int g = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
        ItemTC it;
        int rb, cb;
        if (!unit(u, it, rb, cb)) continue;
        // a unit contracts over it.kspan consecutive operand tiles (1 in
        // the factorisation; the standalone product spans several)
        const int span = it.kspan > 1 ? it.kspan : 1;
        for (int kt = 0; kt < KT * span; ++kt, ++g) {
          const int tk = kt / KT, kx = (kt % KT) * KCH;
          const int ya0 = A.tiles[it.a + tk].idx * b + rb * TC_BM;
          const int yb0 = A.tiles[it.b + tk].idx * b + cb * TC_BN;
          const int q = g % STAGES;
          if (g >= STAGES && !(ok = mbar_wait(&empty[q], ((g / STAGES) - 1) & 1, A.err))) break;
          uint8_t* st = smem + q * STAGE_BYTES;
          mbar_expect_tx(&full[q], STAGE_BYTES);
          tma_load_2d(st, &tmap, kx, ya0, &full[q]);
          if (NA == 2) tma_load_2d(st + TC_BUF, &tmap, kx, A.tiles[it.a2 + tk].idx * b + rb * TC_BM, &full[q]);
          tma_load_2d(st + NA * TC_BUF, &tmap, kx, yb0, &full[q]);
          if (NA == 2) tma_load_2d(st + (NA + 1) * TC_BUF, &tmap, kx, A.tiles[it.b2 + tk].idx * b + cb * TC_BN, &full[q]);
        }
      }
      if (!ok)   // let the copies in flight land before the CTA's memory goes away
        for (int h = (g > STAGES ? g - STAGES : 0); h < g; ++h)
          mbar_wait(&full[h % STAGES], (h / STAGES) & 1, nullptr);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int g = 0, t = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
        ItemTC it;
        int rb, cb;
        if (!unit(u, it, rb, cb)) continue;
        const int buf = t & 1;
        if (t >= 2 && !(ok = mbar_wait(&acce[buf], ((t / 2) - 1) & 1, A.err))) break;
        tc_fence_after();
        const uint32_t acc_t = tmem + (uint32_t)(buf * ACC_COLS);
        const int span = it.kspan > 1 ? it.kspan : 1;
        for (int kt = 0; kt < KT * span; ++kt, ++g) {
          const int q = g % STAGES;
          if (!(ok = mbar_wait(&full[q], (g / STAGES) & 1, A.err))) break;
          tc_fence_after();
          const uint32_t a0 = smem_u32(smem + q * STAGE_BYTES);
          const uint32_t a1 = a0 + TC_BUF;
          const uint32_t b0 = a0 + NA * TC_BUF;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint32_t off = kk * 32;
            const uint32_t acc = (kt | kk) != 0;
            if constexpr (KIND == 3) {
              // B_hi and B_lo are adjacent in the slot: one 256-row operand
              mma<KIND, 2 * TC_BN>(acc_t, smem_desc(a0 + off), smem_desc(b0 + off), acc);
              mma<KIND>(acc_t + TC_BN, smem_desc(a1 + off), smem_desc(b0 + off), 1);
            } else {
              mma<KIND>(acc_t, smem_desc(a0 + off), smem_desc(b0 + off), acc);
            }
          }
          mma_commit(&empty[q]);
        }
        if (!ok) break;
        mma_commit(&accf[buf]);
        ++t;
      }
      // every MMA issued has completed before tensor memory is freed
      mma_commit(fin);
      mbar_wait(fin, 0, A.err);
    }
  } else {
    // epilogue warps 2-5: lane quarter qr = warp % 4 of the accumulator
    const int qr = warp & 3;
    float (*S)[33] = reinterpret_cast<float (*)[33]>(stage_c + (warp - 2) * 32 * 33);
    int t = 0;
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
      ItemTC it;
      int rb, cb;
      if (!unit(u, it, rb, cb)) continue;
      const int buf = t & 1;
      {
        // pull this lane quarter's 32 target rows into L2 while the unit's
        // MMAs run (the read-modify-write below then meets no DRAM latency)
        const TileRef rp = A.tiles[it.c];
        const char* base = tile_bytes(A, it.c);
        const int es = (int)esize(rp.dt);
        const int lpr = TC_BN * es / 128;              // 128-byte lines per row
        const int64_t r0 = (int64_t)rb * TC_BM + qr * 32;
        for (int e = lane; e < 32 * lpr; e += 32) {
          const char* ptr = base + ((r0 + e / lpr) * b + cb * TC_BN) * es + (e % lpr) * 128;
          asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
        }
      }
      if (!mbar_wait(&accf[buf], (t / 2) & 1, A.err)) break;
      tc_fence_after();
      const TileRef rc = A.tiles[it.c];
      char* pc = tile_bytes(A, it.c);
      const float sab = (float)(A.scale[it.a] * A.scale[it.b]);
      const double sc = A.scale[it.c];
      float mx = 0.f;
#pragma unroll 1
      for (int ch = 0; ch < TC_BN / 32; ++ch) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(qr * 32) << 16) + (uint32_t)(buf * ACC_COLS + ch * 32), v);
        if constexpr (KIND == 3) {   // + the hi*lo + lo*hi half
          float w[32];
          tmem_ld32(tmem + ((uint32_t)(qr * 32) << 16) + (uint32_t)(buf * ACC_COLS + TC_BN + ch * 32), w);
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] += w[j];
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) S[lane][j] = v[j] * sab;
        __syncwarp();
        const int col = cb * TC_BN + ch * 32 + lane;
        const int row0 = rb * TC_BM + qr * 32;
        const int rlo = it.syrk ? max(0, cb * TC_BN + ch * 32 - row0) : 0;
        const int64_t o0 = (int64_t)row0 * b + col;
        if (rc.dt == F32) {
          float* c = reinterpret_cast<float*>(pc) + o0;
          float cur[32];
#pragma unroll
          for (int rr = 0; rr < 32; ++rr) cur[rr] = rr >= rlo ? c[(int64_t)rr * b] : 0.f;
#pragma unroll
          for (int rr = 0; rr < 32; ++rr)    // one correctly rounded FP32 subtraction
            if (rr >= rlo) c[(int64_t)rr * b] = __fsub_rn(cur[rr], S[rr][lane]);
        } else if (rc.dt == F64) {
          double* c = reinterpret_cast<double*>(pc) + o0;
          double cur[32];
#pragma unroll
          for (int rr = 0; rr < 32; ++rr) cur[rr] = rr >= rlo ? c[(int64_t)rr * b] : 0.0;
#pragma unroll
          for (int rr = 0; rr < 32; ++rr)
            if (rr >= rlo) c[(int64_t)rr * b] = cur[rr] - (double)S[rr][lane];
        } else {
          float cur[32];
#pragma unroll
          for (int rr = 0; rr < 32; ++rr) cur[rr] = rr >= rlo ? load_f32(pc, rc.dt, o0 + (int64_t)rr * b) : 0.f;
          if (rc.dt == E4M3) {
            const float fs = (float)sc;
#pragma unroll
            for (int rr = 0; rr < 32; ++rr)
              if (rr >= rlo) {
                const float w = cur[rr] * fs - S[rr][lane];
                it.v[o0 + (int64_t)rr * b] = w;
                mx = fmaxf(mx, fabsf(w));
              }
          } else {
#pragma unroll
            for (int rr = 0; rr < 32; ++rr)
              if (rr >= rlo) store_round_f32(pc, rc.dt, o0 + (int64_t)rr * b, cur[rr] - S[rr][lane]);
          }
        }
        __syncwarp();
      }
      // this warp's quarter of the accumulator is read: hand it back
      tc_fence_before();
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[buf])) : "memory");
      ++t;
      if (rc.dt == E4M3) {
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) atomic_max_pos(&A.amax[it.vslot], (double)mx);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * ACC_COLS)
                 : "memory");
  }
}

template <int KIND, int STAGES>
constexpr size_t tc_smem_p() {
  return (size_t)STAGES * 2 * (KIND == 3 ? 2 : 1) * TC_BUF + 4 * 32 * 33 * sizeof(float) +
         8 * (2 * STAGES + 5) + 16 + 1024;
}

// FP32 kind: three MMAs per K step keep the tensor cores busy, one CTA per
// SM with a 3-slot ring; 16- and 8-bit kinds are epilogue-bound, two CTAs
// per SM with a 2-slot ring each.
template <int KIND, int STAGES, int MINB>
void launch_tc(const Arena& A, const ItemTC* items, int count, const CUtensorMap& map,
               cudaStream_t s) {
  static int sms = 0;
  constexpr size_t smem = tc_smem_p<KIND, STAGES>();
  if (!sms) {
    cudaFuncSetAttribute(k_update_tc_p<KIND, STAGES, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const int nsub = A.b / TC_BM;
  const int64_t units = (int64_t)count * nsub * nsub;
  const int grid = (int)std::min<int64_t>(units, (int64_t)MINB * sms);
  k_update_tc_p<KIND, STAGES, MINB><<<grid, 192, smem, s>>>(A, items, map, count);
}

}  // namespace

// kind: BF16, F16, E4M3 or F32 (three TF32 products); map: the tensor map of
// the operand pool (box 128 bytes x 128 rows, 128-byte swizzle).
// ring4: the 16- and 8-bit kinds with a 4-slot ring and one CTA per SM
// instead of a 2-slot ring and two CTAs per SM (a schedule choice of the
// autotuner).
void launch_update_tc(const Arena& A, int kind, const ItemTC* items, int count,
                      const CUtensorMap& map, cudaStream_t s, bool ring4) {
  if (count <= 0) return;
  switch (kind) {
    case BF16: ring4 ? launch_tc<0, 4, 1>(A, items, count, map, s) : launch_tc<0, 2, 2>(A, items, count, map, s); break;
    case F16: ring4 ? launch_tc<1, 4, 1>(A, items, count, map, s) : launch_tc<1, 2, 2>(A, items, count, map, s); break;
    case E4M3: ring4 ? launch_tc<2, 4, 1>(A, items, count, map, s) : launch_tc<2, 2, 2>(A, items, count, map, s); break;
    default: launch_tc<3, 3, 1>(A, items, count, map, s); break;
  }
}

}  // namespace mp
