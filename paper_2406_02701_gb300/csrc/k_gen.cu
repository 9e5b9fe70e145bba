// Locations and covariance tiles.
//
// Morton order: 32-bit Z-curve keys of the 16-bit-quantised coordinates
// (x bits even, y bits odd), made unique by appending the point index, then
// sorted by a bitonic network (global passes for strides >= 1024, shared
// memory for the rest).
//
// Generation (the Matérn model of Sec. 6.2; half-integer nu by the closed
// forms, any other nu in (0, 16] from a Chebyshev table of x^nu K_nu(x)
// built on the host, see matern_nu_table): every entry of a lower tile is
// computed to float64 accuracy from the two locations and rounded once into
// the tile's format.  The coordinate differences and the squared distance
// are float64 (explicit _rn intrinsics, one fused multiply-add); for the
// closed forms the square root, e^{-x} and the polynomial then run in
// 64-bit fixed point on the integer pipe (mp_fixed.cuh), since GB300's FP64
// pipe is 1/64 of its FP32 rate; other nu, and the rare entries outside the
// fixed-point path's range, take float64 with Tang's table-driven e^{-x}.
// Off-diagonal FP32/16-bit tiles of a matrix without a float64 copy of Sigma
// are evaluated in float-float instead (below).  E4M3 tiles first get the
// tile's amax from a separate pass (`gen_amax`), then the power-of-two
// scale.  Rows/columns beyond n are identity padding.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "mp_device.cuh"
#include "mp_fixed.cuh"

namespace mp {

namespace {

// e^{-x} tables (set per device by init_gen_tables): [0, 64) 2^{j/64}
// rounded to double, [64, 128) the remainders 2^{j/64} - hi, [128] the head
// of ln2/64 with 37 significant bits, [129] ln2/64 - head, [130] 64/ln2.
constexpr int GEN_TAB = 131;
__constant__ double c_gen_tab[GEN_TAB];

// The same for float-float evaluation (set by init_gen_tables): [0, 64)
// 2^{j/64} rounded to float, [64, 128) the remainders rounded to float,
// [128] ln2/64 rounded to float, [129] the remainder, [130] 64/ln2, [131]
// 1/3 rounded to float, [132] the remainder.
constexpr int GEN_FTAB = 133;
__constant__ float c_gen_ftab[GEN_FTAB];

// 2^{-j/1024} 2^63 rounded, j in [0, 1024), for the fixed-point e^{-x}
// (set by init_gen_tables; copied into shared memory by each CTA)
constexpr int GEN_T2 = 1024;
__device__ uint64_t g_gen_t2[GEN_T2];

__device__ __forceinline__ uint32_t spread16(uint32_t v) {
  uint32_t k = 0;
  for (int bit = 0; bit < 16; ++bit) k |= ((v >> bit) & 1u) << (2 * bit);
  return k;
}

__global__ void k_morton_keys(const double* __restrict__ locs, int64_t n, int64_t n2,
                              unsigned long long* __restrict__ keys) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n2) return;
  if (i >= n) { keys[i] = ~0ull; return; }
  double qx = fmax(fmin(floor(__dmul_rn(locs[2 * i], 65536.0)), 65535.0), 0.0);
  double qy = fmax(fmin(floor(__dmul_rn(locs[2 * i + 1], 65536.0)), 65535.0), 0.0);
  uint32_t key = spread16((uint32_t)qx) | (spread16((uint32_t)qy) << 1);
  keys[i] = ((unsigned long long)key << 32) | (unsigned long long)i;
}

// One compare-exchange pass of the bitonic network with stride j >= 1024.
__global__ void k_bitonic_global(unsigned long long* keys, int64_t n2, int64_t j, int64_t k) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n2) return;
  int64_t l = i ^ j;
  if (l <= i) return;
  unsigned long long a = keys[i], b = keys[l];
  bool up = (i & k) == 0;
  if (up ? a > b : a < b) { keys[i] = b; keys[l] = a; }
}

// All passes of stage k with stride < 1024 (or the full sort of 1024-element
// blocks when k_hi = 0), inside one 1024-element block in shared memory.
__global__ void k_bitonic_local(unsigned long long* keys, int64_t n2, int64_t k_lo,
                                int64_t k_hi) {
  __shared__ unsigned long long s[1024];
  int64_t base = (int64_t)blockIdx.x * 1024;
  for (int t = threadIdx.x; t < 1024; t += blockDim.x) s[t] = keys[base + t];
  __syncthreads();
  for (int64_t k = k_lo; k <= k_hi; k <<= 1) {
    for (int64_t j = (k >> 1) < 512 ? (k >> 1) : 512; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < 1024; t += blockDim.x) {
        int l = t ^ (int)j;
        if (l > t) {
          unsigned long long a = s[t], b = s[l];
          bool up = ((base + t) & k) == 0;
          if (up ? a > b : a < b) { s[t] = b; s[l] = a; }
        }
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < 1024; t += blockDim.x) keys[base + t] = s[t];
}

__global__ void k_morton_gather(const unsigned long long* __restrict__ keys,
                                const double* __restrict__ in, int64_t n,
                                double* __restrict__ out, int64_t* __restrict__ perm) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t p = (int64_t)(keys[i] & 0xffffffffull);
  perm[i] = p;
  out[2 * i] = in[2 * p];
  out[2 * i + 1] = in[2 * p + 1];
}

// e^{-x} for x >= 0 by Tang's table-driven method (P. T. P. Tang,
// "Table-driven implementation of the exponential function in IEEE
// floating-point arithmetic", ACM TOMS 15, 1989) with a 64-entry table:
// -x = k ln2/64 + r with k = rint(-64 x / ln2) and |r| <= ln2/128 (k times
// the 37-bit head of ln2/64 is exact for |k| < 2^16, i.e. x <= 700);
// k = 64 m + j and e^{-x} = 2^m 2^{j/64} (1 + p), p = e^r - 1 from its
// Taylor polynomial of degree 5 (truncation below r^6/6! < 4e-17),
// 2^{j/64} = T_hi + T_lo, the sum T_hi + (T_lo + T_hi p) rounded once:
// within 0.8 ulp.  Beyond 700 (and for NaN) the library exp.
__device__ __forceinline__ double exp_neg(double x, const double* tab) {
  if (!(x <= 700.0)) return exp(-x);
  const double shifter = 6755399441055744.0;           // 1.5 * 2^52
  const double t = fma(-x, tab[130], shifter);          // low bits: k
  const int k = __double2loint(t);
  const double kd = t - shifter;
  const double r = fma(-kd, tab[129], fma(-kd, tab[128], -x));
  const double q = fma(r, fma(r, fma(r, 1.0 / 120.0, 1.0 / 24.0), 1.0 / 6.0), 0.5);
  const double p = fma(r * r, q, r);
  const int m = k >> 6, j = k & 63;
  const double th = tab[j];
  const double v = th + fma(th, p, tab[64 + j]);   // in [0.99, 2.02]
  // times 2^m (m >= -1010: the result stays normal) on the exponent field
  return __longlong_as_double(__double_as_longlong(v) + ((long long)m << 52));
}

// Matérn correlation for nu without a closed form, from the table of
// matern_nu_table: x = m 2^E (m in [1, 2)) lies in the half octave
// 2 (E - e0) + (m >= 1.5), whose Chebyshev series in u = 4 (m - 1.25) or
// 4 (m - 1.75) -- exact, the piece's centre and half-width being dyadic --
// is summed by Clenshaw's recurrence.  Returns g(x) for x < 1 and g(x) e^x
// for 1 <= x < 2^KNU_EMAX (the caller multiplies by e^{-x}); 1 below
// 2^e0, where g differs from 1 by less than 2^-54.
__device__ __forceinline__ double knu_table(const double* __restrict__ tab, int e0, double x) {
  const int hi = __double2hiint(x);
  const int E = ((hi >> 20) & 0x7ff) - 1023;
  if (E < e0) return 1.0;
  const double m = __hiloint2double((hi & 0x000fffff) | 0x3ff00000, __double2loint(x));
  const int upper = m >= 1.5;
  const double u = 4.0 * (m - (upper ? 1.75 : 1.25));
  const double* c = tab + (2 * (E - e0) + upper) * KNU_COEF;
  const double u2 = u + u;
  double b1 = 0.0, b2 = 0.0;
#pragma unroll
  for (int k = KNU_COEF - 1; k >= 1; --k) {
    const double t = fma(u2, b1, __ldg(c + k) - b2);
    b2 = b1;
    b1 = t;
  }
  return fma(u, b1, __ldg(c) - b2);
}

// Matérn covariance of two locations (closed forms, x = r / range):
// sigma^2 e^{-x} (nu = 1/2), sigma^2 (1 + x) e^{-x} (3/2),
// sigma^2 (1 + x + x^2/3) e^{-x} (5/2).
// r = s rsqrt(s) for s = dx^2 + dy^2 > 0 (one fused multiply-add; rsqrt
// within 1 ulp: r within 1.5 ulp); x is r times the rounded reciprocal of the range (GB300's FP64
// pipe makes a division cost about ten FP64 operations): |dx| <= 3 ulp(x),
// which exp(-x) carries as a relative error of at most 3 x 2^-53.
__device__ __forceinline__ double entry_f64(const ItemGen& it, double inv_range, const double* tab,
                                            double xi, double yi, double xj, double yj, int64_t gi,
                                            int64_t gj) {
  if (gi >= it.n || gj >= it.n) return gi == gj ? 1.0 : 0.0;
  double dx = __dsub_rn(xi, xj), dy = __dsub_rn(yi, yj);
  const double s2 = fma(dx, dx, __dmul_rn(dy, dy));
  double r = s2 > 0.0 ? __dmul_rn(s2, rsqrt(s2)) : 0.0;
  double x = __dmul_rn(r, inv_range);
  // sigma^2 times the closed-form polynomial, Horner with fused multiply-adds
  const double s = it.sigma2;
  double v;
  if (it.ktab) {
    // general nu: g(x) below 1, g(x) e^x times e^{-x} from 1 to 2^KNU_EMAX
    // (beyond, the correlation is below the smallest double)
    if (x < 1.0) v = __dmul_rn(s, knu_table(it.ktab, it.ke0, x));
    else if (x < (double)(1 << KNU_EMAX)) v = __dmul_rn(__dmul_rn(s, knu_table(it.ktab, it.ke0, x)), exp_neg(x, tab));
    else v = 0.0;
  } else {
    double poly;
    if (it.nu == 0.5) poly = s;
    else if (it.nu == 1.5) poly = fma(s, x, s);
    else poly = fma(x, fma(x, s * (1.0 / 3.0), s), s);
    v = __dmul_rn(poly, exp_neg(x, tab));
  }
  if (gi == gj) v = __dadd_rn(v, it.nugget);
  return v;
}

constexpr int GEN_ROWS = 16;   // rows of a tile per CTA

// Per-CTA constants of one item's entries.
struct GenCtx {
  const double* tab;     // Tang's tables (float64 evaluation)
  const uint64_t* t2;    // 2^{-j/1024} (fixed-point evaluation)
  double inv_range;
  double sig2_nug;       // sigma^2 + nugget (the diagonal)
  fx ir, sig2;           // 1/range (from a double-double, truncated to 64 bits), sigma^2
  int kind;              // 0, 1, 2 for nu = 1/2, 3/2, 5/2 in fixed point; -1: float64 only
};

__device__ __forceinline__ GenCtx gen_ctx(const ItemGen& it, const double* tab, const uint64_t* t2) {
  GenCtx g;
  g.tab = tab;
  g.t2 = t2;
  g.inv_range = 1.0 / it.range;
  g.sig2_nug = __dadd_rn(it.sigma2, it.nugget);
  g.kind = -1;
  g.ir = g.sig2 = fx{1ull << 63, 0};
  const double ir = g.inv_range;
  // closed-form nu, sigma^2 and 1/range well inside the normal range (each
  // entry's exponent is checked again before it is rounded)
  if (!it.ktab && (it.nu == 0.5 || it.nu == 1.5 || it.nu == 2.5) && it.sigma2 >= 0x1p-900 &&
      it.sigma2 <= 0x1p900 && ir >= 0x1p-900 && ir <= 0x1p900) {
    g.kind = it.nu == 0.5 ? 0 : it.nu == 1.5 ? 1 : 2;
    g.sig2 = fx_of(it.sigma2);
    // 1/range = ir + lo with lo = ir (1 - range ir), the residual exact
    const double lo = fma(-it.range, ir, 1.0) * ir;
    const fx f = fx_of(ir);
    uint64_t m = f.m + (uint64_t)(int64_t)rint(ldexp(lo, 63 - f.e));
    int e = f.e;
    if (m < (1ull << 63)) {   // ir a power of two just above 1/range
      m <<= 1;
      e -= 1;
    }
    g.ir = fx{m, e};
  }
  return g;
}

// The Matérn entry: in fixed point (mp_fixed.cuh) for the closed forms,
// from the float64 squared distance; the float64 evaluation for other nu,
// subnormal or huge distances, x > 700 and results outside the normal range.
// Within 0.56 ulp of the exact value for x up to 100 (against long double
// over 10^7 random pairs, with the float seeds perturbed by 2^-21).
__device__ __forceinline__ double entry(const ItemGen& it, const GenCtx& g, double xi, double yi,
                                        double xj, double yj, int64_t gi, int64_t gj) {
  if (gi >= it.n || gj >= it.n) return gi == gj ? 1.0 : 0.0;
  if (g.kind >= 0) {
    const double dx = __dsub_rn(xi, xj), dy = __dsub_rn(yi, yj);
    const double s2 = fma(dx, dx, __dmul_rn(dy, dy));
    const uint64_t sb = mpx_bits(s2);
    if (sb == 0) return gi == gj ? g.sig2_nug : it.sigma2;
    const uint32_t be = (uint32_t)(sb >> 52);
    if (be != 0 && be < 0x7ff) {
      const fx s = fx_of(s2);
      float fm;
      const int odd = fx_sqrt_prep(s, fm);
      const float r0 = fm * rsqrtf(fm);
      float y;
      asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(r0));
      const fx x = fx_mul(fx_sqrt_finish(s, odd, r0, y), g.ir);
      if (x.e < 9 || (x.e == 9 && x.m <= (700ull << 54))) {
        fx p = g.sig2;
        if (g.kind == 1) {
          p = fx_mul(p, fx_one_plus(x));
        } else if (g.kind == 2) {
          const fx third{12297829382473034411ull, -2};   // 1/3
          p = fx_mul(p, fx_add(fx_one_plus(x), fx_mul(fx_mul(x, x), third)));
        }
        // (s^2 > 0: two points apart, never the diagonal's nugget)
        const fx v = fx_mul(p, fx_exp_neg(x, g.t2));
        if (v.e >= -1022 && v.e <= 1022) return fx_to_double(v);
      }
    }
  }
  return entry_f64(it, g.inv_range, g.tab, xi, yi, xj, yj, gi, gj);
}

// Values outside FP32's normal range (zero, tiny or huge): the conversion
// instructions, out of line so that they stay a branch.
__device__ __noinline__ void store_cvt(char* base, int dt, int64_t i, double v) {
  if (dt == F32) reinterpret_cast<float*>(base)[i] = __double2float_rn(v);
  else reinterpret_cast<__nv_bfloat16*>(base)[i] = __double2bfloat16(v);
}

// v rounded to nearest into format DT (E4M3: v times the tile's 1/scale),
// stored at element i.  FP32 and BF16 round the double's bits with integer
// operations (one rounding to nearest even, as cvt.rn does) when v lies in
// their normal range, since the conversion instructions from float64 take
// the FP64 pipe.
template <int DT>
__device__ __forceinline__ void store_fmt(char* base, int64_t i, double v, double inv_s) {
  if (DT == F64) {
    reinterpret_cast<double*>(base)[i] = v;
  } else if (DT == F32 || DT == BF16) {
    const uint64_t bv = mpx_bits(v);
    const uint64_t mag = bv & 0x7FFFFFFFFFFFFFFFull;
    const uint32_t ed = (uint32_t)(mag >> 52);
    const int drop = DT == F32 ? 29 : 45;         // fraction bits dropped
    if (ed >= 897 && ed <= 1150) {                // 2^-126 <= |v| < 2^128
      const uint64_t r = (mag + ((1ull << (drop - 1)) - 1) + ((mag >> drop) & 1)) >> drop;
      const uint32_t sgn = (uint32_t)(bv >> 63);
      if (DT == F32)
        reinterpret_cast<uint32_t*>(base)[i] = (uint32_t)(r - (896ull << 23)) | (sgn << 31);
      else
        reinterpret_cast<uint16_t*>(base)[i] = (uint16_t)((uint32_t)(r - (896ull << 7)) | (sgn << 15));
    } else {
      store_cvt(base, DT, i, v);
    }
  } else if (DT == F16) {
    reinterpret_cast<__half*>(base)[i] = __double2half(v);
  } else {
    reinterpret_cast<__nv_fp8_storage_t*>(base)[i] =
        __nv_cvt_double_to_fp8(v * inv_s, __NV_SATFINITE, __NV_E4M3);
  }
}

// GEN_ROWS rows of one tile: entries, their rounding into the tile's format
// and the fixed-point copy of Sigma
template <int DT>
__device__ __forceinline__ void gen_rows(const ItemGen& it, const GenCtx& g, char* dst, double inv_s,
                                         const double* rx, const double* cx, int b, int r0,
                                         int64_t gi0, int64_t gj0) {
  int r = (int)threadIdx.x / b, c = (int)threadIdx.x - r * b;
  while (r < GEN_ROWS) {
    const double v = entry(it, g, rx[2 * r], rx[2 * r + 1], cx[2 * c], cx[2 * c + 1], gi0 + r, gj0 + c);
    const int64_t off = (int64_t)(r0 + r) * b + c;
    store_fmt<DT>(dst, off, v, inv_s);
    if (it.sigfix) it.sigfix[off] = sigma_fix(v, it.sig_e);
    c += blockDim.x;
    while (c >= b) {
      c -= b;
      ++r;
    }
  }
}

// ---------------------------------------------------------- float-float
//
// Tiles stored in FP32 or a 16-bit format, in a matrix that keeps no
// float64 copy of Sigma, only need the entry rounded into their format: it
// is evaluated in float-float arithmetic (pairs h + l of floats, about 2^-44
// relative) on the FP32 pipe, which GB300 runs at 64 times its FP64 rate.
// Error-free transformations: two_sum (Knuth), two_prod (one FMA).
struct ffl { float h, l; };

__device__ __forceinline__ ffl ff_two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ffl ff_fast(float a, float b) {   // |a| >= |b| or a == 0
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ ffl ff_two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ ffl ff_add(ffl a, ffl b) {
  const ffl s = ff_two_sum(a.h, b.h);
  return ff_fast(s.h, s.l + (a.l + b.l));
}
__device__ __forceinline__ ffl ff_mul(ffl a, ffl b) {
  const ffl p = ff_two_prod(a.h, b.h);
  return ff_fast(p.h, fmaf(a.h, b.l, fmaf(a.l, b.h, p.l)));
}
__device__ __forceinline__ ffl ff_sqrt(ffl a) {   // a >= 0
  if (!(a.h > 0.f)) return {0.f, 0.f};
  const float y = __fsqrt_rn(a.h);
  const ffl y2 = ff_two_prod(y, y);
  const float d = ((a.h - y2.h) - y2.l) + a.l;
  return ff_fast(y, d * __fdividef(0.5f, y));
}

// x = h + l with h the first 24 significant bits of x (truncated) and l the
// remaining 29 converted to float (so h + l = x to 2^-48 relative), from
// the bit pattern alone (no FP64 instruction).  ok is false outside
// [2^-60, 2^60] in magnitude (x = 0 is fine).
__device__ __forceinline__ ffl ff_split(double x, bool& ok) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7ff);
  if (e == 0 && (u << 1) == 0) return {0.f, 0.f};
  if (e < 1023 - 60 || e > 1023 + 60) { ok = false; return {0.f, 0.f}; }
  const unsigned sg = (unsigned)(u >> 63) << 31;
  const float h = __uint_as_float(sg | ((unsigned)(e - 1023 + 127) << 23) | (unsigned)((u >> 29) & 0x7fffffu));
  // low 29 bits times 2^(e - 1075), a normal float for e >= 1023 - 60
  const float sc = __uint_as_float((unsigned)(e - 1075 + 127) << 23);
  const float lo = (float)(unsigned)(u & 0x1fffffffu) * sc;
  return {h, sg ? -lo : lo};
}

// e^{-x} for 0 <= x <= 80 in float-float, Tang's table-driven method as in
// exp_neg: -x = (k / 64) ln2 + t with k = rint(-64 x / ln2), t from an exact
// product k (ln2/64)_h (two_prod) and the float remainder of ln2/64 (|t| <=
// ln2/64 with k from a float product); e^t = 1 + q with q = t + t^2/2 in
// float-float and t^3/6 + t^4/24 + t^5/120 in float (below 2.2e-7, the
// truncation below 3e-15); times 2^{j/64} as a float pair and 2^m
// (k = 64 m + j).
__device__ __forceinline__ ffl exp_neg_ff(ffl x, const float* ft) {
  const float kf = rintf(-x.h * ft[130]);                 // k (<= 0)
  const ffl p = ff_two_prod(kf, ft[128]);                 // k (ln2/64)_h exactly
  ffl t = ff_two_sum(-x.h, -p.h);                         // -x - k ln2/64 = t
  t = ff_two_sum(t.h, t.l + ((-x.l - p.l) - kf * ft[129]));
  const ffl t2 = ff_two_prod(t.h, t.h);
  const ffl half_t2 = {0.5f * t2.h, 0.5f * fmaf(2.f * t.h, t.l, t2.l)};
  const float th = t.h;
  const float c = th * th * th * fmaf(th, fmaf(th, 1.f / 120.f, 1.f / 24.f), 1.f / 6.f);
  ffl q = ff_add(t, half_t2);
  q = ff_two_sum(q.h, q.l + c);
  const int k = (int)kf;
  const int m = k >> 6, j = k & 63;                       // k = 64 m + j, 0 <= j < 64
  const ffl T = {ft[j], ft[64 + j]};
  const ffl r = ff_add(T, ff_mul(T, q));                  // 2^{j/64} (1 + q)
  const float sc = __uint_as_float((unsigned)(m + 127) << 23);   // 2^m, m >= -116
  return {r.h * sc, r.l * sc};
}

// Matérn entry in float-float (nu in {1/2, 3/2, 5/2} by `kind` 0, 1, 2;
// off-diagonal tiles): the same formula as `entry` -- x = r (1/range) with
// r = sqrt(dx^2 + dy^2) -- from the float pairs (x_h, x_l, y_h, y_l) of the
// two locations.  big: x > 80 (the caller takes the float64 entry).
__device__ __forceinline__ ffl entry_ff(int kind, ffl inv_range, ffl s2, const float* ft, float4 pi,
                                        float4 pj, bool& big) {
  const ffl dx = ff_add({pi.x, pi.y}, {-pj.x, -pj.y});
  const ffl dy = ff_add({pi.z, pi.w}, {-pj.z, -pj.w});
  const ffl sq = ff_add(ff_mul(dx, dx), ff_mul(dy, dy));
  const ffl x = ff_mul(ff_sqrt(sq), inv_range);
  big = !(x.h <= 80.f);
  if (big) return {0.f, 0.f};
  const ffl e = exp_neg_ff(x, ft);
  ffl poly = s2;
  if (kind == 1) {
    poly = ff_mul(s2, ff_add(x, {1.f, 0.f}));
  } else if (kind == 2) {
    const ffl x2_3 = ff_mul(ff_mul(x, x), {ft[131], ft[132]});
    poly = ff_mul(s2, ff_add(ff_add(x, {1.f, 0.f}), x2_3));
  }
  return ff_mul(poly, e);
}


template <bool AMAX>
__global__ void __launch_bounds__(256, 5) k_generate(Arena A, const ItemGen* __restrict__ items) {
  extern __shared__ double sloc[];           // b column points (x, y) + GEN_ROWS row points
  __shared__ double tab[GEN_TAB];
  __shared__ uint64_t t2[GEN_T2];
  for (int e = threadIdx.x; e < GEN_TAB; e += blockDim.x) tab[e] = c_gen_tab[e];
  for (int e = threadIdx.x; e < GEN_T2; e += blockDim.x) t2[e] = g_gen_t2[e];
  const ItemGen it = items[blockIdx.x];
  const int b = A.b;
  const int r0 = blockIdx.y * GEN_ROWS;
  const int64_t gi0 = (int64_t)it.ti * b + r0, gj0 = (int64_t)it.tj * b;
  double* cx = sloc;
  double* rx = sloc + 2 * b;
  for (int c = threadIdx.x; c < b; c += blockDim.x) {
    int64_t g = gj0 + c;
    cx[2 * c] = g < it.n ? it.locs[2 * g] : 0.0;
    cx[2 * c + 1] = g < it.n ? it.locs[2 * g + 1] : 0.0;
  }
  for (int r = threadIdx.x; r < GEN_ROWS; r += blockDim.x) {
    int64_t g = gi0 + r;
    rx[2 * r] = g < it.n ? it.locs[2 * g] : 0.0;
    rx[2 * r + 1] = g < it.n ? it.locs[2 * g + 1] : 0.0;
  }
  const int dt = A.tiles[it.tile].dt;
  // the item's constants, once per CTA (a division and a few float64
  // operations per thread would add a third to the FP64 work of the entries)
  __shared__ GenCtx s_g;
  __shared__ double s_inv_s;
  if (threadIdx.x == 0) {
    s_g = gen_ctx(it, tab, t2);
    s_inv_s = !AMAX && dt == E4M3 ? 1.0 / e4m3_scale(amax_value(&A.amax[it.tile])) : 1.0;
  }
  __syncthreads();
  char* dst = tile_bytes(A, it.tile);
  const GenCtx& g = s_g;
  const double inv_range = g.inv_range;
  double mx = 0.0;
  const double inv_s = s_inv_s;
  // float-float evaluation: an off-diagonal tile stored in FP32 or a 16-bit
  // format, closed-form nu, no float64 copy of Sigma, locations within
  // [2^-60, 2^60] in magnitude (or zero); the CTA decides as a whole
  bool ff = !AMAX && it.ti != it.tj && !it.sigfix && !it.ktab && (dt == F32 || dt == BF16 || dt == F16);
  if (ff) {
    __shared__ float ftab[GEN_FTAB];
    for (int e = threadIdx.x; e < GEN_FTAB; e += blockDim.x) ftab[e] = c_gen_ftab[e];
    float4* cf = reinterpret_cast<float4*>(sloc + 2 * b + 2 * GEN_ROWS);   // b columns, then GEN_ROWS rows
    bool ok = true;
    const ffl inv = ff_split(inv_range, ok), s2 = ff_split(it.sigma2, ok);
    for (int q = threadIdx.x; q < b + GEN_ROWS; q += blockDim.x) {
      const double* pt = q < b ? cx + 2 * q : rx + 2 * (q - b);
      const ffl px = ff_split(pt[0], ok), py = ff_split(pt[1], ok);
      cf[q] = make_float4(px.h, px.l, py.h, py.l);
    }
    ff = __syncthreads_and(ok);
    if (ff) {
      const int kind = it.nu == 0.5 ? 0 : it.nu == 1.5 ? 1 : 2;
      for (int e = threadIdx.x; e < GEN_ROWS * b; e += blockDim.x) {
        const int r = e / b, c = e - r * b;
        const int64_t gi = gi0 + r, gj = gj0 + c;
        const int64_t off = (int64_t)(r0 + r) * b + c;
        float f;
        if (gi >= it.n || gj >= it.n) {
          f = 0.f;                                 // identity padding (off the diagonal)
        } else {
          bool big;
          const ffl v = entry_ff(kind, inv, s2, ftab, cf[b + r], cf[c], big);
          if (big)                                 // x > 80: the float64 entry
            f = (float)entry(it, g, rx[2 * r], rx[2 * r + 1], cx[2 * c], cx[2 * c + 1], gi, gj);
          else
            f = __fadd_rn(v.h, v.l);
        }
        if (dt == F32) reinterpret_cast<float*>(dst)[off] = f;
        else store_round_f32(dst, dt, off, f);
      }
      if (blockIdx.y == 0 && threadIdx.x == 0) A.scale[it.tile] = 1.0;
      return;
    }
  }
  if (AMAX) {
    for (int e = threadIdx.x; e < GEN_ROWS * b; e += blockDim.x) {
      const int r = e / b, c = e - r * b;
      mx = fmax(mx, fabs(entry(it, g, rx[2 * r], rx[2 * r + 1], cx[2 * c], cx[2 * c + 1], gi0 + r, gj0 + c)));
    }
  } else {
    switch (dt) {
      case F64: gen_rows<F64>(it, g, dst, inv_s, rx, cx, b, r0, gi0, gj0); break;
      case F32: gen_rows<F32>(it, g, dst, inv_s, rx, cx, b, r0, gi0, gj0); break;
      case BF16: gen_rows<BF16>(it, g, dst, inv_s, rx, cx, b, r0, gi0, gj0); break;
      case F16: gen_rows<F16>(it, g, dst, inv_s, rx, cx, b, r0, gi0, gj0); break;
      default: gen_rows<E4M3>(it, g, dst, inv_s, rx, cx, b, r0, gi0, gj0);
    }
  }
  if (AMAX) {
    __shared__ double red[8];
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
      atomic_max_pos(&A.amax[it.tile], mx);
    }
  } else if (blockIdx.y == 0 && threadIdx.x == 0) {
    A.scale[it.tile] = dt == E4M3 ? e4m3_scale(amax_value(&A.amax[it.tile])) : 1.0;
    if (it.sigfix && it.ti == 0 && it.tj == 0) *it.sig_e_out = it.sig_e;
  }
}

// Sum of squares of 16 rows of one generated tile, written to a per-CTA
// partial (reduced in a fixed order by k_reduce_norms: deterministic).
__global__ void __launch_bounds__(256) k_tile_sumsq(int b, const ItemGen* __restrict__ items,
                                                    double* __restrict__ partial) {
  extern __shared__ double sloc[];
  __shared__ double tab[GEN_TAB];
  __shared__ uint64_t t2[GEN_T2];
  for (int e = threadIdx.x; e < GEN_TAB; e += blockDim.x) tab[e] = c_gen_tab[e];
  for (int e = threadIdx.x; e < GEN_T2; e += blockDim.x) t2[e] = g_gen_t2[e];
  const ItemGen it = items[blockIdx.x];
  const int r0 = blockIdx.y * GEN_ROWS;
  const int64_t gi0 = (int64_t)it.ti * b + r0, gj0 = (int64_t)it.tj * b;
  double* cx = sloc;
  double* rx = sloc + 2 * b;
  for (int c = threadIdx.x; c < b; c += blockDim.x) {
    int64_t g = gj0 + c;
    cx[2 * c] = g < it.n ? it.locs[2 * g] : 0.0;
    cx[2 * c + 1] = g < it.n ? it.locs[2 * g + 1] : 0.0;
  }
  for (int r = threadIdx.x; r < GEN_ROWS; r += blockDim.x) {
    int64_t g = gi0 + r;
    rx[2 * r] = g < it.n ? it.locs[2 * g] : 0.0;
    rx[2 * r + 1] = g < it.n ? it.locs[2 * g + 1] : 0.0;
  }
  __shared__ GenCtx s_g;
  if (threadIdx.x == 0) s_g = gen_ctx(it, tab, t2);
  __syncthreads();
  const GenCtx& g = s_g;
  double ss = 0.0;
  for (int e = threadIdx.x; e < GEN_ROWS * b; e += blockDim.x) {
    int r = e / b, c = e - r * b;
    double v = entry(it, g, rx[2 * r], rx[2 * r + 1], cx[2 * c], cx[2 * c + 1], gi0 + r, gj0 + c);
    ss += v * v;
  }
  __shared__ double red[8];
  ss = warp_sum(ss);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) ss += red[w];
    partial[(int64_t)blockIdx.x * gridDim.y + blockIdx.y] = ss;
  }
}

__global__ void k_reduce_norms(const ItemGen* __restrict__ items, int count, int parts, int nt,
                               const double* __restrict__ partial, double* __restrict__ norms) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  double s = 0.0;
  for (int p = 0; p < parts; ++p) s += partial[(int64_t)t * parts + p];
  norms[items[t].ti * nt + items[t].tj] = sqrt(s);
}

}  // namespace

// ---------------------------------------------------------------- general nu
//
// g(x) = 2^(1-nu) / Gamma(nu) x^nu K_nu(x) (g(0) = 1) at a node x > 0 from the
// integral representation K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt
// by the trapezoidal rule, which converges geometrically for this
// integrand (analytic in the strip |Im t| < pi/2 and decaying doubly
// exponentially): step h = the power of two at most min(1/4, 1/(2 sqrt x),
// 1/(nu + 2)) / 2, terms
// summed with Kahan compensation until they fall below 1e-22 of the sum
// past the integrand's peak.  For x >= 1 the factor e^x is folded in
// (exp(-x (cosh t - 1)) in place of exp(-x cosh t), with cosh t - 1 =
// 2 sinh^2(t/2) to keep it accurate), so that the table stays finite where
// K_nu underflows.  The x^nu and cosh(nu t) factors are multiplied, not
// added as logarithms (a logarithm of 30 carries 30 units of rounding).
static double knu_node(double x, double nu) {
  // a power of two at most half the step bound, so that every node t = k h
  // is exact; nu t is then carried as p + e (e from a fused multiply-add)
  // and cosh(p + e) = cosh p + e sinh p to first order
  const double hb = 0.5 * std::fmin(std::fmin(0.25, 0.5 / std::sqrt(x)), 1.0 / (nu + 2.0));
  const double h = std::ldexp(1.0, (int)std::floor(std::log2(hb)));
  const bool scaled = x >= 1.0;
  const double xn = std::pow(x, nu);
  double sum = 0.0, comp = 0.0;
  for (int k = 0; k < 1000000; ++k) {
    const double t = k * h;
    const double sh = std::sinh(0.5 * t);
    const double y = scaled ? 2.0 * x * sh * sh : x * std::cosh(t);
    const double p = nu * t, e = std::fma(nu, t, -p);
    double term = xn * std::fma(e, std::sinh(p), std::cosh(p)) * std::exp(-y);
    if (k == 0) term *= 0.5;
    const double yk = term - comp;
    const double tk = sum + yk;
    comp = (tk - sum) - yk;
    sum = tk;
    if (k > 0 && term < 1e-22 * sum && y > nu * t + 5.0) break;
  }
  return std::exp2(1.0 - nu) / std::tgamma(nu) * sum * h;
}

bool matern_nu_closed(double nu) { return nu == 0.5 || nu == 1.5 || nu == 2.5; }
bool matern_nu_valid(double nu) { return nu > 0.0 && nu <= KNU_NU_MAX; }

// Chebyshev interpolation of g on each half octave at the KNU_COEF
// Chebyshev points of the first kind; the angle of T_m at node j, m (2j+1)
// pi / (2 KNU_COEF), is reduced as an integer before the cosine.  The
// table starts at 2^e0 with e0 = min(-32, floor(-54 / (2 nu))): below it
// both the regular part of g (1 - x^2 / (4 (nu - 1)) + ..., with an
// x^2 log x term at nu = 1) and the singular part (a multiple of x^(2 nu))
// differ from 1 by less than 2^-54, so g = 1 there.
int matern_nu_table(double nu, std::vector<double>& coef, int* e0) {
  if (!matern_nu_valid(nu)) return 1;
  const int lo = std::max(-1022, std::min(-32, (int)std::floor(-54.0 / (2.0 * nu))));
  const int pieces = 2 * (KNU_EMAX - lo);
  coef.assign((size_t)pieces * KNU_COEF, 0.0);
  const double pi = 3.14159265358979323846;
  double f[KNU_COEF], cs[4 * KNU_COEF];
  for (int q = 0; q < 4 * KNU_COEF; ++q) cs[q] = std::cos(pi * q / (2.0 * KNU_COEF));
  for (int p = 0; p < pieces; ++p) {
    const int E = lo + p / 2;
    const double centre = (p & 1) ? 1.75 : 1.25;
    for (int j = 0; j < KNU_COEF; ++j) {
      const double u = cs[2 * j + 1];                 // cos((j + 1/2) pi / KNU_COEF)
      f[j] = knu_node(std::ldexp(centre + 0.25 * u, E), nu);
    }
    for (int m = 0; m < KNU_COEF; ++m) {
      double acc = 0.0;
      for (int j = 0; j < KNU_COEF; ++j) acc += f[j] * cs[(m * (2 * j + 1)) % (4 * KNU_COEF)];
      coef[(size_t)p * KNU_COEF + m] = (m == 0 ? 1.0 : 2.0) / KNU_COEF * acc;
    }
  }
  *e0 = lo;
  return 0;
}

double matern_nu_host(const double* coef, int e0, double x) {
  if (!(x > 0.0)) return 1.0;
  if (x >= std::ldexp(1.0, KNU_EMAX)) return 0.0;
  int ex;
  const double fr = std::frexp(x, &ex);            // x = fr 2^ex, fr in [0.5, 1)
  const int E = ex - 1;
  if (E < e0) return 1.0;
  const double m = 2.0 * fr;
  const int upper = m >= 1.5;
  const double u = 4.0 * (m - (upper ? 1.75 : 1.25));
  const double* c = coef + (size_t)(2 * (E - e0) + upper) * KNU_COEF;
  double b1 = 0.0, b2 = 0.0;
  for (int k = KNU_COEF - 1; k >= 1; --k) {
    const double t = 2.0 * u * b1 - b2 + c[k];
    b2 = b1;
    b1 = t;
  }
  const double g = u * b1 - b2 + c[0];
  return x < 1.0 ? g : g * std::exp(-x);
}

// The e^{-x} tables of the current device, from long double arithmetic on
// the host (2^{j/64} as a double plus its remainder; ln2/64 as a 37-bit head
// plus its remainder).
int init_gen_tables() {
  double h[GEN_TAB];
  for (int j = 0; j < 64; ++j) {
    const long double v = std::exp2((long double)j / 64.0L);
    h[j] = (double)v;
    h[64 + j] = (double)(v - (long double)h[j]);
  }
  const long double l = std::log(2.0L) / 64.0L;
  double head = (double)l;
  uint64_t u;
  std::memcpy(&u, &head, sizeof(u));
  u &= ~(uint64_t)0xFFFF;   // 53 - 16 = 37 significant bits
  std::memcpy(&head, &u, sizeof(u));
  h[128] = head;
  h[129] = (double)(l - (long double)head);
  h[130] = (double)(64.0L / std::log(2.0L));
  float f[GEN_FTAB];
  for (int j = 0; j < 64; ++j) {
    const long double v = std::exp2((long double)j / 64.0L);
    f[j] = (float)v;
    f[64 + j] = (float)(v - (long double)f[j]);
  }
  f[128] = (float)l;
  f[129] = (float)(l - (long double)f[128]);
  f[130] = (float)(64.0L / std::log(2.0L));
  f[131] = (float)(1.0L / 3.0L);
  f[132] = (float)(1.0L / 3.0L - (long double)f[131]);
  if (cudaMemcpyToSymbol(c_gen_ftab, f, sizeof(f)) != cudaSuccess) return 1;
  // 2^{-j/1024} 2^63 to nearest: long double holds it within half a unit
  // of 2^-63 (64 significant bits or more)
  uint64_t t[GEN_T2];
  for (int j = 0; j < GEN_T2; ++j)
    t[j] = (uint64_t)std::floor(std::ldexp(std::exp2(-(long double)j / GEN_T2), 63) + 0.5L);
  if (cudaMemcpyToSymbol(g_gen_t2, t, sizeof(t)) != cudaSuccess) return 1;
  return cudaMemcpyToSymbol(c_gen_tab, h, sizeof(h)) == cudaSuccess ? 0 : 1;
}

int tile_norm_parts(int b) { return b / GEN_ROWS; }

void launch_tile_norms(int b, const ItemGen* items, int count, int nt, double* partial,
                       double* norms, cudaStream_t s) {
  if (count <= 0) return;
  dim3 grid(count, b / GEN_ROWS);
  size_t smem = sizeof(double) * (2 * b + 2 * GEN_ROWS);
  k_tile_sumsq<<<grid, 256, smem, s>>>(b, items, partial);
  k_reduce_norms<<<(count + 127) / 128, 128, 0, s>>>(items, count, b / GEN_ROWS, nt, partial, norms);
}

void launch_morton_keys(const double* locs, int64_t n, int64_t n2, unsigned long long* keys,
                        cudaStream_t s) {
  k_morton_keys<<<(unsigned)((n2 + 255) / 256), 256, 0, s>>>(locs, n, n2, keys);
}

void launch_bitonic(unsigned long long* keys, int64_t n2, cudaStream_t s) {
  // n2 is a power of two >= 1024
  unsigned blocks_local = (unsigned)(n2 / 1024);
  k_bitonic_local<<<blocks_local, 512, 0, s>>>(keys, n2, 2, 1024);
  for (int64_t k = 2048; k <= n2; k <<= 1) {
    for (int64_t j = k >> 1; j >= 1024; j >>= 1)
      k_bitonic_global<<<(unsigned)(n2 / 256), 256, 0, s>>>(keys, n2, j, k);
    k_bitonic_local<<<blocks_local, 512, 0, s>>>(keys, n2, k, k);
  }
}

void launch_morton_gather(const unsigned long long* keys, const double* in, int64_t n,
                          double* out, int64_t* perm, cudaStream_t s) {
  k_morton_gather<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(keys, in, n, out, perm);
}

void launch_gen_amax(const Arena& A, const ItemGen* items, int count, cudaStream_t s) {
  if (count <= 0) return;
  dim3 grid(count, A.b / GEN_ROWS);
  size_t smem = sizeof(double) * (2 * A.b + 2 * GEN_ROWS);
  k_generate<true><<<grid, 256, smem, s>>>(A, items);
}

void launch_generate(const Arena& A, const ItemGen* items, int count, cudaStream_t s) {
  if (count <= 0) return;
  dim3 grid(count, A.b / GEN_ROWS);
  // the locations as doubles, then as float pairs (float-float tiles)
  size_t smem = sizeof(double) * (2 * A.b + 2 * GEN_ROWS) + sizeof(float4) * (A.b + GEN_ROWS);
  k_generate<false><<<grid, 256, smem, s>>>(A, items);
}

}  // namespace mp
