// Matérn closed forms in 64-bit fixed point, on the integer pipe.
//
// GB300 issues integer multiply-adds at about 32 times its FP64 rate, and
// the generation of a covariance entry in float64 (a square root, e^{-x},
// the polynomial) takes about thirty FP64-pipe operations.  Here only the
// coordinate differences and the squared distance stay in float64; the rest
// runs on unsigned 64-bit significands:
//
//   fx = m 2^(e - 63), m in [2^63, 2^64)        (positive reals)
//
// * sqrt: a float seed r0 = sqrt(mv) good to about 2^-22 (mv the
//   significand of s^2 scaled to [1, 4)), the exact residual d = mv - r0^2
//   in integers, and the second-order expansion
//   sqrt(r0^2 + d) = r0 + c - c^2 / (2 r0), c = d / (2 r0) (the next term,
//   c^3 / (2 r0^2), is below 2^-64); 1/r0 from a float reciprocal refined
//   by one Newton step.  Within a few units of 2^-63.
// * e^{-x}, after Tang's table-driven reduction (P. T. P. Tang, ACM TOMS
//   15, 1989) with 1024 subintervals: x 1024/ln2 = k + f (k integer,
//   f in [0, 1)) from the 128-bit product with a 64-bit 1024/ln2, then
//   e^{-x} = 2^{-(k >> 10)} 2^{-(k & 1023)/1024} e^{-u}, u = f ln2/1024 <
//   2^-10.5, and e^{-u} = 1 - u + u^2/2 - u^3 (1/6 - u/24 + u^2/120) (the
//   omitted u^6/720 is below 2^-70); the table holds 2^{-j/1024} rounded to
//   64 bits.
// * Products truncate (each within 2^-62); one rounding to nearest at the
//   end gives the double.  In all about ten units of 2^-63 before that
//   rounding.
#pragma once
#include <cstdint>

#ifndef MPX_FN
#define MPX_FN __device__ __forceinline__
#endif

namespace mp {

struct fx {
  uint64_t m;   // significand, top bit set
  int e;        // value m 2^(e - 63)
};

MPX_FN uint64_t mpx_mulhi(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

MPX_FN int64_t mpx_mulhi_s(int64_t a, int64_t b) {
#ifdef __CUDA_ARCH__
  return __mul64hi(a, b);
#else
  return (int64_t)(((__int128)a * b) >> 64);
#endif
}

MPX_FN int mpx_clz(uint64_t a) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)a);
#else
  return __builtin_clzll(a);
#endif
}

MPX_FN uint64_t mpx_bits(double d) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(d);
#else
  uint64_t u;
  __builtin_memcpy(&u, &d, sizeof(u));
  return u;
#endif
}

MPX_FN double mpx_double(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double d;
  __builtin_memcpy(&d, &u, sizeof(d));
  return d;
#endif
}

// a positive normal double, exactly
MPX_FN fx fx_of(double d) {
  const uint64_t u = mpx_bits(d);
  return fx{(u << 11) | (1ull << 63), (int)(u >> 52) - 1023};
}

// the double nearest a (its exponent within the normal range)
MPX_FN double fx_to_double(fx a) {
  uint64_t mant = a.m >> 11;                    // [2^52, 2^53)
  const uint64_t rem = a.m & 0x7ff;
  mant += (rem > 0x400) | ((rem == 0x400) & (mant & 1));
  // the implicit bit of mant adds one to the exponent field (two on a carry)
  return mpx_double(((uint64_t)(a.e + 1022) << 52) + mant);
}

MPX_FN fx fx_mul(fx a, fx b) {
  const uint64_t p = mpx_mulhi(a.m, b.m);       // [2^62, 2^64): p 2^(a.e + b.e - 62)
  const int top = (int)(p >> 63);
  return fx{top ? p : p << 1, a.e + b.e + top};
}

// a + b for positive a, b
MPX_FN fx fx_add(fx a, fx b) {
  if (a.e < b.e) {
    const fx t = a;
    a = b;
    b = t;
  }
  const int d = a.e - b.e;
  const uint64_t s = a.m + (d < 64 ? b.m >> d : 0);
  if (s < a.m) return fx{(s >> 1) | (1ull << 63), a.e + 1};
  return fx{s, a.e};
}

// 1 + x
MPX_FN fx fx_one_plus(fx x) {
  if (x.e >= 0) {
    const uint64_t s = x.m + (x.e < 64 ? 1ull << (63 - x.e) : 0);
    if (s < x.m) return fx{(s >> 1) | (1ull << 63), x.e + 1};
    return fx{s, x.e};
  }
  const int d = -x.e;
  return fx{(1ull << 63) + (d < 64 ? x.m >> d : 0), 0};
}

// sqrt(s) in two parts around the caller's float seeds: fx_sqrt_prep gives
// mv in [1, 4) as a float (its leading 24 bits) and whether s's exponent is
// odd; the caller forms r0 ~ sqrt(mv) and y ~ 1/r0 (each within about
// 2^-22) and fx_sqrt_finish refines them
MPX_FN int fx_sqrt_prep(fx s, float& fm) {
  const int odd = s.e & 1;                      // s = mv 2^(s.e - odd), mv in [1, 4)
  const uint32_t fb = ((uint32_t)(127 + odd) << 23) | (uint32_t)((s.m >> 40) & 0x7FFFFF);
#ifdef __CUDA_ARCH__
  fm = __uint_as_float(fb);
#else
  __builtin_memcpy(&fm, &fb, sizeof(fm));
#endif
  return odd;
}

MPX_FN uint32_t mpx_fbits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  uint32_t u;
  __builtin_memcpy(&u, &f, sizeof(u));
  return u;
#endif
}

// r0f ~ sqrt(mv) in (0.99, 2], yf ~ 1/r0f in [0.5, 1.01)
MPX_FN fx fx_sqrt_finish(fx s, int odd, float r0f, float yf) {
  const uint64_t Mv = odd ? s.m : s.m >> 1;     // mv 2^62
  const uint32_t rb = mpx_fbits(r0f);
  const int re = (int)(rb >> 23) - 127;         // -1, 0 or 1
  const uint32_t rm = (rb & 0x7FFFFF) | 0x800000;
  const uint32_t R0 = re == 0 ? rm : re > 0 ? rm << 1 : rm >> 1;   // r0 = R0 2^-23
  // d = mv - r0^2 in units of 2^-62 (exact; the difference fits although
  // r0^2 2^62 may reach 2^64)
  const int64_t D = (int64_t)(Mv - (((uint64_t)R0 * R0) << 16));
  // 1/r0 = Y0 2^-29 within 2^-22, then Y1 2^-76 = 1/R0 within 2^-43 (one
  // Newton step; |Y0 dl| < 2^62 for seeds within 2^-20)
  const uint32_t yb = mpx_fbits(yf);
  const int ye = (int)(yb >> 23) - 127;         // -1 or 0
  const uint32_t Y0 = ((yb & 0x7FFFFF) | 0x800000) << (6 + ye);
  const int64_t dl = (int64_t)((1ull << 52) - (uint64_t)R0 * Y0);
  const uint64_t Y1 = ((uint64_t)Y0 << 24) + (uint64_t)(((int64_t)Y0 * dl) >> 28);
  // c = d / (2 r0) and c^2 / (2 r0) in units of 2^-63
  const int64_t c = mpx_mulhi_s((int64_t)((uint64_t)D << 11), (int64_t)Y1);
  const uint64_t ac = (uint64_t)(c < 0 ? -c : c);
  const uint64_t c2 = (mpx_mulhi(ac, ac) * Y0) >> 29;
  uint64_t R = ((uint64_t)R0 << 40) + (uint64_t)c - c2;
  R = R < (1ull << 63) ? (1ull << 63) : R;      // sqrt(mv) >= 1
  return fx{R, (s.e - odd) >> 1};
}

// e^{-x} for 0 < x <= 700 (x.e <= 9); t2[j] = 2^{-j/1024} 2^63 rounded
MPX_FN fx fx_exp_neg(fx x, const uint64_t* t2) {
  const uint64_t L = 13306513097844322492ull;   // 1024/ln2 2^53, rounded
  const uint64_t hi = mpx_mulhi(x.m, L), lo = x.m * L;
  const int sh = 116 - x.e;                     // binary point of hi:lo (>= 107)
  uint32_t k;
  uint64_t F;                                   // f 2^64
  if (sh < 128) {
    k = (uint32_t)(hi >> (sh - 64));
    F = (hi << (128 - sh)) | (lo >> (sh - 64));
  } else {
    k = 0;
    F = sh < 192 ? hi >> (sh - 128) : 0;
  }
  const uint64_t U = mpx_mulhi(F, 12786308645202655660ull);   // u 2^74 (ln2 2^64 rounded)
  const uint64_t U2 = mpx_mulhi(U, U);                        // u^2 2^84
  const uint64_t U3 = mpx_mulhi(U2, U);                       // u^3 2^94
  const uint64_t u32 = U >> 42;                               // u 2^32 (< 2^22)
  // (1/6 - u/24 + u^2/120) 2^32
  const uint64_t q = 715827883ull - ((u32 * 178956971ull) >> 32) +
                     ((((u32 * u32) >> 32) * 35791394ull) >> 32);
  const uint64_t t3 = ((U3 >> 31) * q) >> 32;                 // u^3 q 2^63
  const uint64_t G = (1ull << 63) - (U >> 11) + (U2 >> 22) - t3;   // e^{-u} 2^63
  const uint64_t E = mpx_mulhi(t2[k & 1023], G) << 1;          // 2^{-j/1024} e^{-u} 2^63
  const int z = mpx_clz(E);
  return fx{E << z, -(int)(k >> 10) - z};
}

// The refinement's fixed-point copy of Sigma: round(v 2^(62 - E)) to
// nearest even for 0 <= v < 2^E (exact for v >= 2^(E - 9); entries far
// below 2^E keep their absolute accuracy, 2^(E - 63), which is what a
// residual sum of them needs); values at or above 2^E (the identity
// padding, when sigma^2 + nugget < 1) clamp to 2^62 - 1: the residual only
// ever multiplies them by zero.
MPX_FN uint64_t sigma_fix(double v, int E) {
  const uint64_t bv = mpx_bits(v);
  const int be = (int)(bv >> 52);
  if (be == 0) return 0ull;                      // zero or subnormal: below 2^-1022
  const uint64_t mant = (bv & ((1ull << 52) - 1)) | (1ull << 52);
  const int sh = be - 1075 + 62 - E;             // v = mant 2^(be - 1075)
  if (sh >= 10) return (1ull << 62) - 1;         // v >= 2^E
  if (sh >= 0) return mant << sh;
  const int d = -sh;
  if (d > 54) return 0ull;
  return (mant + (1ull << (d - 1)) - 1 + ((mant >> d) & 1)) >> d;
}

}  // namespace mp
