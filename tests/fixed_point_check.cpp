// Host check of the fixed-point Matérn arithmetic (mp_fixed.cuh) against
// long double: the header's functions compiled for the CPU, the GPU's
// approximate float seeds (rsqrt, reciprocal) replaced by correctly rounded
// ones perturbed by up to 2^-21 relative.  Prints one JSON line:
//   sqrt_units   worst |error| of sqrt(s) in units of 2^-63 (relative)
//   exp_units    worst |error| of e^{-x}, 0 < x <= 100, units of 2^-63
//   exp700_units the same for 0 < x <= 700
//   entry_ulp    worst |error| in ulps of sigma^2 P(x) e^{-x} (nu = 1/2,
//                3/2, 5/2) against long double at the same float64 s^2,
//                less x/128 (x's own error, a few units of 2^-63 relative,
//                is carried x-fold by e^{-x}); ranges 0.05 and 0.005 (x up
//                to about 280 on the unit square)
//   sigma_fix_bad  codes of the refinement's fixed-point copy that differ
//                  from round-half-even of v 2^(62 - E) (0 for v in [0, 2^E),
//                  2^62 - 1 at or above)
// Usage: fixed_point_check <samples>
#define MPX_FN static inline
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>

#include "../paper_2406_02701_gb300/csrc/mp_fixed.cuh"

using mp::fx;

static uint64_t T2[1024];
static std::mt19937_64 rng(7);
static double urand() { return (double)(rng() >> 11) * 0x1.0p-53; }
static float perturb(float f) { return (float)((double)f * (1.0 + (urand() * 2 - 1) * 0x1.0p-21)); }
static long double value(fx a) { return ldexpl((long double)a.m, a.e - 63); }

static fx sqrt_fx(fx s) {
  float fm;
  const int odd = mp::fx_sqrt_prep(s, fm);
  const float r0 = perturb(std::sqrt(fm));
  const float y = perturb(1.0f / r0);
  return mp::fx_sqrt_finish(s, odd, r0, y);
}

int main(int argc, char** argv) {
  const long N = argc > 1 ? atol(argv[1]) : 1000000;
  for (int j = 0; j < 1024; ++j)
    T2[j] = (uint64_t)floorl(ldexpl(exp2l(-(long double)j / 1024.0L), 63) + 0.5L);
  double sq = 0, ex = 0, ex7 = 0, ent = 0;
  for (long t = 0; t < N; ++t) {
    const double s = ldexp(1.0 + urand(), (int)(rng() % 400) - 200);
    const long double r = sqrtl((long double)s);
    sq = fmax(sq, (double)(fabsl((value(sqrt_fx(mp::fx_of(s))) - r) / r) * 0x1.0p63L));
  }
  for (long t = 0; t < N; ++t) {
    const double x = (t & 1) ? urand() * 700 : ldexp(1.0 + urand(), -(int)(rng() % 80));
    if (!(x > 0)) continue;
    const long double r = expl(-(long double)x);
    const double e = (double)(fabsl((value(mp::fx_exp_neg(mp::fx_of(x), T2)) - r) / r) * 0x1.0p63L);
    ex7 = fmax(ex7, e);
    if (x <= 100) ex = fmax(ex, e);
  }
  const fx third{12297829382473034411ull, -2};
  const double sig2 = 1.3;
  for (int kr = 0; kr < 6; ++kr) {
    const int kind = kr % 3;
    const double range = kr < 3 ? 0.05 : 0.005;
    const long double irl = 1.0L / (long double)range;
    int ie;
    frexpl(irl, &ie);
    const fx IR{(uint64_t)floorl(ldexpl(irl, 64 - ie) + 0.5L), ie - 1};
    for (long t = 0; t < N; ++t) {
      const double xi = urand(), yi = urand();
      double xj = urand(), yj = urand();
      if (t % 7 == 0) {
        xj = xi + (urand() - 0.5) * 1e-6;
        yj = yi + (urand() - 0.5) * 1e-6;
      }
      const double dx = xi - xj, dy = yi - yj;
      const double s2 = std::fma(dx, dx, dy * dy);
      if (s2 == 0) continue;
      const fx X = mp::fx_mul(sqrt_fx(mp::fx_of(s2)), IR);
      if (X.e > 9) continue;
      const fx E = mp::fx_exp_neg(X, T2);
      fx P = mp::fx_of(sig2);
      if (kind == 1) P = mp::fx_mul(P, mp::fx_one_plus(X));
      if (kind == 2) P = mp::fx_mul(P, mp::fx_add(mp::fx_one_plus(X), mp::fx_mul(mp::fx_mul(X, X), third)));
      const double v = mp::fx_to_double(mp::fx_mul(P, E));
      const long double xl = sqrtl((long double)s2) / (long double)range;
      const long double pl = kind == 0 ? 1.0L : kind == 1 ? 1.0L + xl : 1.0L + xl + xl * xl / 3.0L;
      const long double ref = (long double)sig2 * pl * expl(-xl);
      int e;
      frexpl(ref, &e);
      ent = fmax(ent, (double)(fabsl(((long double)v - ref) / ldexpl(1.0L, e - 53)) - xl / 128));
    }
  }
  long bad = 0;
  for (long t = 0; t < N; ++t) {
    const int E = (int)(rng() % 2001) - 1000;
    const int k = (int)(rng() % 80);             // v about 2^(E - k)
    double v = ldexp(urand(), E - k);
    if (t % 97 == 0) v = ldexp(1.0, E - 1 - (int)(rng() % 3));
    if (t % 101 == 0) v = ldexp(1.0 + urand(), E + (int)(rng() % 3));   // at or above 2^E
    if (t % 103 == 0) v = 0.0;
    if (!(v < 0x1p1023) || (v != 0 && v < 0x1p-1022)) continue;   // normal doubles and zero
    uint64_t want;
    if (v >= ldexp(1.0, E)) want = (1ull << 62) - 1;
    else want = (uint64_t)nearbyintl(ldexpl((long double)v, 62 - E));
    if (mp::sigma_fix(v, E) != want) ++bad;
  }
  printf("{\"sqrt_units\": %.4f, \"exp_units\": %.4f, \"exp700_units\": %.4f, \"entry_ulp\": %.4f, "
         "\"sigma_fix_bad\": %ld}\n", sq, ex, ex7, ent, bad);
  return 0;
}
