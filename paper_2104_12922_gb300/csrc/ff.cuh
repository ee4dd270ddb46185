// ff.cuh -- float-float ("double-single") arithmetic for the control-rate
// pitch chain.
//
// GB300's FP64 units issue at a small fraction of the FP32 rate, so the
// precision-critical control-rate values (envelopes, LFOs, modulation sums,
// pitch, per-interval phase sums) are carried as an unevaluated sum hi + lo
// of two floats (about 48 significant bits). The building blocks are the
// error-free transformations of Dekker (1971) and Knuth (TAOCP vol. 2): TwoSum,
// Fast-TwoSum and FMA-based TwoProd, combined as in the double-double
// algorithms of Hida, Li and Bailey (QD library, ARITH-15, 2001).
// Transcendentals are written from their series with table-based argument
// reduction; their tables are built from FP64 values at run time.
//
// The header compiles for host (g++) and device (nvcc) so that its accuracy
// can be tested on the CPU.
#pragma once

#include <math.h>

#ifdef __CUDACC__
#define FF_HD __host__ __device__ __forceinline__
#else
#define FF_HD inline
#endif

namespace synth {

struct ff {
  float hi, lo;
};

FF_HD ff ff_make(float a) { return {a, 0.0f}; }
FF_HD ff ff_from_double(double d) {
  const float hi = (float)d;
  return {hi, (float)(d - (double)hi)};
}
FF_HD double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }
FF_HD float ff_to_float(ff a) { return a.hi + a.lo; }

// Knuth TwoSum: s + e == a + b exactly.
FF_HD ff two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
// Dekker Fast-TwoSum, valid when |a| >= |b| (or a == 0).
FF_HD ff quick_two_sum(float a, float b) {
  const float s = a + b;
  const float e = b - (s - a);
  return {s, e};
}
// TwoProd with a fused multiply-add: p + e == a * b exactly.
FF_HD ff two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}

FF_HD ff ff_add(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  const ff t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}
FF_HD ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
FF_HD ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
FF_HD ff ff_add_f(ff a, float b) {
  ff s = two_sum(a.hi, b);
  s.lo += a.lo;
  return quick_two_sum(s.hi, s.lo);
}
FF_HD ff ff_mul(ff a, ff b) {
  ff p = two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return quick_two_sum(p.hi, p.lo);
}
FF_HD ff ff_mul_f(ff a, float b) {
  ff p = two_prod(a.hi, b);
  p.lo = fmaf(a.lo, b, p.lo);
  return quick_two_sum(p.hi, p.lo);
}
// Scale by a power of two (exact barring under/overflow).
FF_HD ff ff_ldexp(ff a, int e) { return {ldexpf(a.hi, e), ldexpf(a.lo, e)}; }
// a / b: long division, two quotient digits and a correction.
FF_HD ff ff_div(ff a, ff b) {
  const float q1 = a.hi / b.hi;
  ff r = ff_sub(a, ff_mul_f(b, q1));
  const float q2 = r.hi / b.hi;
  r = ff_sub(r, ff_mul_f(b, q2));
  const float q3 = r.hi / b.hi;
  ff q = quick_two_sum(q1, q2);
  return ff_add_f(q, q3);
}
FF_HD bool ff_lt(ff a, ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
FF_HD bool ff_gt(ff a, ff b) { return ff_lt(b, a); }
FF_HD ff ff_min(ff a, ff b) { return ff_lt(b, a) ? b : a; }
FF_HD ff ff_max(ff a, ff b) { return ff_lt(a, b) ? b : a; }
FF_HD ff ff_abs(ff a) { return a.hi < 0.0f ? ff_neg(a) : a; }
// floor, for values whose integer part fits a float exactly
FF_HD ff ff_floor(ff a) {
  float f = floorf(a.hi);
  if (f == a.hi) return quick_two_sum(f, floorf(a.lo));
  return {f, 0.0f};
}
FF_HD ff ff_frac(ff a) { return ff_sub(a, ff_floor(a)); }

// Tables for argument reduction, filled from FP64 by ff_tables_init:
//  exp2_tab[j + 16] = 2^(j/32), j = -16..16
//  sin_tab[m] = sin(2 pi m / 128), cos_tab[m] = cos(2 pi m / 128), m = 0..16
struct FFTables {
  ff exp2_tab[33];
  ff sin_tab[17];
  ff cos_tab[17];
};

// ln 2 and 2 pi as float pairs.
FF_HD ff ff_ln2() { return {0.693147182464599609375f, -1.904654323148236e-09f}; }
FF_HD ff ff_2pi() { return {6.283185482025146484375f, -1.7484555314695172e-07f}; }
FF_HD ff ff_log2e() { return {1.44269502162933349609375f, 1.925963033500011e-08f}; }

// 1/6 as a float pair.
FF_HD ff ff_sixth() { return {0.16666667163372040f, -4.967053879312289e-09f}; }

// e^z - 1 for |z| <= ln2/64 (about 0.0109): z + z^2/2 + z^3/6 in float-float
// plus z^4 (1/24 + z/120 + z^2/720 + z^3/5040) in float (|term| < 6e-10, so
// its rounding stays below 1e-16 relative to the result).
FF_HD ff ff_expm1_small(ff z) {
  const float zh = z.hi;
  const ff z2 = ff_mul(z, z);
  const ff z3 = ff_mul(z2, z);
  const float z4 = z2.hi * z2.hi;
  const float t = z4 * (1.0f / 24.0f + zh * (1.0f / 120.0f + zh * (1.0f / 720.0f + zh * (1.0f / 5040.0f))));
  ff p = ff_add(z, ff_ldexp(z2, -1));
  p = ff_add(p, ff_mul(z3, ff_sixth()));
  return ff_add_f(p, t);
}

// 2^y. y = n + j/32 + s with integer n, j in [-16, 16], |s| <= 1/64;
// 2^s = 1 + expm1(s ln 2).
FF_HD ff ff_exp2(ff y, const FFTables& T) {
  if (y.hi < -150.0f) return {0.0f, 0.0f};
  if (y.hi > 127.0f) return {INFINITY, 0.0f};
  const float n = rintf(y.hi);
  ff r = ff_add_f(y, -n);
  const float j = rintf(r.hi * 32.0f);
  r = ff_add_f(r, -j * (1.0f / 32.0f));
  const ff z = ff_mul(r, ff_ln2());
  const ff e = ff_add_f(ff_expm1_small(z), 1.0f);
  const ff m = ff_mul(e, T.exp2_tab[(int)j + 16]);
  return ff_ldexp(m, (int)n);
}

// log2 x for x > 0: y0 = log2f(x.hi), then one Newton step on 2^y:
// d = x 2^-y0 - 1, log2 x = y0 + (d - d^2/2 + d^3/3) / ln 2.
FF_HD ff ff_log2(ff x, const FFTables& T) {
  const float y0 = log2f(x.hi);
  const ff p = ff_exp2(ff_make(-y0), T);
  const ff d = ff_add_f(ff_mul(x, p), -1.0f);
  const float dh = d.hi;
  const ff corr = ff_add_f(d, dh * dh * (-0.5f + dh * (1.0f / 3.0f)));
  return ff_add_f(ff_div(corr, ff_ln2()), y0);
}

// x^a for x in [0, 1] (0 at x <= 0).
FF_HD ff ff_pow01(ff x, ff a, const FFTables& T) {
  if (!(x.hi > 0.0f)) return {0.0f, 0.0f};
  if (x.hi >= 1.0f && x.lo >= 0.0f) return {1.0f, 0.0f};
  return ff_exp2(ff_mul(a, ff_log2(x, T)), T);
}

// e^x - 1 with full relative accuracy near 0: for |x| < 1/4 the argument is
// halved 5 times, the series is summed, and expm1(2y) = E (E + 2) undoes the
// halvings; larger |x| use 2^(x log2 e) - 1.
FF_HD ff ff_expm1(ff x, const FFTables& T) {
  if (fabsf(x.hi) >= 0.25f) return ff_add_f(ff_exp2(ff_mul(x, ff_log2e()), T), -1.0f);
  ff e = ff_expm1_small(ff_ldexp(x, -5));
#pragma unroll
  for (int i = 0; i < 5; ++i) e = ff_mul(e, ff_add_f(e, 2.0f));
  return e;
}

// sin(2 pi p) for p in [0, 1): quadrant q = rint(4p), then m/128 steps from a
// table and a short series for the remainder angle a = 2 pi s, |s| <= 1/256.
FF_HD ff ff_sin2pi(ff p, const FFTables& T) {
  const float q = rintf(p.hi * 4.0f);
  ff r = ff_add_f(p, -q * 0.25f);              // r in [-1/8, 1/8]
  const float m = rintf(r.hi * 128.0f);         // m in [-16, 16]
  const ff s = ff_add_f(r, -m * (1.0f / 128.0f));
  const ff a = ff_mul(s, ff_2pi());
  const ff a2 = ff_mul(a, a);
  const float ah2 = a2.hi;
  // sin a = a - a^3/6 + a^5/120 - a^7/5040; cos a = 1 - a^2/2 + a^4/24 - a^6/720
  // (a^3/6 in float-float; the higher terms are below 1e-10 and stay in float)
  const ff a3_6 = ff_mul(ff_mul(a2, a), ff_sixth());
  const ff sin_a = ff_add_f(ff_sub(a, a3_6), a.hi * ah2 * ah2 * (1.0f / 120.0f - ah2 * (1.0f / 5040.0f)));
  const ff cos_a = ff_add_f(ff_add_f(ff_ldexp(ff_neg(a2), -1), ah2 * ah2 * (1.0f / 24.0f - ah2 * (1.0f / 720.0f))), 1.0f);
  const int mi = (int)fabsf(m);
  const float sg = m < 0.0f ? -1.0f : 1.0f;
  const ff sm = {sg * T.sin_tab[mi].hi, sg * T.sin_tab[mi].lo};  // sin(2 pi m/128), odd
  const ff cm = T.cos_tab[mi];                                    // cos, even
  // sin(x) and cos(x) of x = 2 pi r
  const ff sx = ff_add(ff_mul(sm, cos_a), ff_mul(cm, sin_a));
  const ff cx = ff_sub(ff_mul(cm, cos_a), ff_mul(sm, sin_a));
  const int qi = ((int)q) & 3;
  if (qi == 0) return sx;
  if (qi == 1) return cx;
  if (qi == 2) return ff_neg(sx);
  return ff_neg(cx);
}

// Fills the tables from FP64 values (host or device).
FF_HD void ff_tables_fill_entry(FFTables& T, int i) {
  if (i < 33) T.exp2_tab[i] = ff_from_double(exp2((double)(i - 16) / 32.0));
  if (i < 17) {
    const double ang = 6.283185307179586476925 * (double)i / 128.0;
    T.sin_tab[i] = ff_from_double(sin(ang));
    T.cos_tab[i] = ff_from_double(cos(ang));
  }
}

}  // namespace synth
