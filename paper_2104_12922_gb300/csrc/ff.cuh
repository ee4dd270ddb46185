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
#include <stdint.h>
#include <string.h>

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

// a + b with one TwoSum on the high parts and the low parts added in float
// (the "sloppy" addition of Hida, Li and Bailey): error below about
// 2^-47 (|a| + |b|). A second TwoSum on the low parts would bound it by
// 2^-47 |a + b| instead; no sum of the control chain needs that (the one
// with the largest cancellation, the pitch difference of neighbouring
// control points, then carries an absolute error of some 1e-12 semitones,
// 1e-13 cycles of phase per interval), and this form takes 11 instead of
// 20 instructions.
FF_HD ff ff_add(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
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

// Bit-level helpers (host and device).
FF_HD float ff_bits_to_float(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f;
  memcpy(&f, &b, sizeof f);
  return f;
#endif
}
FF_HD uint32_t ff_float_to_bits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  uint32_t b;
  memcpy(&b, &f, sizeof b);
  return b;
#endif
}
// 2^n for an integer n in [-126, 127], built from its exponent bits.
FF_HD float ff_exp2i(int n) { return ff_bits_to_float((uint32_t)(n + 127) << 23); }
FF_HD ff ff_scale2i(ff a, int n) {
  if (n >= -126 && n <= 127) {
    const float s = ff_exp2i(n);
    return {a.hi * s, a.lo * s};
  }
  return {ldexpf(a.hi, n), ldexpf(a.lo, n)};
}
// Scale by a power of two (exact barring under/overflow): a product by the
// constant 2^e for the small exponents the control chain uses.
FF_HD ff ff_ldexp(ff a, int e) { return ff_scale2i(a, e); }

// Tables for argument reduction. They are computed on the host from FP64
// values (ff_tables_fill) and handed to the kernels with the configuration:
//  e2[j + 128]   = 2^(j/256),      j = -128..128
//  e2m1[j + 128] = 2^(j/256) - 1,  j = -128..128 (full relative accuracy)
//  lg_r[j]       = the float nearest 1 / (1 + j/128), j = 0..128
//  lg_l[j]       = -log2(lg_r[j])
//  sin_tab[m] = sin(2 pi m / 128), cos_tab[m] = cos(2 pi m / 128), m = 0..16
struct FFTables {
  ff e2[257];
  ff e2m1[257];
  ff lg_l[129];
  float lg_r[129];
  float pad_;
  ff sin_tab[17];
  ff cos_tab[17];
};

// ln 2, 2 pi, log2 e, 1/6 and ln2/256 as float pairs.
FF_HD ff ff_ln2() { return {0.693147182464599609375f, -1.904654323148236e-09f}; }
FF_HD ff ff_2pi() { return {6.283185482025146484375f, -1.7484555314695172e-07f}; }
FF_HD ff ff_log2e() { return {1.44269502162933349609375f, 1.925963033500011e-08f}; }
FF_HD ff ff_sixth() { return {0.16666667163372040f, -4.967053879312289e-09f}; }
FF_HD ff ff_ln2_256() { return {0.0027076061815023422f, -7.440055516116928e-12f}; }

// e^z - 1 for |z| <= ln2/512 (about 1.354e-3): z + z^2/2 + z^3/6 + z^4/24
// + z^5/120. z^2 is split exactly (TwoProd); the terms from z^3 on are below
// 4.2e-10 and summed in float (error below 3e-17).
FF_HD ff ff_expm1_tiny(ff z) {
  const float zh = z.hi;
  const ff sq = two_prod(zh, zh);
  const float half = 0.5f * sq.hi;
  const float rest = fmaf(0.5f, sq.lo, zh * z.lo) +
                     sq.hi * zh * (1.0f / 6.0f + zh * (1.0f / 24.0f + zh * (1.0f / 120.0f)));
  const ff s = two_sum(zh, half);
  return quick_two_sum(s.hi, s.lo + (z.lo + rest));
}

// 2^y. y = n + j/256 + s with integers n, j (|j| <= 128) and |s| <= 1/512:
// 2^y = 2^n 2^(j/256) (1 + expm1(s ln 2)).
FF_HD ff ff_exp2(ff y, const FFTables& T) {
  if (y.hi != y.hi) return y;
  if (y.hi < -126.0f) return {0.0f, 0.0f};
  if (y.hi > 127.0f) return {INFINITY, 0.0f};
  const float N = rintf(y.hi * 256.0f);
  const float n = rintf(N * (1.0f / 256.0f));
  const int j = (int)fmaf(-256.0f, n, N);
  const ff s = two_sum(fmaf(N, -1.0f / 256.0f, y.hi), y.lo);  // the fmaf is exact
  const ff p = ff_expm1_tiny(ff_mul(s, ff_ln2()));
  ff one_p = quick_two_sum(1.0f, p.hi);
  one_p = quick_two_sum(one_p.hi, one_p.lo + p.lo);
  return ff_scale2i(ff_mul(T.e2[j + 128], one_p), (int)n);
}

// e^x - 1 with full relative accuracy: the series for |x| < 1.3e-3; else
// x = N ln2/256 + z (Cody-Waite with a float-float ln2/256), N = 256 n + j,
// and e^x - 1 = (2^(j/256) - 1) + 2^(j/256) expm1(z) when n = 0 (no
// cancellation: both terms come from tables or the series), or
// 2^n 2^(j/256) (1 + expm1(z)) - 1 otherwise (|result| >= 1/2).
FF_HD ff ff_expm1(ff x, const FFTables& T) {
  if (fabsf(x.hi) < 1.3e-3f) return ff_expm1_tiny(x);
  if (x.hi > 88.0f) return {INFINITY, 0.0f};
  if (x.hi < -88.0f) return {-1.0f, 0.0f};
  const float N = rintf(x.hi * (256.0f * 1.44269504088896341f));
  const float n = rintf(N * (1.0f / 256.0f));
  const int j = (int)fmaf(-256.0f, n, N);
  const ff z = ff_sub(x, ff_mul_f(ff_ln2_256(), N));
  const ff p = ff_expm1_tiny(z);
  if (n == 0.0f) return ff_add(T.e2m1[j + 128], ff_mul(T.e2[j + 128], p));
  ff one_p = quick_two_sum(1.0f, p.hi);
  one_p = quick_two_sum(one_p.hi, one_p.lo + p.lo);
  return ff_add_f(ff_scale2i(ff_mul(T.e2[j + 128], one_p), (int)n), -1.0f);
}

// log2 x for x > 0: x = 2^e m with m in [1, 2); m lg_r[j] = 1 + d with
// j = rint(128 (m - 1)) and |d| <= 2^-8; log2 x = e + lg_l[j] + ln(1 + d) log2 e
// with ln(1 + d) = d - d^2/2 + d^3/3 - ... - d^6/6 (d^2 split exactly).
FF_HD ff ff_log2(ff x, const FFTables& T) {
  float xh = x.hi, xl = x.lo;
  int e_adj = 0;
  if (xh < 0x1p-100f) {
    xh *= 0x1p100f;
    xl *= 0x1p100f;
    e_adj = -100;
  }
  const uint32_t b = ff_float_to_bits(xh);
  const int e = (int)((b >> 23) & 0xffu) - 127;
  const float mh = ff_bits_to_float((b & 0x7fffffu) | 0x3f800000u);
  const float ml = xl * ff_exp2i(-e);
  const int j = (int)rintf((mh - 1.0f) * 128.0f);
  const float r = T.lg_r[j];
  const ff pr = two_prod(mh, r);
  const ff d = two_sum(pr.hi - 1.0f, fmaf(ml, r, pr.lo));  // pr.hi - 1 is exact
  const float dh = d.hi;
  const ff sq = two_prod(dh, dh);
  const float rest =
      fmaf(-0.5f, sq.lo, -dh * d.lo) +
      sq.hi * dh * (1.0f / 3.0f - dh * (0.25f - dh * (0.2f - dh * (1.0f / 6.0f))));
  const ff s = two_sum(dh, -0.5f * sq.hi);
  const ff lnp = quick_two_sum(s.hi, s.lo + (d.lo + rest));
  return ff_add_f(ff_add(T.lg_l[j], ff_mul(lnp, ff_log2e())), (float)(e + e_adj));
}

// x^a for x in [0, 1] (0 at x <= 0, 1 at x >= 1).
FF_HD ff ff_pow01(ff x, ff a, const FFTables& T) {
  if (!(x.hi > 0.0f)) return {0.0f, 0.0f};
  if (x.hi >= 1.0f && x.lo >= 0.0f) return {1.0f, 0.0f};
  return ff_exp2(ff_mul(a, ff_log2(x, T)), T);
}

// 1 / b: a float reciprocal refined by one Newton step in float-float.
FF_HD ff ff_rcp(ff b) {
  const float r0 = 1.0f / b.hi;
  const float e = fmaf(-b.hi, r0, 1.0f) - b.lo * r0;  // 1 - b r0, first order
  return quick_two_sum(r0, r0 * e);
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
  // sin(2 pi p) = sin(q pi/2 + x) with x = 2 pi r: sin x, cos x, -sin x,
  // -cos x for q mod 4 = 0..3; sin x = sm cos a + cm sin a and
  // cos x = cm cos a - sm sin a, so one u cos a + w sin a with the pair
  // chosen (and negated) first
  const int qi = ((int)q) & 3;
  const float sgn = qi >= 2 ? -1.0f : 1.0f;
  const ff u = (qi & 1) ? cm : sm, w = (qi & 1) ? ff_neg(sm) : cm;
  return ff_add(ff_mul({sgn * u.hi, sgn * u.lo}, cos_a), ff_mul({sgn * w.hi, sgn * w.lo}, sin_a));
}

// ---------------------------------------------------------------------------
// Phases as 64-bit fixed-point fractions of a cycle: the integer u stands for
// u 2^-64 cycles, so integer addition (mod 2^64) is addition of phases mod 1.
// Running sums in this form are exact, associative and independent of the
// summation order.
// ---------------------------------------------------------------------------
// a mod 1 as a fixed-point phase, for |a| < 2^31 (error below 2^-52 cycles
// once |a| < 2^8).
FF_HD uint64_t ff_to_fix64(ff a) {
  const float x = a.hi * 0x1p32f;  // exact
  const float xi = floorf(x);
  const float rem = fmaf(a.lo, 0x1p64f, (x - xi) * 0x1p32f);  // x - xi is exact
  return ((uint64_t)(int64_t)xi << 32) + (uint64_t)(int64_t)llrintf(rem);
}
// A fixed-point phase as a float-float value in [0, 1) (48 bits kept).
FF_HD ff fix64_to_ff(uint64_t u) {
  const float t1 = (float)(uint32_t)(u >> 40) * 0x1p-24f;
  const float t2 = (float)(uint32_t)((u >> 16) & 0xffffffu) * 0x1p-48f;
  return quick_two_sum(t1, t2);
}
// A fixed-point phase as a float in [0, 1] (the top 32 bits, rounded to
// nearest; 1.0 only for phases within 2^-25 of a whole cycle).
FF_HD float fix64_to_float(uint64_t u) { return (float)(uint32_t)(u >> 32) * 0x1p-32f; }

// Fills the tables from FP64 values (host).
inline void ff_tables_fill(FFTables& T) {
  const double ln2 = 0.69314718055994530942;
  for (int j = -128; j <= 128; ++j) {
    T.e2[j + 128] = ff_from_double(exp2((double)j / 256.0));
    T.e2m1[j + 128] = ff_from_double(expm1((double)j * ln2 / 256.0));
  }
  for (int j = 0; j <= 128; ++j) {
    const float r = (float)(1.0 / (1.0 + (double)j / 128.0));
    T.lg_r[j] = r;
    T.lg_l[j] = ff_from_double(-log2((double)r));
  }
  T.pad_ = 0.0f;
  for (int i = 0; i < 17; ++i) {
    const double ang = 6.283185307179586476925 * (double)i / 128.0;
    T.sin_tab[i] = ff_from_double(sin(ang));
    T.cos_tab[i] = ff_from_double(cos(ang));
  }
}

}  // namespace synth
