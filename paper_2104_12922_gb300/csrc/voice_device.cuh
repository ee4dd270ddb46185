// voice_device.cuh -- device-side definition of the Voice (sm_103a).
//
// Paper: Turian et al., DAFx 2021. Sec. 3.1 (audio / control / parameter
// modules, 44.1 kHz audio, 441 Hz control), Sec. 3.2 (the Voice: keyboard,
// 2 LFOs, 6 ADSRs -- each LFO owns a rate and an amplitude ADSR -- sine and
// square-saw VCOs, noise, VCAs, modulation and audio mixers; 78 parameters),
// Sec. 3.3 (normalized parameters and the curve/symmetric range map), Sec. 2.1
// (deterministic random numbers, noise included).
//
// The paper gives module names, not formulas. The library's reading of each
// module is stated at its function below.
#pragma once

#include <cmath>

#include <cstdint>

#include "ff.cuh"

namespace synth {

constexpr int kNumParams = 78;
constexpr int kNumFmParams = 30;  // the 4-operator FM voice (fm_voice.cu)

// Parameter slots of the Voice.
enum : int {
  kMidi = 0, kDuration = 1,
  kAdsr = 2,   // 6 ADSRs x {attack s, decay s, sustain, release s, alpha}
  kLfo = 32,   // 2 LFOs x {freq Hz, rate depth Hz, phase0 rad, w_sin, w_tri, w_saw, w_rsaw, w_sqr}
  kMod = 48,   // modulation weight [source i][destination j] at kMod + 5 i + j
  kSine = 68,  // {tune st, depth st, phase0 rad}
  kSqr = 71,   // {tune st, depth st, phase0 rad, shape}
  kMix = 75,   // levels {sine, square-saw, noise}
};
// ADSR a: 0, 1 free sources; 2 + 2l = LFO l rate, 3 + 2l = LFO l amplitude.
// Sources: ADSR0, ADSR1, LFO0, LFO1. Destinations: 0 sine pitch, 1 sine
// amplitude, 2 square-saw pitch, 3 square-saw amplitude, 4 noise amplitude.

constexpr double kLfoMaxHz = 20.0;
constexpr double kBrightnessMax = 50.0;
constexpr uint32_t kStreamParam = 0;
constexpr uint32_t kStreamNoise = 1;

// Everything a render kernel needs about the configuration (passed by value
// as a __grid_constant__ kernel parameter). The float-float fields and the
// tables are derived on the host (voice_const_derive), so that the kernels
// need no FP64 arithmetic for them.
struct VoiceConst {
  double lo[kNumParams], hi[kNumParams], curve[kNumParams];
  int32_t sym[kNumParams];
  double sample_rate, control_rate;
  double m_nyq;      // Nyquist pitch in midi, 69 + 12 log2(SR / 2 / 440)
  int64_t n_samples; // N
  int32_t R;         // samples per control interval (general_r: ceil(a / b))
  int32_t K;         // control intervals holding samples, floor((N - 1) b / a) + 1
  int32_t carry_fp32;
  // Sec. 3.3 map as y = map_base + map_scale a^curve (range_map_ff)
  ff map_base[kNumParams], map_scale[kNumParams], map_curve[kNumParams];
  int32_t map_code[kNumParams];  // 1, 2, 3 for those integer curves, else 0
  ff inv_cr;            // 1 / control rate
  ff inv_R;             // 1 / R = b / a
  ff ln2_12R;           // ln 2 / (12 R)
  ff inv_a;             // 1 / a
  float r_f;            // R
  ff m_nyq_ff;          // m_nyq
  ff log2_440_over_sr;  // log2(440 / SR)
  ff inv_2pi;           // 1 / (2 pi)
  alignas(16) FFTables T;
  // Samples per control interval R = SR / CR = rate_a / rate_b in lowest
  // terms: an integer R, or, for a fractional R, integer rates in Hz. Sample n
  // lies in interval k = floor(n b / a) at the fraction (n b - k a) / a; the
  // interval starts at sample ceil(k a / b).
  int64_t rate_a, rate_b;
  int32_t general_r; // 0: R is an integer multiple of 4 (quads align with intervals)
};

// The render geometry of sample rate sr, control rate cr and duration
// `seconds` (host): n_samples, rate_a / rate_b, general_r, R and K. Returns
// false for what the renders do not support: N not an integer or >= 2^31, a
// fractional R from rates that are not integers in Hz, R < 4 (a 4-sample
// quad then spans at most two intervals), or R > 65532 (an interval's sample
// index fits 16 bits).
inline bool voice_geometry(VoiceConst& vc, double sr, double cr, double seconds) {
  const double n = seconds * sr;
  const long long N = std::llround(n);
  if (std::fabs(n - (double)N) > 1e-6 || N < 1 || N > (1LL << 31)) return false;
  const double r = sr / cr;
  const long long ri = std::llround(r);
  long long a, b;
  if (ri >= 1 && std::fabs(r - (double)ri) <= 1e-9) {
    a = ri;
    b = 1;
  } else {
    const long long si = std::llround(sr), ci = std::llround(cr);
    if (std::fabs(sr - (double)si) > 1e-9 || std::fabs(cr - (double)ci) > 1e-9) return false;
    long long x = si, y = ci;
    while (y != 0) {
      const long long t = x % y;
      x = y;
      y = t;
    }
    a = si / x;
    b = ci / x;
  }
  if (a < 4 * b || a > 65532 * b || a >= (1LL << 31) || b >= (1LL << 31)) return false;
  vc.n_samples = N;
  vc.rate_a = a;
  vc.rate_b = b;
  vc.general_r = (b != 1 || (a & 3) != 0) ? 1 : 0;
  vc.R = (int32_t)((a + b - 1) / b);
  const long long K = (N - 1) * b / a + 1;
  if (K >= (1LL << 31)) return false;
  vc.K = (int32_t)K;
  return true;
}

// Fills the derived fields of vc from its FP64 fields (host).
inline void voice_const_derive(VoiceConst& vc) {
  for (int p = 0; p < kNumParams; ++p) {
    const double span = vc.hi[p] - vc.lo[p];
    const double scale = vc.sym[p] ? 0.5 * span : span;
    vc.map_base[p] = ff_from_double(vc.sym[p] ? vc.lo[p] + scale : vc.lo[p]);
    vc.map_scale[p] = ff_from_double(scale);
    vc.map_curve[p] = ff_from_double(vc.curve[p]);
    const double c = vc.curve[p];
    vc.map_code[p] = c == 1.0 ? 1 : (c == 2.0 ? 2 : (c == 3.0 ? 3 : 0));
  }
  vc.inv_cr = ff_from_double(1.0 / vc.control_rate);
  vc.inv_R = ff_from_double((double)vc.rate_b / (double)vc.rate_a);
  vc.ln2_12R = ff_from_double(0.69314718055994530942 * (double)vc.rate_b / (12.0 * (double)vc.rate_a));
  vc.inv_a = ff_from_double(1.0 / (double)vc.rate_a);
  vc.r_f = (float)((double)vc.rate_a / (double)vc.rate_b);
  vc.m_nyq_ff = ff_from_double(vc.m_nyq);
  vc.log2_440_over_sr = ff_from_double(log2(440.0 / vc.sample_rate));
  vc.inv_2pi = ff_from_double(0.15915494309189533577);
  ff_tables_fill(vc.T);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two
// 32x32->64 products on counter words 0 and 2, permuted and xor-ed with the
// remaining words and the key; the key advances by the Weyl increments.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// The same generator with each 32 x 32 -> 64-bit product as one wide
// multiply (bit-identical). It issues more slowly than the split high and low
// products, but holds fewer registers across the rounds: the peak-normalising
// render, whose audio loop otherwise spills, runs faster with it.
__device__ __forceinline__ uint4 philox4x32_10_wide(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k.x, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k.y,
                   (uint32_t)p0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// Top 24 bits of a draw, times 2^-24: exact in float, in [0,1).
__device__ __forceinline__ float u01f(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

// ---------------------------------------------------------------------------
// Sec. 3.3 range map, FP64. Integer curves 1, 2, 3 use multiplications.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double curve_pow(double x, double c) {
  if (c == 1.0) return x;
  if (c == 2.0) return x * x;
  if (c == 3.0) return x * x * x;
  return x <= 0.0 ? 0.0 : pow(x, c);
}

__device__ __forceinline__ double range_map(double u, double lo, double hi, double c, int sym) {
  if (!sym) return lo + (hi - lo) * curve_pow(u, c);
  const double s = 2.0 * u - 1.0;
  const double a = curve_pow(fabs(s), c);
  return lo + (hi - lo) * (1.0 + (s < 0.0 ? -a : a)) * 0.5;
}

// x^alpha for x in [0, 1], 0 at x <= 0.
__device__ __forceinline__ double pow01(double x, double alpha) {
  return x <= 0.0 ? 0.0 : pow(x, alpha);
}

// Sec. 3.1 ADSR, gate-on part: attack (t/a)^alpha while t < a; decay
// 1 - (1 - s) ((t - a)/dc)^alpha while t < a + dc; sustain s after.
__device__ __forceinline__ double adsr_gate_on(double t, double a, double dc, double s, double al) {
  if (t < a) return pow01(t / a, al);
  if (t < a + dc) return 1.0 - (1.0 - s) * pow01((t - a) / dc, al);
  return s;
}

// Full envelope with note-off at d: release from L = gate_on(d) as
// L (1 - ((t - d)/r)^alpha) while t - d < r, then 0. One pow per call: the
// section is chosen first, then a single x^alpha is evaluated.
__device__ __forceinline__ double adsr_eval(double t, const double* q, double d, double level_at_d) {
  const double a = q[0], dc = q[1], s = q[2], r = q[3], al = q[4];
  double base, scale, x;
  if (t < d) {
    if (t < a) { base = 0.0; scale = 1.0; x = t / a; }
    else if (t < a + dc) { base = 1.0; scale = -(1.0 - s); x = (t - a) / dc; }
    else { return s; }
  } else {
    const double tau = t - d;
    if (!(tau < r)) return 0.0;
    base = level_at_d; scale = -level_at_d; x = tau / r;
  }
  return base + scale * pow01(x, al);
}

// LFO shapes at phase p in [0,1): sin 2 pi p, triangle 1 - 4|p - 1/2|,
// saw 2p - 1, reverse saw 1 - 2p, square +1 for p < 1/2 else -1; mixed by
// the five weights over their sum (0 when the sum is below 1e-12).
__device__ __forceinline__ double lfo_mix(double p, const double* w, double wsum) {
  if (wsum < 1e-12) return 0.0;
  const double sn = sinpi(2.0 * p);
  const double tri = 1.0 - 4.0 * fabs(p - 0.5);
  const double saw = 2.0 * p - 1.0;
  const double sqr = p < 0.5 ? 1.0 : -1.0;
  return (w[0] * sn + w[1] * tri + w[2] * saw + w[3] * (-saw) + w[4] * sqr) / wsum;
}

__device__ __forceinline__ double frac64(double x) { return x - floor(x); }

}  // namespace synth
