// control_ff.cuh -- the Voice's control-rate chain in float-float arithmetic.
//
// Everything that feeds a VCO's pitch -- the 6 ADSRs (Sec. 3.1; LFO rate and
// amplitude envelopes, Sec. 3.2), the LFO shapes, the modulation mixer, the
// pitch in midi and the phase advanced over each control interval -- is
// computed in float-float (about 48 bits), because a pitch error that holds
// over many intervals integrates into phase drift: at 4 s and 10 kHz a
// relative frequency error of 1e-8 is already 4e-4 cycles. Running sums of
// phases across intervals are 64-bit fixed point (ff.cuh).
#pragma once

#include "ff.cuh"
#include "render_common.cuh"
#include "voice_device.cuh"

namespace synth {

// Per-voice constants of the control chain, derived once per tile from the
// human-range parameters y (float-float).
struct VoiceFF {
  ff a[6], dc[6], s[6], r[6], alpha[6];
  ff inv_a[6], inv_dc[6], inv_r[6];
  ff level_d[6];      // gate-on level at note-off
  ff dur;             // note-on duration d
  ff lfo_freq[2], lfo_depth[2];
  ff lfo_w[2][4];     // sine, triangle, saw (saw minus reverse saw), square weights over their sum
  int lfo_on[2];      // the shape weights sum to at least 1e-12
  ff mod_w[4][5];     // modulation weight [source][destination]
  ff inv_norm[5];     // 1 / max(1, column sum of modulation weights)
  ff pitch_base[2];   // midi f0 + tune, per VCO
  ff depth[2];        // pitch modulation depth (semitones), per VCO
  ff pitch_w[2][4];   // depth_o w[s][d_o] / norm[d_o]: VCO o pitch = base + sum_s pitch_w src_s
  float amp_w[3][4];  // w[s][d] / norm[d] for the sine, square-saw and noise amplitudes
};

// Copies the argument-reduction tables (a kernel parameter) into shared
// memory; every thread of the block takes part, the caller synchronizes.
__device__ __forceinline__ void load_tables(FFTables& dst, const FFTables& src) {
  static_assert(sizeof(FFTables) % 16 == 0, "tables copy as 16-byte vectors");
  const float4* a = reinterpret_cast<const float4*>(&src);
  float4* b = reinterpret_cast<float4*>(&dst);
  const int n = (int)(sizeof(FFTables) / 16);
  const int nt = blockDim.x * blockDim.y * blockDim.z;
  for (int i = threadIdx.x; i < n; i += nt) b[i] = a[i];
}

// Sec. 3.1 ADSR at time t: the section is chosen first, then one x^alpha.
// Section boundaries are continuous, so a comparison that rounds the other
// way at an exact tie gives the same value.
__device__ __forceinline__ ff adsr_ff(ff t, int i, const VoiceFF& V, const FFTables& T) {
  ff base, scale, x;
  if (ff_lt(t, V.dur)) {
    if (ff_lt(t, V.a[i])) {
      base = ff_make(0.f); scale = ff_make(1.f); x = ff_mul(t, V.inv_a[i]);
    } else {
      const ff ta = ff_sub(t, V.a[i]);
      if (ff_lt(ta, V.dc[i])) {
        base = ff_make(1.f); scale = ff_sub(V.s[i], ff_make(1.f)); x = ff_mul(ta, V.inv_dc[i]);
      } else {
        return V.s[i];
      }
    }
  } else {
    const ff tau = ff_sub(t, V.dur);
    if (!ff_lt(tau, V.r[i])) return ff_make(0.f);
    base = V.level_d[i]; scale = ff_neg(V.level_d[i]); x = ff_mul(tau, V.inv_r[i]);
  }
  return ff_add(base, ff_mul(scale, ff_pow01(x, V.alpha[i], T)));
}

// Gate-on level at note-off d (attack, decay or sustain value at t = d).
__device__ __forceinline__ ff gate_level_ff(int i, const VoiceFF& V, const FFTables& T) {
  const ff t = V.dur;
  if (ff_lt(t, V.a[i])) return ff_pow01(ff_mul(t, V.inv_a[i]), V.alpha[i], T);
  const ff ta = ff_sub(t, V.a[i]);
  if (ff_lt(ta, V.dc[i]))
    return ff_add(ff_make(1.f), ff_mul(ff_sub(V.s[i], ff_make(1.f)),
                                       ff_pow01(ff_mul(ta, V.inv_dc[i]), V.alpha[i], T)));
  return V.s[i];
}

// Fills VoiceFF from y (float-float). `part` selects which slice this thread
// fills so that the work spreads over several threads; call with part = 0..15.
__device__ inline void voice_ff_fill(VoiceFF& V, const ff* y, int part) {
  if (part < 6) {
    const int i = part;
    const ff* q = y + kAdsr + 5 * i;
    V.a[i] = q[0];
    V.dc[i] = q[1];
    V.s[i] = q[2];
    V.r[i] = q[3];
    V.alpha[i] = q[4];
    V.inv_a[i] = ff_rcp(q[0]);
    V.inv_dc[i] = ff_rcp(q[1]);
    V.inv_r[i] = ff_rcp(q[3]);
  } else if (part < 8) {
    const int l = part - 6;
    const ff* q = y + kLfo + 8 * l;
    V.lfo_freq[l] = q[0];
    V.lfo_depth[l] = q[1];
    ff ws = q[3];
    for (int s = 1; s < 5; ++s) ws = ff_add(ws, q[3 + s]);
    V.lfo_on[l] = ws.hi >= 1e-12f;
    const ff inv = V.lfo_on[l] ? ff_rcp(ws) : ff_make(0.f);
    V.lfo_w[l][0] = ff_mul(q[3], inv);
    V.lfo_w[l][1] = ff_mul(q[4], inv);
    V.lfo_w[l][2] = ff_mul(ff_sub(q[5], q[6]), inv);
    V.lfo_w[l][3] = ff_mul(q[7], inv);
  } else if (part < 13) {
    const int j = part - 8;
    ff ws = y[kMod + j];
    V.mod_w[0][j] = ws;
    for (int i = 1; i < 4; ++i) {
      V.mod_w[i][j] = y[kMod + 5 * i + j];
      ws = ff_add(ws, y[kMod + 5 * i + j]);
    }
    V.inv_norm[j] = ff_lt(ws, ff_make(1.f)) ? ff_make(1.f) : ff_rcp(ws);
    if (j == 1 || j == 3 || j == 4) {
      const int k = j == 1 ? 0 : (j == 3 ? 1 : 2);
      for (int i = 0; i < 4; ++i)
        V.amp_w[k][i] = ff_to_float(ff_mul(y[kMod + 5 * i + j], V.inv_norm[j]));
    }
  } else if (part < 15) {
    const int o = part - 13;
    const int base = o == 0 ? kSine : kSqr;
    const int d = o == 0 ? 0 : 2;
    V.pitch_base[o] = ff_add(y[kMidi], y[base]);
    V.depth[o] = y[base + 1];
    ff ws = y[kMod + d];
    for (int i = 1; i < 4; ++i) ws = ff_add(ws, y[kMod + 5 * i + d]);
    const ff scale = ff_lt(ws, ff_make(1.f)) ? y[base + 1] : ff_mul(y[base + 1], ff_rcp(ws));
    for (int i = 0; i < 4; ++i) V.pitch_w[o][i] = ff_mul(y[kMod + 5 * i + d], scale);
  } else {
    V.dur = y[kDuration];
  }
}

// LFO output at phase p in [0,1): shapes sin 2 pi p, triangle 1 - 4|p - 1/2|,
// saw 2p - 1, reverse saw 1 - 2p, square sign(1/2 - p) (+1 at p < 1/2),
// mixed by weight over the weight sum, times the amplitude envelope.
__device__ __forceinline__ ff lfo_ff(ff p, int l, ff env_amp, const VoiceFF& V, const FFTables& T) {
  if (!V.lfo_on[l]) return ff_make(0.f);
  const ff sn = ff_sin2pi(p, T);
  const ff saw = ff_add_f(ff_ldexp(p, 1), -1.f);
  const ff tri = ff_add_f(ff_ldexp(ff_neg(ff_abs(ff_add_f(p, -0.5f))), 2), 1.f);
  const float sqr = ff_lt(p, ff_make(0.5f)) ? 1.f : -1.f;
  ff acc = ff_mul(V.lfo_w[l][0], sn);
  acc = ff_add(acc, ff_mul(V.lfo_w[l][1], tri));
  acc = ff_add(acc, ff_mul(V.lfo_w[l][2], saw));
  acc = ff_add(acc, ff_mul_f(V.lfo_w[l][3], sqr));
  return ff_mul(env_amp, acc);
}

// Per-VCO phase increment (cycles per sample) at pitch m (midi), uncapped:
// 440 * 2^((m - 69)/12) / SR = 2^((m - 69)/12 + log2(440/SR)).
__device__ __forceinline__ ff inc_at_ff(ff m, ff log2_440_over_sr, const FFTables& T) {
  const ff twelfth = {0.0833333358168602f, -2.483526865641276e-09f};
  return ff_exp2(ff_add(ff_mul(ff_add_f(m, -69.f), twelfth), log2_440_over_sr), T);
}

// Sum of k geometric increments starting at c with ratio e^x:
// c expm1(k x) / expm1(x), or c k when x == 0.
__device__ __forceinline__ ff geo_sum_ff(ff c, ff x, int k, const FFTables& T) {
  if (k <= 0) return ff_make(0.f);
  if (x.hi == 0.f) return ff_mul_f(c, (float)k);
  return ff_mul(c, ff_mul(ff_expm1(ff_mul_f(x, (float)k), T), ff_rcp(ff_expm1(x, T))));
}

// The description (SegVco) of how a VCO's phase advances over one control
// interval of Rk samples, from the pitch at its two control points; returns
// the phase advanced (cycles) and, in *inc_first, the increment of the
// interval's first sample (cycles per sample, capped at 1/2). Sample j of the
// interval has pitch m_a + (j / R)(m_b - m_a), capped at the Nyquist pitch.
__device__ inline ff vco_interval_ff(ff m_a, ff m_b, float R, int Rk, ff inv_R, ff ln2_12R,
                                     ff m_nyq, ff log2_440_over_sr, const FFTables& T,
                                     SegVco* out, float* inc_first) {
  const ff dm = ff_sub(m_b, m_a);
  const ff x = ff_mul(dm, ln2_12R);
  auto capped = [&](int j) {
    return ff_gt(ff_add(m_a, ff_mul(dm, ff_mul_f(inv_R, (float)j))), m_nyq);
  };
  // The pitch is linear between the two points: when both lie clearly on one
  // side of the cap, so does every sample of the interval.
  bool c_first, c_last;
  const float top = fmaxf(m_a.hi, m_b.hi), bot = fminf(m_a.hi, m_b.hi);
  if (top < m_nyq.hi - 1e-3f) {
    c_first = false; c_last = false;
  } else if (bot > m_nyq.hi + 1e-3f) {
    c_first = true; c_last = true;
  } else {
    c_first = capped(0); c_last = capped(Rk - 1);
  }
  // Cases: no cap (one geometric piece A over Rk samples), all capped (one
  // linear piece at 1/2), rising through the cap at jc (geometric A, then
  // 1/2), falling out of it at jc (1/2, then geometric B). Each has at most
  // one geometric piece: its first pitch m_g and length k_g.
  int jc = Rk;
  if (c_first != c_last) {
    const float js = (m_nyq.hi - m_a.hi) * R / dm.hi;
    jc = (int)fminf(fmaxf(ceilf(js), 0.f), (float)(Rk - 1));
    if (!c_first) {  // rising: first capped sample
      while (jc > 0 && capped(jc - 1)) --jc;
      while (jc < Rk && !capped(jc)) ++jc;
    } else {  // falling: first uncapped sample
      while (jc > 0 && !capped(jc - 1)) --jc;
      while (jc < Rk && capped(jc)) ++jc;
    }
  } else if (c_first) {
    jc = 0;
  }
  const ff half = ff_make(0.5f);
  const bool geo = !(c_first && c_last);
  const int k_g = c_first ? Rk - jc : jc;  // samples of the geometric piece
  ff c_g = half, s_g = ff_make(0.5f * (float)k_g);  // all capped: k_g samples at 1/2
  if (geo) {
    const ff m_g = c_first ? ff_add(m_a, ff_mul(dm, ff_mul_f(inv_R, (float)jc))) : m_a;
    c_g = inc_at_ff(m_g, log2_440_over_sr, T);
    s_g = geo_sum_ff(c_g, x, k_g, T);
  }
  const bool xz = x.hi == 0.f;
  ff cA, cB, LB, total;
  bool a_lin, b_lin;
  if (!c_first) {  // A geometric (jc = Rk when never capped), B at 1/2
    cA = c_g; cB = half; LB = s_g; a_lin = xz; b_lin = true;
    total = ff_add_f(s_g, 0.5f * (float)(Rk - jc));
  } else {         // A at 1/2 (jc samples), B geometric (none when all capped)
    cA = half; cB = geo ? c_g : half; LB = ff_make(0.5f * (float)jc); a_lin = true;
    b_lin = geo ? xz : true;
    total = ff_add(LB, s_g);
  }
  if (!c_first && !c_last) LB = ff_make(0.f);
  const float xf = x.hi;
  const bool tiny = fabsf(xf) < 1e-30f;
  // every piece linear: the quad steps (and the geometric constants, which
  // no linear piece reads) are those of x = 0
  const bool all_lin = tiny || (a_lin && b_lin);
  const float e1 = all_lin ? 0.f : expm1f(xf);
  out->cA = cA.hi + cA.lo;
  out->cB = cB.hi + cB.lo;
  out->LB = LB.hi + LB.lo;
  out->x = xf;
  out->q2 = 2.f + e1;                 // 1 + r, r = 1 + e1
  out->q3 = fmaf(e1, e1 + 3.f, 3.f);  // 1 + r + r^2 = 3 + 3 e1 + e1^2
  out->invE = all_lin ? 0.f : 1.0f / e1;
  out->ih = all_lin ? 1.f : xf * out->invE;
  out->q4 = fmaf(e1, fmaf(e1, e1 + 4.f, 6.f), 4.f);  // (r^4 - 1) / (r - 1) = 4 + 6 e1 + 4 e1^2 + e1^3
  out->r4m1 = e1 * out->q4;
  out->jc_flags = jc | ((a_lin || tiny) ? 1 << 16 : 0) | ((b_lin || tiny) ? 1 << 17 : 0) |
                  (c_first ? 1 << 18 : 0) | (c_last ? 1 << 19 : 0) | (all_lin ? 1 << 20 : 0);
  *inc_first = out->cA;
  return total;
}

// Sec. 3.3 range map in float-float from a normalized parameter u in [0, 1]:
// y = base + scale a^c, with a = u (scale = hi - lo, base = lo) or, for a
// symmetric parameter, a = |2u - 1| signed by 2u - 1 (scale = (hi - lo)/2,
// base = lo + scale). Curves 1, 2, 3 use exact products.
__device__ inline ff range_map_ff(float u, ff base, ff scale, ff curve, int code, int sym,
                                  const FFTables& T) {
  ff a = ff_make(u);
  bool neg = false;
  if (sym) {
    a = two_sum(2.f * u, -1.f);  // exact
    neg = a.hi < 0.f;
    if (neg) a = ff_neg(a);
  }
  ff pw;
  if (code == 1) pw = a;
  else if (code == 2) pw = ff_mul(a, a);
  else if (code == 3) pw = ff_mul(ff_mul(a, a), a);
  else pw = ff_pow01(a, curve, T);
  if (neg) pw = ff_neg(pw);
  return ff_add(base, ff_mul(scale, pw));
}

}  // namespace synth
