// render_backward.cu -- adjoint of the Voice render: grad_u = (d audio / d u)^T
// grad_audio for the 78 normalized parameters of every voice.
//
// "Stress-tested differentiable modules" are future work in the paper
// (Sec. 7); this is the reverse-mode derivative of the library's own render.
// Where the forward takes a branch (envelope section, clamp, Nyquist cap,
// square LFO) the derivative is that of the branch taken.
//
// Passes (all on the caller's stream, buffers in the caller's workspace):
//  1. forward recomputation of the control rate (control_pipeline.cuh: the
//     plain form's module steps in one kernel, one CTA per voice); its
//     per-interval phase descriptions are the checkpoints from which the
//     audio-rate values are rebuilt;
//  2. audio-rate reverse pass, one warp per control interval: rebuilds every
//     sample, forms d/d(phase) of both VCOs, the amplitude, drive, shape and
//     mixer-gain partials, and the interval's moments for the reverse phase
//     scan (see bwd_samples);
//  3. reverse scan over intervals (FP64): with C_k = sum of d/d(phase) over
//     all samples from interval k on, the pitch adjoint of control point k is
//     (ln 2 / 12) (M1_k + F1_k C_{k+1} + M2_{k-1} + F2_{k-1} C_k);
//  4. control-rate reverse sweep per voice: modulation mixer, LFOs (with a
//     reverse scan of the LFO phase adjoint), ADSRs, range map -> d/du.

#include "control_pipeline.cuh"
#include "internal.h"

namespace synth {

namespace {

constexpr int kBT = 256;
constexpr int kStat = 21;  // per-interval partial sums written by bwd_samples
// stat layout: [0..4] sine T, M1, F1, M2, F2; [5..9] square-saw T, M1, F1, M2, F2;
// [10..12] amp grads to the left point (sine, sq, noise); [13..15] to the right
// point; [16] d/d kappa; [17..19] mixer gains g0, g1, g2; [20] d/d shape.

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

struct BwdLayout {
  size_t stat, gpt, vacc, dtheta, denv, total;
};

BwdLayout bwd_layout(const VoiceConst& vc, int B, size_t base) {
  const size_t P = (size_t)vc.K + 1, K = (size_t)vc.K;
  BwdLayout L;
  size_t o = base;
  auto take = [&](size_t bytes) { size_t at = o; o = al256(o + bytes); return at; };
  L.stat = take(sizeof(float) * B * K * kStat);
  L.gpt = take(sizeof(double) * 2 * B * P * 5);
  L.vacc = take(sizeof(double) * B * 8);
  L.dtheta = take(sizeof(float) * B * 2 * P);
  L.denv = take(sizeof(float) * B * 6 * P);
  L.total = o;
  return L;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// 2. audio-rate reverse pass. Warp w of a block takes control interval k; lane
// l takes samples 4l..4l+3 of it (R <= 128). Four blocks per SM (64
// registers, a small spill) run it faster than three with no spill.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBT, 4) bwd_samples(const __grid_constant__ VoiceConst vc,
                                                   uint64_t seed, uint64_t batch_index, int batch,
                                                   const float* __restrict__ mixc,
                                                   const ff* __restrict__ dest,
                                                   const SegVco* __restrict__ seg,
                                                   const float* __restrict__ kappa,
                                                   const float* __restrict__ grad_audio,
                                                   float* __restrict__ stat, ScratchHeader* hdr) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int v = blockIdx.y;
  const int K = vc.K, P = K + 1, R = vc.R;
  const int k = blockIdx.x * (kBT / 32) + warp;
  if (k >= K) return;
  // the interval's control points k and k + 1, its descriptions and its row
  // of statistics belong to voice v of this batch
  if (!in_bounds(hdr, v, batch) || !in_bounds(hdr, k + 1, P)) return;
  const int64_t N = vc.n_samples;
  // mixer gains and square-saw shape as the control pass stored them (the
  // FP64 quotients rounded to float: no FP64 arithmetic in this kernel)
  const float* mc = mixc + (size_t)v * 5;
  const float g[3] = {mc[0], mc[1], mc[2]};
  const float sigma = mc[3];
  const float ip = 1.f / (1.f + sigma);
  const int dj[3] = {1, 3, 4};
  float a0[3], a1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    a0[c] = ff_to_float(dest[((size_t)v * 5 + dj[c]) * P + k]);
    a1[c] = ff_to_float(dest[((size_t)v * 5 + dj[c]) * P + k + 1]);
  }
  const SegVco s0 = seg[((size_t)v * 2 + 0) * K + k];
  const SegVco s1 = seg[((size_t)v * 2 + 1) * K + k];
  const float kap = kappa[((size_t)v * 2 + 0) * K + k];
  const float itk = kappa[((size_t)v * 2 + 1) * K + k];
  const int64_t rem = N - (int64_t)k * R;
  const int Rk = rem < R ? (int)rem : R;
  const float invR = 1.f / (float)R;
  const uint64_t gv = batch_index * (uint64_t)batch + (uint64_t)v;

  float acc[kStat];
#pragma unroll
  for (int i = 0; i < kStat; ++i) acc[i] = 0.f;
  float dphi[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
  float inc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
  bool capd[2][4] = {{false, false, false, false}, {false, false, false, false}};
  const int j0 = 4 * lane;
  const bool active = j0 < Rk;
  if (active) {
    float ps[4], pq[4];
    vco_quad(s0, j0, ps);
    vco_quad(s1, j0, pq);
    vco_inc_quad(s0, j0, inc[0], capd[0]);
    vco_inc_quad(s1, j0, inc[1], capd[1]);
    const int64_t n0 = (int64_t)k * R + j0;
    const uint4 nz = philox4x32_10(
        make_uint4((uint32_t)gv, (uint32_t)(gv >> 32), (uint32_t)(n0 >> 2), kStreamNoise),
        make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const uint32_t nw[4] = {nz.x, nz.y, nz.z, nz.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int j = j0 + i;
      if (j >= Rk) {
        inc[0][i] = inc[1][i] = 0.f;
        continue;
      }
      const float go = in_bounds(hdr, (long long)v * N + n0 + i, (long long)batch * N)
                           ? grad_audio[(size_t)v * N + n0 + i]
                           : 0.f;
      const float fj = (float)j * invR;
      float A[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) A[c] = fmaf(fj, a1[c] - a0[c], a0[c]);
      // SFU sine, cosine and tanh, as in the forward render
      float xs, xc;
      __sincosf(kTwoPiF * ps[i], &xs, &xc);
      float sn, cs;
      __sincosf(kTwoPiF * pq[i], &sn, &cs);
      const float th = tanh_from_y(kTwoLog2e * kap * sn);
      const float shp = fmaf(sigma, cs, 1.f);
      const float xq = th * itk * shp * ip;
      const float xn = fmaf(2.f, u01f(nw[i]), -1.f);
      const float x[3] = {xs, xq, xn};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float dA = go * g[c] * x[c];
        acc[10 + c] += dA * (1.f - fj);
        acc[13 + c] += dA * fj;
        acc[17 + c] += go * A[c] * x[c];
      }
      dphi[0][i] = go * g[0] * A[0] * kTwoPiF * xc;
      const float sech2 = 1.f - th * th;
      const float dxq_dth = itk * ip * (kap * cs * sech2 * shp - th * sigma * sn);
      dphi[1][i] = go * g[1] * A[1] * kTwoPiF * dxq_dth;
      // d xq / d kappa with d(1/tanh k)/dk = 1 - (1/tanh k)^2
      acc[16] += go * g[1] * A[1] * ip * shp * (sn * sech2 * itk + th * (1.f - itk * itk));
      acc[20] += go * g[1] * A[1] * th * itk * (cs - 1.f) * ip * ip;
    }
  }
  // reverse phase scan inside the interval: LS_j = sum of dphi over samples
  // after j in this interval
#pragma unroll
  for (int o = 0; o < 2; ++o) {
    const float lt = dphi[o][0] + dphi[o][1] + dphi[o][2] + dphi[o][3];
    float suf = lt;  // inclusive suffix over lanes >= lane
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const float t = __shfl_down_sync(0xffffffffu, suf, d);
      if (lane + d < 32) suf += t;
    }
    float after = __shfl_down_sync(0xffffffffu, suf, 1);
    if (lane == 31) after = 0.f;
    float ls = after;  // strict suffix, walking from sample 3 down to 0
    float M1 = 0.f, F1 = 0.f, M2 = 0.f, F2 = 0.f;
#pragma unroll
    for (int i = 3; i >= 0; --i) {
      const int j = j0 + i;
      if (active && j < Rk && !capd[o][i]) {
        const float fj = (float)j * invR;
        const float wl = inc[o][i] * (1.f - fj), wr = inc[o][i] * fj;
        M1 += wl * ls;
        F1 += wl;
        M2 += wr * ls;
        F2 += wr;
      }
      ls += dphi[o][i];
    }
    acc[5 * o + 0] += lt;
    acc[5 * o + 1] += M1;
    acc[5 * o + 2] += F1;
    acc[5 * o + 3] += M2;
    acc[5 * o + 4] += F2;
  }
  // butterfly reduce-scatter of the kStat (<= 32) sums over the warp: at
  // step s a lane keeps half of its slots (the upper half when bit s of its
  // lane index is set) and adds its partner's copy of that half; after 31
  // shuffles lane i holds the warp's total of sum i (instead of 5 shuffles
  // for each of the kStat sums)
  static_assert(kStat <= 32, "one sum per lane");
  float r[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) r[i] = i < kStat ? acc[i] : 0.f;
#pragma unroll
  for (int sh = 16; sh >= 1; sh >>= 1) {
    const bool up = (lane & sh) != 0;
#pragma unroll
    for (int i = 0; i < sh; ++i) {
      const float send = up ? r[i] : r[i + sh];
      const float keep = up ? r[i + sh] : r[i];
      r[i] = keep + __shfl_xor_sync(0xffffffffu, send, sh);
    }
  }
  if (lane < kStat) stat[((size_t)v * K + k) * kStat + lane] = r[0];
}

// ---------------------------------------------------------------------------
// 3. reverse scan over intervals and the per-point pitch / amplitude adjoints.
// One block per voice. gpt[half][v][k] = {dm_sine, dm_sq, dA_sine, dA_sq,
// dA_noise}: half 0 from interval k (point k its left end), half 1 from
// interval k - 1 (its right end); the point's adjoint is their sum.
// vacc[v] = {dphase0_sine, dphase0_sq (cycles), dg0, dg1, dg2, dshape, 0, 0}.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBT) bwd_interval_scan(const __grid_constant__ VoiceConst vc,
                                                         const float* __restrict__ stat,
                                                         const SegVco* __restrict__ seg,
                                                         const float* __restrict__ kappa,
                                                         double* __restrict__ gpt,
                                                         double* __restrict__ vacc,
                                                         ScratchHeader* hdr) {
  __shared__ double warp_tot[2 * (kBT / 32)];
  __shared__ double red[8][kBT / 32];
  const int v = blockIdx.x;
  const int K = vc.K, P = K + 1;
  const double l12 = kLn2 / 12.0;
  double carry0 = 0.0, carry1 = 0.0;
  double part[4] = {0.0, 0.0, 0.0, 0.0};  // dg0, dg1, dg2, dshape
  double* gv = gpt + (size_t)v * P * 5;
  for (int base = 0; base < K; base += kBT) {
    const int idx = K - 1 - (base + (int)threadIdx.x);  // reversed order
    const bool ok = idx >= 0;
    const float* st = stat + ((size_t)v * K + (ok ? idx : 0)) * kStat;
    double t0 = ok ? (double)st[0] : 0.0, t1 = ok ? (double)st[5] : 0.0;
    double e0 = t0, e1 = t1, tot0, tot1;
    block_exclusive_scan2<double, kBT>(e0, e1, warp_tot, tot0, tot1);
    if (ok) {
      // C_{idx+1}: sum of d/d(phase) over all later intervals
      const double c0 = carry0 + e0, c1 = carry1 + e1;
      const double dl0 = l12 * ((double)st[1] + (double)st[2] * c0);
      const double dr0 = l12 * ((double)st[3] + (double)st[4] * c0);
      const double dl1 = l12 * ((double)st[6] + (double)st[7] * c1);
      const double dr1 = l12 * ((double)st[8] + (double)st[9] * c1);
      // square-saw drive kappa_k = min(50, 1 + SR/(8 f_k)): d kappa / d m =
      // -(kappa - 1) ln2/12 while below the bound and the pitch is uncapped
      const SegVco s1 = seg[((size_t)v * 2 + 1) * K + idx];
      const float kap = kappa[((size_t)v * 2 + 0) * K + idx];
      double dk = 0.0;
      if (kap < (float)kBrightnessMax && !((s1.jc_flags >> 18) & 1))
        dk = (double)st[16] * (-(double)(kap - 1.f) * l12);
      // interval idx reaches points idx (left end) and idx + 1 (right end):
      // the left parts go to gv, the right parts to gr, one store each; the
      // consumer adds the two halves of a point
      double* gl = gv + (size_t)idx * 5;
      double* gr = gv + (size_t)P * 5 * gridDim.x + (size_t)(idx + 1) * 5;
      if (in_bounds(hdr, idx + 1, P)) {  // both halves stay in the voice's P points
        gl[0] = dl0;
        gr[0] = dr0;
        gl[1] = dl1 + dk;
        gr[1] = dr1;
        for (int c = 0; c < 3; ++c) {
          gl[2 + c] = (double)st[10 + c];
          gr[2 + c] = (double)st[13 + c];
        }
      }
      for (int c = 0; c < 4; ++c) part[c] += (double)st[17 + c];
    }
    carry0 += tot0;
    carry1 += tot1;
  }
  // per-voice sums of the gain / shape partials
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = 0; c < 4; ++c) {
    const double w = warp_sum_d(part[c]);
    if (lane == 0) red[c][warp] = w;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double* va = vacc + (size_t)v * 8;
    va[0] = carry0;  // sum over every sample: d/d(initial phase, cycles)
    va[1] = carry1;
    for (int c = 0; c < 4; ++c) {
      double s = 0.0;
      for (int w = 0; w < kBT / 32; ++w) s += red[c][w];
      va[2 + c] = s;
    }
    va[6] = va[7] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// 4. control-rate reverse sweep, one block per voice, in FP32: a gradient
// needs a relative accuracy of about 1e-3, not the forward's float-float (the
// forward values it differentiates at are recomputed in float-float and FP64
// and rounded to float here).
// ---------------------------------------------------------------------------
constexpr int kGY = 80;  // slots of the per-voice human-range gradient d/dy (78 used)
constexpr int kBC = 512;  // threads of the control-rate reverse sweep (one block per voice)

// x^a for x >= 0 and its partials (0 at x <= 0, as the forward's convention).
__device__ __forceinline__ void pow_d(float x, float a, float& p, float& dpx, float& dpa) {
  if (x <= 0.f) { p = 0.f; dpx = 0.f; dpa = 0.f; return; }
  const float lx = logf(x);
  p = expf(a * lx);
  dpx = a * p / x;
  dpa = p * lx;
}

// Gate-on level g(t) and its partials wrt (t, a, dc, s, alpha).
__device__ void gate_on_d(float t, const float* q, float& val, float d[5]) {
  const float a = q[0], dc = q[1], s = q[2], al = q[4];
  for (int i = 0; i < 5; ++i) d[i] = 0.f;
  if (t < a) {
    float p, px, pa;
    pow_d(t / a, al, p, px, pa);
    val = p;
    d[0] = px / a;             // d/dt
    d[1] = -px * t / (a * a);  // d/da
    d[4] = pa;                 // d/dalpha
  } else if (t < a + dc) {
    float p, px, pa;
    const float x = (t - a) / dc;
    pow_d(x, al, p, px, pa);
    val = 1.f - (1.f - s) * p;
    const float dx = -(1.f - s) * px;
    d[0] = dx / dc;
    d[1] = -dx / dc;
    d[2] = -dx * x / dc;
    d[3] = p;
    d[4] = -(1.f - s) * pa;
  } else {
    val = s;
    d[3] = 1.f;
  }
}

// Envelope (Sec. 3.1 reading) partials wrt (a, dc, s, r, alpha, d) at time t.
__device__ void adsr_d(float t, const float* q, float dur, float out[6]) {
  for (int i = 0; i < 6; ++i) out[i] = 0.f;
  float gd[5], val;
  if (t < dur) {
    gate_on_d(t, q, val, gd);
    out[0] = gd[1]; out[1] = gd[2]; out[2] = gd[3]; out[4] = gd[4];
    return;
  }
  const float r = q[3], al = q[4];
  const float tau = t - dur;
  if (!(tau < r)) return;
  gate_on_d(dur, q, val, gd);  // L = g(d)
  const float L = val;
  float p, px, pa;
  const float x = tau / r;
  pow_d(x, al, p, px, pa);
  const float dL = 1.f - p;           // d env / d L
  const float dx = -L * px;           // d env / d x
  out[0] = dL * gd[1];
  out[1] = dL * gd[2];
  out[2] = dL * gd[3];
  out[3] = -dx * x / r;
  out[4] = dL * gd[4] - L * pa;
  out[5] = dL * gd[0] - dx / r;       // via L = g(d) and tau = t - d
}

// Forward LFO shape mix and its derivative wrt the phase.
__device__ __forceinline__ void lfo_shapes(float p, float sh[5], float dsh[5]) {
  float sn, cs;
  sincospif(2.f * p, &sn, &cs);
  sh[0] = sn; dsh[0] = 6.28318530717958647692f * cs;
  sh[1] = 1.f - 4.f * fabsf(p - 0.5f); dsh[1] = (p - 0.5f) < 0.f ? 4.f : -4.f;
  sh[2] = 2.f * p - 1.f; dsh[2] = 2.f;
  sh[3] = 1.f - 2.f * p; dsh[3] = -2.f;
  sh[4] = p < 0.5f ? 1.f : -1.f; dsh[4] = 0.f;
}

// Adds a warp's values into its own row of the per-voice gradient (one row
// per warp, no atomics: the rows are summed in warp order at the end, so the
// gradient is the same on every run).
__device__ __forceinline__ void acc_y(float* gy_warp, int slot, float val) {
  const float w = warp_sum(val);
  if ((threadIdx.x & 31) == 0) gy_warp[slot] += w;
}

// d y / d u of the range map for parameter p at u (FP32: the FP64 pipe is
// narrow on this GPU, and the gradient needs ~1e-6).
__device__ __forceinline__ float range_map_dydu(const VoiceConst& vc, int p, float u_raw) {
  const float u = fminf(fmaxf(u_raw, 0.f), 1.f);
  const float c = ff_to_float(vc.map_curve[p]);
  const float span = vc.sym[p] ? 2.f * ff_to_float(vc.map_scale[p]) : ff_to_float(vc.map_scale[p]);
  if (!vc.sym[p]) return u <= 0.f ? 0.f : span * c * powf(u, c - 1.f);
  const float s = fabsf(2.f * u - 1.f);
  return s <= 0.f ? 0.f : span * c * powf(s, c - 1.f);
}

__global__ void __launch_bounds__(kBC) bwd_control(const __grid_constant__ VoiceConst vc,
                                                   const double* __restrict__ y,
                                                   const ff* __restrict__ env,
                                                   const double* __restrict__ lfo_phase,
                                                   const ff* __restrict__ dest,
                                                   const double* __restrict__ gpt,
                                                   const double* __restrict__ vacc,
                                                   float* __restrict__ dtheta,
                                                   float* __restrict__ denv,
                                                   const float* __restrict__ u_in,
                                                   float* __restrict__ grad_params,
                                                   int batch, ScratchHeader* hdr) {
  __shared__ float gy[kGY];
  __shared__ float gyw_all[kBC / 32][kGY];  // per-warp partial gradients
  __shared__ float yv[kNumParams];
  __shared__ float warp_tot[2 * (kBC / 32)];
  const int v = blockIdx.x;
  const int P = vc.K + 1;
  const float inv_cr = (float)(1.0 / vc.control_rate);
  const float inv_2pi = 0.15915494309189533577f;
  float* gyw = gyw_all[threadIdx.x >> 5];
  for (int i = threadIdx.x; i < kGY * (kBC / 32); i += kBC) (&gyw_all[0][0])[i] = 0.f;
  for (int i = threadIdx.x; i < kNumParams; i += kBC) yv[i] = (float)y[(size_t)v * kNumParams + i];
  __syncthreads();
  float inv_norm[5], wsum_col[5];
  for (int j = 0; j < 5; ++j) {
    float ws = 0.f;
    for (int i = 0; i < 4; ++i) ws += yv[kMod + 5 * i + j];
    wsum_col[j] = ws;
    inv_norm[j] = 1.f / fmaxf(1.f, ws);
  }
  float lfo_wsum[2];
  for (int l = 0; l < 2; ++l) {
    float ws = 0.f;
    for (int s = 0; s < 5; ++s) ws += yv[kLfo + 8 * l + 3 + s];
    lfo_wsum[l] = ws;
  }
  const double* gv = gpt + (size_t)v * P * 5;
  const double* gvr = gv + (size_t)P * 5 * gridDim.x;  // the right-end halves
  float* dth = dtheta + (size_t)v * 2 * P;
  float* de = denv + (size_t)v * 6 * P;

  // pass A: modulation mixer, LFO outputs, pitch
  for (int base = 0; base < P; base += kBC) {
    const int k = base + threadIdx.x;
    const bool ok = k < P;
    const int kk = ok ? k : 0;
    float e[6];
    for (int a = 0; a < 6; ++a) e[a] = ff_to_float(env[((size_t)v * 6 + a) * P + kk]);
    float mix[2], sh[2][5], dsh[2][5], lfo[2];
    for (int l = 0; l < 2; ++l) {
      const float th = (float)lfo_phase[((size_t)v * 2 + l) * P + kk];
      lfo_shapes(th, sh[l], dsh[l]);
      float accm = 0.f;
      for (int s = 0; s < 5; ++s) accm += yv[kLfo + 8 * l + 3 + s] * sh[l][s];
      mix[l] = lfo_wsum[l] < 1e-12f ? 0.f : accm / lfo_wsum[l];
      lfo[l] = e[3 + 2 * l] * mix[l];
    }
    const float src[4] = {e[0], e[1], lfo[0], lfo[1]};
    float dd[5] = {0, 0, 0, 0, 0}, dst[5];
    float gk[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (ok)
      for (int j = 0; j < 5; ++j) gk[j] = (float)(gv[(size_t)k * 5 + j] + gvr[(size_t)k * 5 + j]);
    if (ok) {
      dd[0] = yv[kSine + 1] * gk[0];
      dd[2] = yv[kSqr + 1] * gk[1];
      dd[1] = gk[2];
      dd[3] = gk[3];
      dd[4] = gk[4];
    }
    for (int j = 0; j < 5; ++j) dst[j] = ff_to_float(dest[((size_t)v * 5 + j) * P + kk]);
    // pitch: m = midi + tune + depth * dest
    const float dm0 = gk[0];
    const float dm1 = gk[1];
    acc_y(gyw, kMidi, dm0 + dm1);
    acc_y(gyw, kSine, dm0);
    acc_y(gyw, kSqr, dm1);
    acc_y(gyw, kSine + 1, dm0 * dst[0]);
    acc_y(gyw, kSqr + 1, dm1 * dst[2]);
    // dest_j = (sum_i W_ij src_i) / max(1, sum_i W_ij)
    float dsrc[4] = {0, 0, 0, 0};
    for (int j = 0; j < 5; ++j) {
      const float over = wsum_col[j] > 1.f ? 1.f : 0.f;
      for (int i = 0; i < 4; ++i) {
        dsrc[i] += dd[j] * yv[kMod + 5 * i + j] * inv_norm[j];
        acc_y(gyw, kMod + 5 * i + j, dd[j] * (src[i] * inv_norm[j] - over * dst[j] * inv_norm[j]));
      }
    }
    float dea[6] = {dsrc[0], dsrc[1], 0.f, 0.f, 0.f, 0.f};
    for (int l = 0; l < 2; ++l) {
      const float dl = dsrc[2 + l];
      dea[3 + 2 * l] = dl * mix[l];
      const float dmix = dl * e[3 + 2 * l];
      float dthv = 0.f;
      if (lfo_wsum[l] >= 1e-12f) {
        for (int s = 0; s < 5; ++s) {
          acc_y(gyw, kLfo + 8 * l + 3 + s, dmix * (sh[l][s] - mix[l]) / lfo_wsum[l]);
          dthv += yv[kLfo + 8 * l + 3 + s] * dsh[l][s];
        }
        dthv *= dmix / lfo_wsum[l];
      }
      if (ok) dth[(size_t)l * P + k] = dthv;
    }
    if (ok)
      for (int a = 0; a < 6; ++a) de[(size_t)a * P + k] = dea[a];
  }
  __syncthreads();

  // pass B: reverse scan of the LFO phase adjoint -> d/d(phase increment);
  // increments rate_k / CR with rate = clamp(freq + depth * env_rate, 0, 20)
  float carry0 = 0.f, carry1 = 0.f;
  for (int base = 0; base < P; base += kBC) {
    const int idx = P - 1 - (base + (int)threadIdx.x);
    const bool ok = idx >= 0;
    float a0 = ok ? dth[idx] : 0.f, a1 = ok ? dth[(size_t)P + idx] : 0.f, t0, t1;
    block_exclusive_scan2<float, kBC>(a0, a1, warp_tot, t0, t1);
    for (int l = 0; l < 2; ++l) {
      float dinc = 0.f, er = 0.f, rate_raw = 0.f;
      if (ok) {
        dinc = (l == 0 ? carry0 + a0 : carry1 + a1);  // sum of dtheta over points after idx
        er = ff_to_float(env[((size_t)v * 6 + 2 + 2 * l) * P + idx]);
        rate_raw = yv[kLfo + 8 * l] + yv[kLfo + 8 * l + 1] * er;
      }
      const bool inside = ok && rate_raw >= 0.f && rate_raw <= (float)kLfoMaxHz;
      const float dr = inside ? dinc * inv_cr : 0.f;
      acc_y(gyw, kLfo + 8 * l, dr);
      acc_y(gyw, kLfo + 8 * l + 1, dr * er);
      if (ok) de[(size_t)(2 + 2 * l) * P + idx] = dr * yv[kLfo + 8 * l + 1];
    }
    carry0 += t0;
    carry1 += t1;
  }
  if (threadIdx.x == 0) {
    gyw[kLfo + 2] += carry0 * inv_2pi;  // theta_0 = frac(phase0 / 2 pi)
    gyw[kLfo + 8 + 2] += carry1 * inv_2pi;
  }
  __syncthreads();

  // pass C: the ADSRs' partials, the (envelope, point) pairs spread over
  // the block; each thread sums its pairs' partials per envelope, then one
  // block-wide sum per partial
  float dur_acc = 0.f;
  float acc[6][5];
#pragma unroll
  for (int a = 0; a < 6; ++a)
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[a][q] = 0.f;
  for (int i = threadIdx.x; i < 6 * P; i += kBC) {
    const int a = i / P, k = i - a * P;
    const float g = de[(size_t)a * P + k];
    if (g != 0.f) {
      float out[6];
      // t_k = k / CR: the float-float product the forward pass uses,
      // rounded to float (no FP64 division per point and envelope)
      adsr_d(ff_to_float(ff_mul_f(vc.inv_cr, (float)k)), yv + kAdsr + 5 * a, yv[kDuration], out);
#pragma unroll
      for (int b = 0; b < 6; ++b)
        if (b == a) {
#pragma unroll
          for (int q = 0; q < 5; ++q) acc[b][q] += g * out[q];
        }
      dur_acc += g * out[5];
    }
  }
#pragma unroll
  for (int a = 0; a < 6; ++a)
#pragma unroll
    for (int q = 0; q < 5; ++q) acc_y(gyw, kAdsr + 5 * a + q, acc[a][q]);
  acc_y(gyw, kDuration, dur_acc);
  __syncthreads();
  for (int i = threadIdx.x; i < kGY; i += kBC) {
    float t = 0.f;
    for (int w = 0; w < kBC / 32; ++w) t += gyw_all[w][i];
    gy[i] = t;
  }
  __syncthreads();

  if (threadIdx.x == 0) {
    const double* va = vacc + (size_t)v * 8;
    gy[kSine + 2] += (float)va[0] * inv_2pi;
    gy[kSqr + 2] += (float)va[1] * inv_2pi;
    gy[kSqr + 3] += (float)va[5];
    // mixer gains g_i = l_i / max(1, sum l)
    const float l0 = yv[kMix], l1 = yv[kMix + 1], l2 = yv[kMix + 2];
    const float sum = l0 + l1 + l2, norm = fmaxf(1.f, sum);
    const float dotg = (float)va[2] * l0 + (float)va[3] * l1 + (float)va[4] * l2;
    for (int c = 0; c < 3; ++c)
      gy[kMix + c] += (float)va[2 + c] / norm - (sum > 1.f ? dotg / (norm * norm) : 0.f);
  }
  __syncthreads();
  // through the range map: d/du = d/dy dy/du
  if (threadIdx.x < kNumParams &&
      in_bounds(hdr, (long long)v * kNumParams + threadIdx.x, (long long)batch * kNumParams)) {
    const size_t i = (size_t)v * kNumParams + threadIdx.x;
    grad_params[i] = gy[threadIdx.x] * range_map_dydu(vc, threadIdx.x, u_in[i]);
  }
}


}  // namespace

size_t backward_workspace_bytes(const VoiceConst& vc, int batch) {
  return bwd_layout(vc, batch, control_bytes(vc, batch)).total;
}

cudaError_t launch_render_backward(const VoiceConst& vc, uint64_t seed, uint64_t batch_index,
                                   int batch, const float* params, const float* grad_audio,
                                   float* grad_params, void* workspace, ScratchHeader* hdr,
                                   cudaStream_t st) {
  if (vc.R > 128) return cudaErrorInvalidValue;
  const ControlBuffers cb = control_carve(vc, batch, workspace);
  const BwdLayout L = bwd_layout(vc, batch, control_bytes(vc, batch));
  char* ws = static_cast<char*>(workspace);
  float* stat = reinterpret_cast<float*>(ws + L.stat);
  double* gpt = reinterpret_cast<double*>(ws + L.gpt);
  double* vacc = reinterpret_cast<double*>(ws + L.vacc);
  float* dtheta = reinterpret_cast<float*>(ws + L.dtheta);
  float* denv = reinterpret_cast<float*>(ws + L.denv);
  const int K = vc.K, P = K + 1;
  launch_control_fused(vc, seed, batch_index, batch, params, nullptr, cb, hdr, st);
  cudaMemsetAsync(gpt, 0, sizeof(double) * 2 * (size_t)batch * P * 5, st);
  dim3 gs((K + kBT / 32 - 1) / (kBT / 32), batch);
  bwd_samples<<<gs, kBT, 0, st>>>(vc, seed, batch_index, batch, cb.mixc, cb.dest, cb.seg, cb.kappa,
                                  grad_audio, stat, hdr);
  bwd_interval_scan<<<batch, kBT, 0, st>>>(vc, stat, cb.seg, cb.kappa, gpt, vacc, hdr);
  bwd_control<<<batch, kBC, 0, st>>>(vc, cb.y, cb.env, cb.lfo_phase, cb.dest, gpt, vacc, dtheta,
                                     denv, params, grad_params, batch, hdr);
  return cudaGetLastError();
}

}  // namespace synth
