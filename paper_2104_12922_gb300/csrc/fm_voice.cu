// fm_voice.cu -- the 4-operator FM voice: four sine operators in a serial
// phase-modulation stack op3 -> op2 -> op1 -> op0 (Chowning's FM as phase
// modulation), each at f0 x ratio_i with the Voice's ADSR gated by the
// keyboard's note-on duration; out(n) = y_0(n) with y_4 = 0 and
// y_i(n) = level_i E_i(n) sin(2 pi phi_i(n) + y_(i+1)(n)). The paper names a
// 4-operator FM architecture as in development (Sec. 3.2) and specifies no
// more; parameter ranges and the stack are this library's choices.
//
// One CTA renders one voice's chunk of kFmChunk samples: it draws (or loads)
// the 30 normalized parameters, maps them, turns each operator's frequency
// into a 64-bit fixed-point phase increment (the phase of sample n is the
// exact product n x inc mod 2^64), evaluates the four envelopes at the
// control points the chunk spans, and then renders 4-sample quads. No FP64:
// the increments come from the float-float exp2 of the Voice's control chain.
#include <cuda_runtime.h>

#include <cstdint>

#include "control_ff.cuh"
#include "internal.h"
#include "voice_device.cuh"

namespace synth {
namespace {

constexpr int kFmThreads = 256;
constexpr int kFmChunk = 8192;                  // samples per CTA (a multiple of 4)
constexpr uint32_t kStreamFmParam = 2;

struct FmConst {
  int64_t N, rate_a, rate_b;  // samples; R = rate_a / rate_b samples per control interval
  ff inv_cr;                  // 1 / control rate
  int max_pts;                // control points a chunk can span
  ff log2_440_over_sr;        // log2(440 / SR)
  alignas(16) FFTables T;     // float-float exp2 tables
};

// Normalized parameter p -> human value, y = lo + (hi - lo) u^c with c = 1
// or 2 (exact products). Layout: midi f0, note-on duration, then per
// operator (0 = carrier) ratio, level, attack, decay, sustain, release, alpha.
__host__ __device__ inline void fm_range(int p, float& lo, float& hi, int& c) {
  if (p < 2) {
    lo = 0.f;
    hi = p == 0 ? 127.f : 4.f;
    c = 1;
    return;
  }
  const int i = (p - 2) / 7, q = (p - 2) % 7;
  const float los[7] = {0.5f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.1f};
  const float his[7] = {8.f, 8.f, 2.f, 2.f, 1.f, 5.f, 6.f};
  const int cs[7] = {2, 2, 2, 2, 1, 2, 2};
  lo = los[q];
  hi = (q == 1 && i == 0) ? 1.f : his[q];  // the carrier's level is an amplitude in [0, 1]
  c = (q == 1 && i == 0) ? 1 : cs[q];
}

// The Voice's ADSR (attack (t/a)^alpha, decay to s, release from the level at
// note-off d); zero-length sections are skipped. The section lengths, the
// note-on duration and the time are float-float, and so are the section
// choice and the time into the section (t - a, t - d): the argument x of
// x^alpha then carries a relative error of a few float roundings wherever
// the section falls in the note. (In FP32 the time alone is off by up to
// t 2^-24 s, which near a section start with alpha < 1 -- where x^alpha is
// steep -- moves the envelope by 1e-5 and more.) x^alpha itself is FP32.
struct FmEnv {
  ff a, dc, r, d;  // attack, decay, release, note-on duration (s)
  float s, alpha;  // sustain level, curve exponent
};
__device__ __forceinline__ float fm_gate_on(ff t, const FmEnv& E) {
  if (ff_lt(t, E.a)) return powf(ff_to_float(t) / ff_to_float(E.a), E.alpha);
  const ff ta = ff_sub(t, E.a);
  if (ff_lt(ta, E.dc)) return 1.f - (1.f - E.s) * powf(ff_to_float(ta) / ff_to_float(E.dc), E.alpha);
  return E.s;
}
__device__ __forceinline__ float fm_adsr(ff t, const FmEnv& E) {
  if (ff_lt(t, E.d)) return fm_gate_on(t, E);
  const ff tau = ff_sub(t, E.d);
  if (!ff_lt(tau, E.r)) return 0.f;
  return fm_gate_on(E.d, E) * (1.f - powf(ff_to_float(tau) / ff_to_float(E.r), E.alpha));
}

// Operator i's envelope constants from its normalized parameters uo (ratio,
// level, attack, decay, sustain, release, alpha) and the duration parameter
// ud: attack and decay 2 u^2, release 5 u^2 (u^2 exact as a float-float
// product), duration 4 u, sustain u; alpha = 0.1 + 5.9 u^2 as in the
// parameter map.
__device__ __forceinline__ FmEnv fm_env(const float* uo, float ud) {
  FmEnv E;
  E.a = ff_mul_f(two_prod(uo[2], uo[2]), 2.f);
  E.dc = ff_mul_f(two_prod(uo[3], uo[3]), 2.f);
  E.r = ff_mul_f(two_prod(uo[5], uo[5]), 5.f);
  E.d = ff_make(4.f * ud);
  E.s = uo[4];
  E.alpha = fmaf(6.f - 0.1f, uo[6] * uo[6], 0.1f);
  return E;
}

struct __align__(16) FmSmem {
  float u[32];
  float y[kNumFmParams];
  unsigned long long inc[4];
};

// sin(2 pi t) for |t| <= 1/2: a quarter-turn reduction t = q/4 + r,
// |r| <= 1/8, then sin(2 pi t) = sin x, cos x, -sin x, -cos x (x = 2 pi r)
// for q = 0, 1, 2, 3 (mod 4), with the Taylor series of sin to x^9 and of
// cos to x^10 in Horner form (truncation below 2e-9 at |x| = pi/4).
__device__ __forceinline__ float sin2pi_poly(float t) {
  const float q = rintf(4.f * t);
  const float x = fmaf(q, -0.25f, t) * 6.28318530717958648f;
  const float z = x * x;
  float ps = fmaf(z, 1.f / 362880.f, -1.f / 5040.f);
  ps = fmaf(z, ps, 1.f / 120.f);
  ps = fmaf(z, ps, -1.f / 6.f);
  const float sn = fmaf(z * x, ps, x);
  float pc = fmaf(z, -1.f / 3628800.f, 1.f / 40320.f);
  pc = fmaf(z, pc, -1.f / 720.f);
  pc = fmaf(z, pc, 1.f / 24.f);
  pc = fmaf(z, pc, -0.5f);
  const float cs = fmaf(z, pc, 1.f);
  const int qi = (int)q & 3;
  const float v = (qi & 1) ? cs : sn;
  return (qi & 2) ? -v : v;
}

__global__ void __launch_bounds__(kFmThreads) fm_render_kernel(const __grid_constant__ FmConst fc,
                                                               uint64_t seed,
                                                               uint64_t batch_index, int batch,
                                                               const float* __restrict__ params_in,
                                                               float* __restrict__ audio,
                                                               float* __restrict__ params_out) {
  __shared__ FmSmem S;
  // per control point the chunk spans: the four envelopes, the first sample
  // of its interval (chunk-relative) and that sample's fraction
  extern __shared__ __align__(16) float fm_dyn[];
  const int max_pts = fc.max_pts;
  float* env = fm_dyn;                                         // [4][max_pts]
  int* sst = reinterpret_cast<int*>(fm_dyn + 4 * max_pts);     // [max_pts]
  float* fr0 = fm_dyn + 5 * max_pts;                           // [max_pts]
  const int tid = threadIdx.x;
  const int v = blockIdx.y;
  const uint64_t g = batch_index * (uint64_t)batch + (uint64_t)v;
  const int64_t s0 = (int64_t)blockIdx.x * kFmChunk;
  const int64_t N = fc.N;
  const int64_t s1 = min(s0 + (int64_t)kFmChunk, N);
  // ---- parameters
  if (params_in == nullptr) {
    if (tid < 8) {
      const uint4 r = philox4x32_10(
          make_uint4((uint32_t)g, (uint32_t)(g >> 32), (uint32_t)tid, kStreamFmParam),
          make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
      S.u[4 * tid + 0] = u01f(r.x);
      S.u[4 * tid + 1] = u01f(r.y);
      S.u[4 * tid + 2] = u01f(r.z);
      S.u[4 * tid + 3] = u01f(r.w);
    }
  } else if (tid < kNumFmParams) {
    S.u[tid] = fminf(fmaxf(params_in[(size_t)v * kNumFmParams + tid], 0.f), 1.f);
  }
  __syncthreads();
  if (tid < kNumFmParams) {
    const float u = S.u[tid];
    if (blockIdx.x == 0 && params_out) params_out[(size_t)v * kNumFmParams + tid] = u;
    float lo, hi;
    int c;
    fm_range(tid, lo, hi, c);
    S.y[tid] = fmaf(hi - lo, c == 2 ? u * u : u, lo);
  }
  if (tid < 4) {
    // the operator's increment in cycles per sample, f0 ratio / SR with
    // f0 = 440 2^((m - 69)/12), in float-float (relative error ~1e-14), then
    // its fraction as 64-bit fixed point: phase(n) = n inc mod 2^64 exactly
    const float ur = S.u[2 + 7 * tid];
    const ff m = ff_mul_f(ff_make(127.f), S.u[0]);
    const ff ratio = ff_add_f(ff_mul_f(ff_mul_f(ff_make(ur), ur), 7.5f), 0.5f);
    S.inc[tid] = ff_to_fix64(ff_mul(inc_at_ff(m, fc.log2_440_over_sr, fc.T), ratio));
  }
  __syncthreads();
  // ---- envelopes at the control points the chunk spans
  const int64_t k_lo = s0 * fc.rate_b / fc.rate_a;
  const int64_t k_hi = (s1 - 1) * fc.rate_b / fc.rate_a + 1;
  const int npts = (int)(k_hi - k_lo + 1);
  for (int j = tid; j < npts; j += kFmThreads) {
    const int64_t k = k_lo + j;
    const ff t = ff_mul_f(fc.inv_cr, (float)k);  // k < 2^24: exact in a float
#pragma unroll 1
    for (int i = 0; i < 4; ++i) env[i * max_pts + j] = fm_adsr(t, fm_env(S.u + 2 + 7 * i, S.u[1]));
    const int64_t sk = (k * fc.rate_a + fc.rate_b - 1) / fc.rate_b;
    sst[j] = (int)(sk - s0);
    fr0[j] = (float)(sk * fc.rate_b - k * fc.rate_a) / (float)fc.rate_a;
  }
  __syncthreads();
  // ---- audio
  const float lev[4] = {S.y[3], S.y[10], S.y[17], S.y[24]};
  const float invR = (float)fc.rate_b / (float)fc.rate_a;
  const float kInv2Pi = 0.15915494309189535f;
  const int n_c = (int)(s1 - s0);
  float* out = audio + (size_t)v * (size_t)N + (size_t)s0;
  const bool vec = (N & 3) == 0 && (reinterpret_cast<uintptr_t>(audio) & 15) == 0;
  for (int q = tid; 4 * q < n_c; q += kFmThreads) {
    const int r0 = 4 * q;
    int j = min((int)((float)r0 * invR), npts - 2);
    while (j + 1 < npts - 1 && sst[j + 1] <= r0) ++j;
    while (j > 0 && sst[j] > r0) --j;
    const unsigned long long n0 = (unsigned long long)(s0 + r0);
    // per operator: the quad's first phase (one 64-bit product, then sums),
    // and the envelope of the quad's interval(s) (it meets at most two)
    unsigned long long ph[4];
    float ea[4], da[4], eb[4], db[4];
    const bool two = j + 1 < npts - 1 && r0 + 3 >= sst[j + 1];
#pragma unroll
    for (int op = 0; op < 4; ++op) {
      ph[op] = n0 * S.inc[op];
      ea[op] = env[op * max_pts + j];
      da[op] = env[op * max_pts + j + 1] - ea[op];
      eb[op] = two ? env[op * max_pts + j + 1] : ea[op];
      db[op] = two ? env[op * max_pts + j + 2] - eb[op] : da[op];
    }
    float o4[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + i;
      const bool in_b = two && r >= sst[j + 1];
      const int jj = in_b ? j + 1 : j;
      const float fu = fmaf((float)(r - sst[jj]), invR, fr0[jj]);
      float yv = 0.f;
#pragma unroll
      for (int op = 3; op >= 0; --op) {
        // the phase's top 24 bits are exact in a float (converted from 32
        // bits: a 64-bit conversion would take the FP64 pipe); add the
        // modulation (radians -> cycles), reduce to [-1/2, 1/2]
        float t = fmaf(yv, kInv2Pi, (float)(uint32_t)(ph[op] >> 40) * 0x1p-24f);
        t -= rintf(t);
        const float e = in_b ? fmaf(fu, db[op], eb[op]) : fmaf(fu, da[op], ea[op]);
        // a modulator's sine error is amplified by the levels below it: a
        // sine accurate to an ulp or two there; the carrier's is not: the
        // SFU sine
        const float sn = op == 0 ? __sinf(6.283185307179586f * t) : sin2pi_poly(t);
        yv = lev[op] * e * sn;
        ph[op] += S.inc[op];
      }
      o4[i] = yv;
    }
    if (vec && r0 + 3 < n_c) {
      __stcs(reinterpret_cast<float4*>(out + r0), make_float4(o4[0], o4[1], o4[2], o4[3]));
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (r0 + i < n_c) out[r0 + i] = o4[i];
    }
  }
}

}  // namespace

cudaError_t launch_fm_render(const VoiceConst& vc, uint64_t seed, uint64_t batch_index, int batch,
                             const float* params_in, float* audio, float* params_out,
                             cudaStream_t stream) {
  if (batch <= 0) return cudaSuccess;
  if (batch > 65535) return cudaErrorInvalidValue;
  FmConst fc;
  fc.N = vc.n_samples;
  fc.rate_a = vc.rate_a;
  fc.rate_b = vc.rate_b;
  fc.inv_cr = ff_from_double(1.0 / vc.control_rate);
  fc.log2_440_over_sr = vc.log2_440_over_sr;
  fc.T = vc.T;
  fc.max_pts = (int)((int64_t)kFmChunk * vc.rate_b / vc.rate_a) + 3;
  const size_t smem = sizeof(float) * 6 * (size_t)fc.max_pts;
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(fm_render_kernel,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
    if (e != cudaSuccess) return e;
  }
  const dim3 grid((unsigned)((vc.n_samples + kFmChunk - 1) / kFmChunk), (unsigned)batch);
  fm_render_kernel<<<grid, kFmThreads, smem, stream>>>(fc, seed, batch_index, batch, params_in,
                                                       audio, params_out);
  return cudaGetLastError();
}

}  // namespace synth
