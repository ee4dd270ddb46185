// render_common.cuh -- pieces shared by the fused and the plain render kernels:
// per-interval VCO phase description, its per-sample evaluation, the block
// scan, the decoupled look-back, and the audio-rate oscillators.
#pragma once

#include <cuda/atomic>

#include "internal.h"
#include "voice_device.cuh"

namespace synth {

// How a VCO's phase advances inside one control interval. The pitch in midi
// is linear in the sample index j (Sec. 3.2 upsampling), so the per-sample
// increment f(j)/SR is geometric in j -- until the pitch reaches the Nyquist
// cap, after which it is the constant 1/2. The interval is therefore at most
// two pieces, A for j < jc and B for j >= jc, each either geometric (first
// increment c, ratio e^x) or linear (constant increment c).
struct __align__(16) SegVco {
  float phase0;  // phase in cycles at the interval's first sample, in [0, 1)
  float cA;      // first increment of piece A
  float cB;      // first increment of piece B
  float LB;      // phase advanced over piece A (cycles) = local phase where B starts
  float x;       // log of the per-sample increment ratio
  float invE;    // 1 / expm1(x)
  float ih;      // x / expm1(x) (1 when x = 0)
  int jc_flags;  // jc | (A linear) << 16 | (B linear) << 17 | (A capped) << 18 | (B capped) << 19
                 // | (every piece linear: the steps q2..r4m1 are those of x = 0) << 20
  // the four steps of a run, one 16-byte vector:
  float q2, q3;  // 1 + r and 1 + r + r^2 with r = e^x (a quad's phase steps, in units of
                 // its first increment)
  float q4;      // 1 + r + r^2 + r^3: four samples' phase in units of the first increment
  float r4m1;    // r^4 - 1: a quad's change of the increment
};
static_assert(sizeof(SegVco) == 48, "interval description: three 16-byte vectors");

// expm1(z) for the in-interval phase of a geometric piece, z = d x (d samples
// into the piece, x the log of the per-sample increment ratio). |z| < 1/4
// covers nearly every quad: the Taylor series to z^7, whose remainder is
// below z^7 / 8! < 2e-9 relative there, in Horner form; larger |z| (steep
// pitch sweeps) takes the library expm1f.
__device__ __forceinline__ float expm1_phase(float z) {
  if (fabsf(z) < 0.25f) {
    float p = fmaf(z, 1.f / 5040.f, 1.f / 720.f);
    p = fmaf(z, p, 1.f / 120.f);
    p = fmaf(z, p, 1.f / 24.f);
    p = fmaf(z, p, 1.f / 6.f);
    p = fmaf(z, p, 0.5f);
    p = fmaf(z, p, 1.f);
    return z * p;
  }
  return expm1f(z);
}

// expm1(z) / z (1 at z = 0): the same Taylor series for |z| < 1/4, one
// division by z beyond.
__device__ __forceinline__ float expm1_over_z(float z) {
  if (fabsf(z) < 0.25f) {
    float p = fmaf(z, 1.f / 5040.f, 1.f / 720.f);
    p = fmaf(z, p, 1.f / 120.f);
    p = fmaf(z, p, 1.f / 24.f);
    p = fmaf(z, p, 1.f / 6.f);
    p = fmaf(z, p, 0.5f);
    return fmaf(z, p, 1.f);
  }
  return expm1f(z) / z;
}

// Per-sample phase increments (cycles/sample) of samples j0..j0+3 and whether
// each sample's pitch is capped at Nyquist (used by the adjoint).
__device__ __forceinline__ void vco_inc_quad(const SegVco& s, int j0, float inc[4], bool capped[4]) {
  const int jc = s.jc_flags & 0xffff;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int j = j0 + i;
    const bool in_b = j >= jc;
    const float c = in_b ? s.cB : s.cA;
    const bool lin = (s.jc_flags >> (in_b ? 17 : 16)) & 1;
    capped[i] = (s.jc_flags >> (in_b ? 19 : 18)) & 1;
    const int d = j - (in_b ? jc : 0);
    inc[i] = lin ? c : c * (1.f + expm1_phase((float)d * s.x));
  }
}

constexpr double kLn2 = 0.69314718055994530942;

// Phases (cycles, wrapped to [-1/2, 1/2]) of samples j0..j0+3 of an interval.
// Inside one piece the phase of sample j0 + i is base + g e_i: linear pieces
// have g = c and e_i = i; geometric pieces (E = expm1(x), r = e^x)
// phase0 + L + (c/E)(r^(d0+i) - 1) = [phase0 + L + (c/E) E0] + c r^d0 q_i
// with E0 = expm1(d0 x), c r^d0 = c + c E0 and q_i = (r^i - 1)/(r - 1) =
// 1 + r + ... + r^(i-1): q_1 = 1 and the interval's q_2, q_3.
// The base is wrapped once (exactly), so each sample adds a term below
// 2 cycles to a number below 1/2 and wraps again.
// With kWrap = false the phases are left in (-1/2, 2) (the wrapped base plus
// at most three increments of at most 1/2), which the sine unit takes as
// they are after scaling by 2 pi.
// Wrapped phase of sample j of an interval (pieces split at jc), evaluated on
// its own.
__device__ __forceinline__ float vco_phase_at(const SegVco& s, int jc, int j) {
  const bool in_b = j >= jc;
  const float L = in_b ? s.LB : 0.f;
  const float c = in_b ? s.cB : s.cA;
  const bool lin = (s.jc_flags >> (in_b ? 17 : 16)) & 1;
  const int d = j - (in_b ? jc : 0);
  const float loc = lin ? fmaf(c, (float)d, L) : fmaf(c * s.invE, expm1_phase((float)d * s.x), L);
  const float p = s.phase0 + loc;
  return p - rintf(p);
}

// kRolled: a quad that straddles the piece boundary is evaluated by a rolled
// loop (one copy of the per-sample code: a smaller loop body where such quads
// are rare, i.e. whenever quads align with the intervals); unrolled otherwise.
template <bool kWrap = true, bool kRolled = true>
__device__ __forceinline__ void vco_quad(const SegVco& s, int j0, float ph[4]) {
  const int jc = s.jc_flags & 0xffff;
  if (j0 + 3 < jc || j0 >= jc) {
    const bool in_b = j0 >= jc;
    const float L = in_b ? s.LB : 0.f;
    const float c = in_b ? s.cB : s.cA;
    const bool lin = (s.jc_flags >> (in_b ? 17 : 16)) & 1;
    const float d0 = (float)(j0 - (in_b ? jc : 0));
    // one formula for both kinds of piece: a linear piece is the geometric
    // one with x = 0 (expm1(z)/z = 1, steps 1, 2, 3), so no branch on the kind
    const float x = lin ? 0.f : s.x;
    const float z = d0 * x;
    const float h = expm1_over_z(z);  // expm1(d0 x) = z h
    float base = s.phase0 + fmaf(c * (lin ? 1.f : s.ih), d0 * h, L);
    const float g = c * fmaf(z, h, 1.f);
    const float e2 = lin ? 2.f : s.q2, e3 = lin ? 3.f : s.q3;
    base -= rintf(base);
    ph[0] = base;
    const float p1 = base + g, p2 = fmaf(g, e2, base), p3 = fmaf(g, e3, base);
    ph[1] = kWrap ? p1 - rintf(p1) : p1;
    ph[2] = kWrap ? p2 - rintf(p2) : p2;
    ph[3] = kWrap ? p3 - rintf(p3) : p3;
  } else if (kRolled) {  // the quad straddles the piece boundary: one rolled loop
#pragma unroll 1
    for (int i = 0; i < 4; ++i) {
      const float w = vco_phase_at(s, jc, j0 + i);
      if (i == 0) ph[0] = w;
      if (i == 1) ph[1] = w;
      if (i == 2) ph[2] = w;
      if (i == 3) ph[3] = w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) ph[i] = vco_phase_at(s, jc, j0 + i);
  }
}

// A run of consecutive quads inside one piece of an interval, stepped quad
// to quad, in radians (the sine unit's argument, so no scaling per sample):
// the base phase of the current quad (wrapped to [-pi, pi]) and its first
// increment. The steps (q2, q3 inside a quad, q4 and r^4 - 1 from quad to
// quad) are read from the interval's description at each quad; they are
// those of the piece the run is in, since runs are only started in pieces of
// the kind the steps describe.
constexpr float kTwoPiRun = 6.28318530717958647692f;
constexpr float kInvTwoPiRun = 0.159154943091895335769f;
struct VcoRun {
  float base, g;
};

// Starts a run at sample j0 of the interval for `len` samples; false when
// the samples straddle the piece boundary jc, or lie in a piece of another
// kind than the interval's steps describe (a linear piece beside a geometric
// one): the caller then evaluates each quad on its own. The start is the
// quad formula of vco_quad.
__device__ __forceinline__ bool vco_run_start(const SegVco& s, int j0, int len, VcoRun& r) {
  const int jc = s.jc_flags & 0xffff;
  if (!(j0 + len - 1 < jc || j0 >= jc)) return false;
  const bool in_b = j0 >= jc;
  const float L = in_b ? s.LB : 0.f;
  const float c = in_b ? s.cB : s.cA;
  const bool lin = (s.jc_flags >> (in_b ? 17 : 16)) & 1;
  if (lin != (bool)((s.jc_flags >> 20) & 1)) return false;
  const float d0 = (float)(j0 - (in_b ? jc : 0));
  const float z = d0 * (lin ? 0.f : s.x);
  const float h = expm1_over_z(z);
  const float base = s.phase0 + fmaf(c * (lin ? 1.f : s.ih), d0 * h, L);
  r.base = kTwoPiRun * (base - rintf(base));
  r.g = kTwoPiRun * (c * fmaf(z, h, 1.f));
  return true;
}

// The current quad's four phases in radians (left in (-pi, 4 pi), as
// vco_quad<false> in cycles), then one quad on: base + g q4 wrapped (the
// float 2 pi differs from 2 pi by 1.7e-7, a drift of that much per wrapped
// cycle that ends with the run, at most a few cycles), g r^4.
__device__ __forceinline__ void vco_run_quad(const SegVco& s, VcoRun& r, float ph[4]) {
  const float4 q = *reinterpret_cast<const float4*>(&s.q2);  // q2, q3, q4, r4m1
  ph[0] = r.base;
  ph[1] = r.base + r.g;
  ph[2] = fmaf(r.g, q.x, r.base);
  ph[3] = fmaf(r.g, q.y, r.base);
  const float nb = fmaf(r.g, q.z, r.base);
  r.base = fmaf(-kTwoPiRun, rintf(nb * kInvTwoPiRun), nb);
  r.g = fmaf(r.g, q.w, r.g);
}

constexpr float kTwoPiF = 6.28318530717958647692f;

// The SFU's approximate 2^x and 1/x (PTX ex2.approx / rcp.approx; ftz).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// tanh z = 1 - 2 / (1 + e^{2z}), given y = 2 z log2(e): e^{2z} = 2^y. No
// clamp is needed: 2^y overflows to +inf (tanh = 1) or flushes to 0
// (tanh = -1), and the reciprocal of +inf is 0.
__device__ __forceinline__ float tanh_from_y(float y) {
  return fmaf(-2.f, rcp_approx(1.f + ex2_approx(y)), 1.f);
}
constexpr float kTwoLog2e = 2.88539008177792681f;  // 2 log2(e)

// Square-saw from sin and cos of the phase angle and per-interval constants
// k2 = 2 kappa log2(e), c1 = g / (tanh(kappa) (1 + shape)), c2 = c1 shape:
// g tanh(kappa sin) / tanh(kappa) * (1 + shape cos) / (1 + shape).
__device__ __forceinline__ float square_saw_sc(float sn, float cs, float k2, float c1, float c2) {
  return tanh_from_y(k2 * sn) * fmaf(c2, cs, c1);
}

// Square-saw at phase p (cycles in [-1/2, 1/2]): theta = 2 pi p,
// tanh(kappa sin theta) / tanh(kappa) * (1 + shape cos theta) / (1 + shape).
__device__ __forceinline__ float square_saw(float p, float kappa, float inv_tanh_kappa, float shape,
                                            float inv_1p_shape) {
  float sn, cs;
  __sincosf(kTwoPiF * p, &sn, &cs);
  const float c1 = inv_tanh_kappa * inv_1p_shape;
  return square_saw_sc(sn, cs, kTwoLog2e * kappa, c1, c1 * shape);
}

// ---------------------------------------------------------------------------
// Block-wide exclusive scan of two values per thread (all threads take part).
// ---------------------------------------------------------------------------
template <class T, int NT>
__device__ __forceinline__ void block_exclusive_scan2(T& a, T& b, T* warp_tot /*[2][NT/32]*/,
                                                      T& tot_a, T& tot_b) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T ia = a, ib = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T na = __shfl_up_sync(0xffffffffu, ia, o);
    T nb = __shfl_up_sync(0xffffffffu, ib, o);
    if (lane >= o) { ia += na; ib += nb; }
  }
  if (lane == 31) { warp_tot[warp] = ia; warp_tot[NT / 32 + warp] = ib; }
  __syncthreads();
  if (warp == 0) {
    T wa = lane < NT / 32 ? warp_tot[lane] : T(0);
    T wb = lane < NT / 32 ? warp_tot[NT / 32 + lane] : T(0);
#pragma unroll
    for (int o = 1; o < NT / 32; o <<= 1) {
      T na = __shfl_up_sync(0xffffffffu, wa, o);
      T nb = __shfl_up_sync(0xffffffffu, wb, o);
      if (lane >= o) { wa += na; wb += nb; }
    }
    if (lane < NT / 32) { warp_tot[lane] = wa; warp_tot[NT / 32 + lane] = wb; }
  }
  __syncthreads();
  const T pa = warp > 0 ? warp_tot[warp - 1] : T(0);
  const T pb = warp > 0 ? warp_tot[NT / 32 + warp - 1] : T(0);
  tot_a = warp_tot[NT / 32 - 1];
  tot_b = warp_tot[2 * (NT / 32) - 1];
  // exclusive prefix within the warp = the previous lane's inclusive prefix
  T ea = __shfl_up_sync(0xffffffffu, ia, 1);
  T eb = __shfl_up_sync(0xffffffffu, ib, 1);
  if (lane == 0) { ea = T(0); eb = T(0); }
  a = pa + ea;
  b = pb + eb;
  __syncthreads();
}

template <class T> __device__ __forceinline__ T wrap01(T x) { return x - floor(x); }
template <> __device__ __forceinline__ float wrap01<float>(float x) { return x - floorf(x); }

// Carry values of the look-back: 64-bit fixed-point phases (exact, mod 1 by
// integer wrap-around) or floats (the FP32-carry mode, wrapped to [0, 1)).
__device__ __forceinline__ unsigned long long carry_bits(unsigned long long v) { return v; }
__device__ __forceinline__ unsigned long long carry_bits(float v) { return __float_as_uint(v); }
template <class T> __device__ __forceinline__ T carry_from_bits(unsigned long long b);
template <> __device__ __forceinline__ unsigned long long carry_from_bits(unsigned long long b) {
  return b;
}
template <> __device__ __forceinline__ float carry_from_bits(unsigned long long b) {
  return __uint_as_float((unsigned int)b);
}
__device__ __forceinline__ unsigned long long carry_wrap(unsigned long long v) { return v; }
__device__ __forceinline__ float carry_wrap(float v) { return v - floorf(v); }

// ---------------------------------------------------------------------------
// Look-back along one voice's windows (after Merrill & Garland's single-pass
// prefix scan): each window publishes its aggregate as soon as its own block
// scan is done, then sums the aggregates of all earlier windows of the voice.
// The sum runs in a fixed order (lane j of warp 0 adds windows j, j+32, ...
// in turn, then a fixed shuffle tree), so the carry -- and with it the audio
// -- is bitwise reproducible whatever order the windows finish in (fixed-point
// carries are exact in any order; float carries need the fixed order).
// Every wait is bounded; a timeout sets the error bit in the header, and
// once the bit is set no wait of any window spins any more (fail fast).
// Called by all 32 lanes of one warp.
// ---------------------------------------------------------------------------
constexpr int kLookbackSpinLimit = 1 << 20;

// Publishes this window's aggregate of one chain (one lane writes).
template <class T>
__device__ __forceinline__ void lookback_publish(TileState* voice_tiles, int w, int chain,
                                                 unsigned int epoch, T own0, T own1) {
  TileState* me = voice_tiles + w;
  const unsigned int tag = (epoch & 0x3fffffffu) << 2;
  __stcg(&me->agg[chain][0], carry_bits(own0));
  __stcg(&me->agg[chain][1], carry_bits(own1));
  cuda::atomic_ref<unsigned int, cuda::thread_scope_device> my_flag(me->flag[chain]);
  my_flag.store(tag | 1u, cuda::memory_order_release);
}

// Sums the published aggregates of windows 0 .. w-1 (all 32 lanes of a warp;
// every lane receives the wrapped sum).
template <class T>
__device__ inline void lookback_consume(TileState* voice_tiles, int w, int chain,
                                        unsigned int epoch, T& ex0, T& ex1, ScratchHeader* hdr) {
  const int lane = threadIdx.x & 31;
  const unsigned int tag = (epoch & 0x3fffffffu) << 2;
  T s0 = T(0), s1 = T(0);
  for (int j = lane; j < w; j += 32) {
    TileState* p = voice_tiles + j;
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> pf(p->flag[chain]);
    bool ready = false;
    for (int spins = 0; spins < kLookbackSpinLimit; ++spins) {
      const unsigned int f = pf.load(cuda::memory_order_acquire);
      if (f == (tag | 1u)) { ready = true; break; }
      if (*(volatile unsigned int*)&hdr->error & kErrLookbackTimeout) break;
      __nanosleep(64);
    }
    if (!ready) {
      atomicOr(&hdr->error, kErrLookbackTimeout);
      break;
    }
    s0 += carry_from_bits<T>(__ldcg(&p->agg[chain][0]));
    s1 += carry_from_bits<T>(__ldcg(&p->agg[chain][1]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  ex0 = carry_wrap(s0);
  ex1 = carry_wrap(s1);
}

// Publish, then consume (all 32 lanes of one warp).
template <class T>
__device__ inline void lookback(TileState* voice_tiles, int w, int chain, unsigned int epoch,
                                T own0, T own1, T& ex0, T& ex1, ScratchHeader* hdr) {
  if ((threadIdx.x & 31) == 0) lookback_publish<T>(voice_tiles, w, chain, epoch, own0, own1);
  lookback_consume<T>(voice_tiles, w, chain, epoch, ex0, ex1, hdr);
}

// End-of-launch bookkeeping of the persistent kernels: the last CTA to finish
// resets the work counters and advances the epoch for the next launch.
__device__ inline void persistent_finish(ScratchHeader* hdr) {
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int prev = atomicAdd(&hdr->done, 1u);
    if (prev == gridDim.x - 1) {
      hdr->work = 0;
      hdr->done = 0;
      hdr->epoch = hdr->epoch + 1;
      __threadfence();
    }
  }
}

}  // namespace synth
