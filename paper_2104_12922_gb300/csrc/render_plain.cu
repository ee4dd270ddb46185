// render_plain.cu -- the plain, unfused Voice render: one kernel per module,
// each reading its inputs from and writing its output to device memory, the
// way a framework of batched tensor ops renders the Voice (Sec. 3.1: "all
// modules render audio in batches"; Sec. 3.2 routing). It computes the same
// quantities as the fused kernel with the same control-rate arithmetic, so
// the two differ in how the work is scheduled and how much memory traffic it
// makes, and in the last bits of the parameters and running sums.
//
// Workspace (caller-owned, 256-byte aligned sections), B voices, P = K + 1
// control points, N samples:
//   y[B][78] f64 | vff[B] VoiceFF | env[B][6][P] ff | lfo_inc[B][2][P] f64
//   lfo_phase[B][2][P] f64 | dest[B][5][P] ff | seg[B][2][K] SegVco
//   seg_sum[B][2][K] f64 | kappa[B][2][K] f32 | amp[B][3][N] f32
//   phase[B][2][N] f32 | osc[B][3][N] f32
// Control-rate values are float-float (control_ff.cuh), as in the fused
// kernel; the parameters and the running phase sums are FP64 here.

#include "internal.h"
#include "control_pipeline.cuh"

namespace synth {

namespace {

constexpr int kPT = 256;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct AudioLayout {
  size_t amp, phase, osc, total;
};

AudioLayout audio_layout(const VoiceConst& vc, int B, size_t base) {
  const size_t N = (size_t)vc.n_samples;
  AudioLayout L;
  size_t o = base;
  auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
  L.amp = take(sizeof(float) * B * 3 * N);
  L.phase = take(sizeof(float) * B * 2 * N);
  L.osc = take(sizeof(float) * B * 3 * N);
  L.total = o;
  return L;
}

// The control modules' work per element, shared by the module kernels below
// (one element per thread of a grid) and by control_fused_kernel (one CTA
// per voice looping over the voice's elements), so both write the same bits.

// Parameter module: draw (or read) and range-map parameter p of voice v.
__device__ __forceinline__ void params_elem(const VoiceConst& vc, uint64_t seed,
                                            uint64_t batch_index, int batch, const float* params_in,
                                            float* params_out, double* y, int v, int p) {
  const uint64_t g = batch_index * (uint64_t)batch + (uint64_t)v;
  float u;
  if (params_in) {
    u = fminf(fmaxf(params_in[(size_t)v * kNumParams + p], 0.f), 1.f);
  } else {
    const uint4 r = philox4x32_10(make_uint4((uint32_t)g, (uint32_t)(g >> 32), (uint32_t)(p >> 2),
                                             kStreamParam),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
    u = u01f(w[p & 3]);
  }
  if (params_out) params_out[(size_t)v * kNumParams + p] = u;
  y[(size_t)v * kNumParams + p] = range_map((double)u, vc.lo[p], vc.hi[p], vc.curve[p], vc.sym[p]);
}

// Per-voice constants of the control modules (float-float), by the threads
// of one block (at least 33): yff and T in shared memory, T loaded.
__device__ __forceinline__ void voice_consts_block(const double* y, VoiceFF* vff, float* mixc,
                                                   int v, ff* yff, const FFTables& T) {
  for (int p = threadIdx.x; p < kNumParams; p += blockDim.x)
    yff[p] = ff_from_double(y[(size_t)v * kNumParams + p]);
  __syncthreads();
  VoiceFF& V = vff[v];
  if (threadIdx.x < 16) {
    voice_ff_fill(V, yff, threadIdx.x);
  } else if (threadIdx.x == 32) {  // audio mixer gains and square-saw shape
    const double* yv = y + (size_t)v * kNumParams;
    const double norm = fmax(1.0, yv[kMix] + yv[kMix + 1] + yv[kMix + 2]);
    for (int c = 0; c < 3; ++c) mixc[(size_t)v * 5 + c] = (float)(yv[kMix + c] / norm);
    mixc[(size_t)v * 5 + 3] = (float)yv[kSqr + 3];
    mixc[(size_t)v * 5 + 4] = (float)(1.0 / (1.0 + yv[kSqr + 3]));
  }
  __syncthreads();
  __threadfence_block();
  if (threadIdx.x < 6) V.level_d[threadIdx.x] = gate_level_ff(threadIdx.x, V, T);
}

// ADSR a = i / P of voice v at control point k = i mod P.
__device__ __forceinline__ void adsr_elem(const VoiceConst& vc, const VoiceFF& V,
                                          const FFTables& T, ff* env, int v, int i) {
  const int P = vc.K + 1;
  const int a = i / P, k = i - a * P;
  const ff tk = ff_mul_f(vc.inv_cr, (float)k);
  env[((size_t)v * 6 + a) * P + k] = adsr_ff(tk, a, V, T);
}

// LFO rate: phase increment per control interval (rate / CR, FP64 for the scan).
__device__ __forceinline__ void lfo_rate_elem(const VoiceConst& vc, const VoiceFF& V,
                                              const ff* env, double* lfo_inc, int v, int k) {
  const int P = vc.K + 1;
  const ff inv_cr = vc.inv_cr;
  for (int l = 0; l < 2; ++l) {
    const ff e = env[((size_t)v * 6 + 2 + 2 * l) * P + k];
    const ff rate = ff_min(ff_max(ff_add(V.lfo_freq[l], ff_mul(V.lfo_depth[l], e)), ff_make(0.f)),
                           ff_make((float)kLfoMaxHz));
    lfo_inc[((size_t)v * 2 + l) * P + k] = ff_to_double(ff_mul(rate, inv_cr));
  }
}

// Synchronises the first kPT threads (warps 0 .. kPT/32 - 1) of a larger
// block on named barrier 1: the phase scans of control_fused_kernel run on
// those warps alone, with the module kernel's width and summation order.
__device__ __forceinline__ void sync_scan_warps() {
  asm volatile("bar.sync 1, %0;" ::"n"(kPT) : "memory");
}

// Exclusive block scan of two values over kPT threads (block_exclusive_scan2
// of render_common.cuh, the same arithmetic and order), synchronised by
// `sync`: __syncthreads in a block of kPT threads, sync_scan_warps in a
// larger one.
template <class Sync>
__device__ __forceinline__ void scan2_kpt(double& a, double& b, double* warp_tot, double& tot_a,
                                          double& tot_b, Sync sync) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double ia = a, ib = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    double na = __shfl_up_sync(0xffffffffu, ia, o);
    double nb = __shfl_up_sync(0xffffffffu, ib, o);
    if (lane >= o) { ia += na; ib += nb; }
  }
  if (lane == 31) { warp_tot[warp] = ia; warp_tot[kPT / 32 + warp] = ib; }
  sync();
  if (warp == 0) {
    double wa = lane < kPT / 32 ? warp_tot[lane] : 0.0;
    double wb = lane < kPT / 32 ? warp_tot[kPT / 32 + lane] : 0.0;
#pragma unroll
    for (int o = 1; o < kPT / 32; o <<= 1) {
      double na = __shfl_up_sync(0xffffffffu, wa, o);
      double nb = __shfl_up_sync(0xffffffffu, wb, o);
      if (lane >= o) { wa += na; wb += nb; }
    }
    if (lane < kPT / 32) { warp_tot[lane] = wa; warp_tot[kPT / 32 + lane] = wb; }
  }
  sync();
  const double pa = warp > 0 ? warp_tot[warp - 1] : 0.0;
  const double pb = warp > 0 ? warp_tot[kPT / 32 + warp - 1] : 0.0;
  tot_a = warp_tot[kPT / 32 - 1];
  tot_b = warp_tot[2 * (kPT / 32) - 1];
  double ea = __shfl_up_sync(0xffffffffu, ia, 1);
  double eb = __shfl_up_sync(0xffffffffu, ib, 1);
  if (lane == 0) { ea = 0.0; eb = 0.0; }
  a = pa + ea;
  b = pb + eb;
  sync();
}

// Exclusive running sum of per-step phase increments, wrapped to [0,1),
// starting from an initial phase: the two sequences of voice v, by kPT
// threads (see scan2_kpt for `sync`).
template <class Sync>
__device__ __forceinline__ void phase_scan_block(const double* inc, double* phase, int len,
                                                 int stride_seq, const double* y, int init_slot0,
                                                 int init_slot1, int v, double* warp_tot,
                                                 Sync sync) {
  const double two_pi = 6.28318530717958647692;
  const double* yv = y + (size_t)v * kNumParams;
  double carry0 = wrap01(yv[init_slot0] / two_pi);
  double carry1 = wrap01(yv[init_slot1] / two_pi);
  const double* in0 = inc + (size_t)(2 * v) * stride_seq;
  const double* in1 = inc + (size_t)(2 * v + 1) * stride_seq;
  double* out0 = phase + (size_t)(2 * v) * stride_seq;
  double* out1 = phase + (size_t)(2 * v + 1) * stride_seq;
  for (int base = 0; base < len; base += kPT) {
    const int i = base + threadIdx.x;
    double a = i < len ? in0[i] : 0.0, b = i < len ? in1[i] : 0.0;
    double ta, tb;
    scan2_kpt(a, b, warp_tot, ta, tb, sync);
    if (i < len) {
      out0[i] = wrap01(carry0 + a);
      out1[i] = wrap01(carry1 + b);
    }
    carry0 = wrap01(carry0 + ta);
    carry1 = wrap01(carry1 + tb);
  }
}

// LFO outputs and modulation mixer at control point k of voice v.
__device__ __forceinline__ void modmix_elem(const VoiceConst& vc, const VoiceFF& V,
                                            const FFTables& T, const ff* env,
                                            const double* lfo_phase, ff* dest, int v, int k) {
  const int P = vc.K + 1;
  ff lfo[2];
  for (int l = 0; l < 2; ++l) {
    const double th = lfo_phase[((size_t)v * 2 + l) * P + k];
    lfo[l] = lfo_ff(ff_from_double(th), l, env[((size_t)v * 6 + 3 + 2 * l) * P + k], V, T);
  }
  const ff src[4] = {env[((size_t)v * 6 + 0) * P + k], env[((size_t)v * 6 + 1) * P + k], lfo[0],
                     lfo[1]};
  for (int j = 0; j < 5; ++j) {
    ff acc = ff_mul(V.mod_w[0][j], src[0]);
    for (int i = 1; i < 4; ++i) acc = ff_add(acc, ff_mul(V.mod_w[i][j], src[i]));
    dest[((size_t)v * 5 + j) * P + k] = ff_mul(acc, V.inv_norm[j]);
  }
}

// VCO interval k of voice v: descriptions and the phase each VCO advances.
__device__ __forceinline__ void vco_interval_elem(const VoiceConst& vc, const VoiceFF& V,
                                                  const FFTables& T, const ff* dest, SegVco* seg,
                                                  double* seg_sum, float* kappa, int v, int k) {
  const int P = vc.K + 1, K = vc.K;
  const int64_t rem = vc.n_samples - (int64_t)k * vc.R;
  const int Rk = rem < vc.R ? (int)rem : vc.R;
  for (int o = 0; o < 2; ++o) {
    const ff* pd = dest + ((size_t)v * 5 + (o == 0 ? 0 : 2)) * P;
    const ff ma = ff_add(V.pitch_base[o], ff_mul(V.depth[o], pd[k]));
    const ff mb = ff_add(V.pitch_base[o], ff_mul(V.depth[o], pd[k + 1]));
    float inc_first;
    seg_sum[((size_t)v * 2 + o) * K + k] = ff_to_double(
        vco_interval_ff(ma, mb, (float)vc.R, Rk, vc.inv_R, vc.ln2_12R, vc.m_nyq_ff, vc.log2_440_over_sr, T,
                        &seg[((size_t)v * 2 + o) * K + k], &inc_first));
    if (o == 1) {  // drive 1 + SR / (8 f) at the (capped) frequency of the interval start
      const float kap = fminf((float)kBrightnessMax, 1.f + 0.125f / inc_first);
      kappa[((size_t)v * 2 + 0) * K + k] = kap;
      kappa[((size_t)v * 2 + 1) * K + k] = 1.f / tanhf(kap);
    }
  }
}

// Parameter module.
__global__ void plain_params(const __grid_constant__ VoiceConst vc, uint64_t seed,
                             uint64_t batch_index, int batch, const float* params_in,
                             float* params_out, double* y) {
  if (threadIdx.x >= kNumParams) return;
  params_elem(vc, seed, batch_index, batch, params_in, params_out, y, blockIdx.x, threadIdx.x);
}

// Per-voice constants of the control modules (float-float).
__global__ void plain_voice_consts(const __grid_constant__ VoiceConst vc, const double* y,
                                   VoiceFF* vff, float* mixc) {
  __shared__ FFTables T;
  __shared__ ff yff[kNumParams];
  load_tables(T, vc.T);
  voice_consts_block(y, vff, mixc, blockIdx.x, yff, T);
}

// ADSR modules (6 per voice) at the control points.
__global__ void plain_adsr(const __grid_constant__ VoiceConst vc, const VoiceFF* vff, ff* env) {
  __shared__ FFTables T;
  load_tables(T, vc.T);
  __syncthreads();
  const int P = vc.K + 1;
  const int v = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 6 * P) return;
  adsr_elem(vc, vff[v], T, env, v, i);
}

// LFO rate: phase increment per control interval.
__global__ void plain_lfo_rate(const __grid_constant__ VoiceConst vc, const VoiceFF* vff,
                               const ff* env, double* lfo_inc) {
  const int P = vc.K + 1;
  const int v = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P) return;
  lfo_rate_elem(vc, vff[v], env, lfo_inc, v, k);
}

// Running phase sums; one block scans the two sequences of a voice.
__global__ void plain_phase_scan(const double* inc, double* phase, int len, int stride_seq,
                                 const double* y, int init_slot0, int init_slot1) {
  __shared__ double warp_tot[2 * (kPT / 32)];
  phase_scan_block(inc, phase, len, stride_seq, y, init_slot0, init_slot1, blockIdx.x, warp_tot,
                   [] { __syncthreads(); });
}

// LFO outputs and modulation mixer at the control points.
__global__ void plain_modmix(const __grid_constant__ VoiceConst vc, const VoiceFF* vff,
                             const ff* env, const double* lfo_phase, ff* dest) {
  __shared__ FFTables T;
  load_tables(T, vc.T);
  __syncthreads();
  const int P = vc.K + 1;
  const int v = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P) return;
  modmix_elem(vc, vff[v], T, env, lfo_phase, dest, v, k);
}

// VCO interval descriptions and the phase each interval advances.
__global__ void plain_vco_intervals(const __grid_constant__ VoiceConst vc, const VoiceFF* vff,
                                    const ff* dest, SegVco* seg, double* seg_sum, float* kappa) {
  __shared__ FFTables T;
  load_tables(T, vc.T);
  __syncthreads();
  const int v = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= vc.K) return;
  vco_interval_elem(vc, vff[v], T, dest, seg, seg_sum, kappa, v, k);
}

// Writes the scanned interval start phases into the interval descriptions.
__global__ void plain_seg_phase(const __grid_constant__ VoiceConst vc, const double* seg_phase,
                                SegVco* seg, int batch) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)batch * 2 * vc.K) return;
  seg[i].phase0 = (float)seg_phase[i];
}

// The whole control pipeline of one voice per CTA (kFusedCtl threads): the
// same steps and per-element code as the module kernels above, in the same
// order, separated by barriers instead of launches; the two phase scans run
// on the first kPT threads, as wide as the module kernel's and in its order,
// so every buffer gets the same bits. The adjoint's forward recomputation
// runs it: at its batch sizes the nine module launches are each a few
// microseconds of mostly idle GPU.
constexpr int kFusedCtl = 1024;
__global__ void __launch_bounds__(kFusedCtl) control_fused_kernel(
    const __grid_constant__ VoiceConst vc, uint64_t seed, uint64_t batch_index, int batch,
    const float* params_in, float* params_out, const ControlBuffers cb, ScratchHeader* hdr) {
  __shared__ FFTables T;
  __shared__ ff yff[kNumParams];
  __shared__ double warp_tot[2 * (kPT / 32)];
  const int v = blockIdx.x, tid = threadIdx.x;
  const int P = vc.K + 1, K = vc.K;
  // every buffer below is addressed at voice v of this batch
  if (!in_bounds(hdr, v, batch)) return;
  load_tables(T, vc.T);
  if (tid < kNumParams)
    params_elem(vc, seed, batch_index, batch, params_in, params_out, cb.y, v, tid);
  __syncthreads();
  voice_consts_block(cb.y, cb.vff, cb.mixc, v, yff, T);
  __syncthreads();
  const VoiceFF& V = cb.vff[v];
  for (int i = tid; i < 6 * P; i += kFusedCtl) adsr_elem(vc, V, T, cb.env, v, i);
  __syncthreads();
  for (int k = tid; k < P; k += kFusedCtl) lfo_rate_elem(vc, V, cb.env, cb.lfo_inc, v, k);
  __syncthreads();
  if (tid < kPT)
    phase_scan_block(cb.lfo_inc, cb.lfo_phase, P, P, cb.y, kLfo + 2, kLfo + 8 + 2, v, warp_tot,
                     sync_scan_warps);
  __syncthreads();
  for (int k = tid; k < P; k += kFusedCtl)
    modmix_elem(vc, V, T, cb.env, cb.lfo_phase, cb.dest, v, k);
  __syncthreads();
  for (int k = tid; k < K; k += kFusedCtl)
    if (in_bounds(hdr, k + 1, P))  // the interval's end point
      vco_interval_elem(vc, V, T, cb.dest, cb.seg, cb.seg_sum, cb.kappa, v, k);
  __syncthreads();
  if (tid < kPT)
    phase_scan_block(cb.seg_sum, cb.seg_start, K, K, cb.y, kSine + 2, kSqr + 2, v, warp_tot,
                     sync_scan_warps);
  __syncthreads();
  for (int i = tid; i < 2 * K; i += kFusedCtl)
    cb.seg[(size_t)v * 2 * K + i].phase0 = (float)cb.seg_start[(size_t)v * 2 * K + i];
}

// Upsampled amplitudes (VCA control inputs) at audio rate.
__global__ void plain_upsample_amp(const __grid_constant__ VoiceConst vc, int batch,
                                   const ff* dest, float* amp) {
  const int64_t N = vc.n_samples;
  const int P = vc.K + 1;
  const size_t total = (size_t)batch * N;
  const float invR = 1.0f / (float)vc.R;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int v = (int)(i / N);
    const int64_t n = (int64_t)(i - (size_t)v * N);
    const int k = (int)(n / vc.R);
    const float fj = (float)(n - (int64_t)k * vc.R) * invR;
    const int dj[3] = {1, 3, 4};
    for (int c = 0; c < 3; ++c) {
      const ff* d = dest + ((size_t)v * 5 + dj[c]) * P;
      const float a0 = ff_to_float(d[k]), a1 = ff_to_float(d[k + 1]);
      amp[((size_t)v * 3 + c) * N + n] = fmaf(fj, a1 - a0, a0);
    }
  }
}

// VCO phase at audio rate (one thread per quad of samples).
__global__ void plain_vco_phase(const __grid_constant__ VoiceConst vc, int batch, const SegVco* seg,
                                float* phase) {
  const int64_t N = vc.n_samples;
  const int64_t nq = (N + 3) / 4;
  const size_t total = (size_t)batch * 2 * nq;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t vo = i / nq;
    const int64_t q = (int64_t)(i - vo * nq);
    const int64_t n0 = 4 * q;
    const int k = (int)(n0 / vc.R);
    const int j0 = (int)(n0 - (int64_t)k * vc.R);
    float ph[4];
    vco_quad(seg[vo * vc.K + k], j0, ph);
    for (int t = 0; t < 4; ++t)
      if (n0 + t < N) phase[vo * N + n0 + t] = ph[t];
  }
}

__global__ void plain_sine(const __grid_constant__ VoiceConst vc, int batch, const float* phase,
                           float* osc) {
  const int64_t N = vc.n_samples;
  const size_t total = (size_t)batch * N;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t v = i / N;
    const int64_t n = (int64_t)(i - v * N);
    osc[(v * 3 + 0) * N + n] = __sinf(kTwoPiF * phase[(v * 2 + 0) * N + n]);
  }
}

__global__ void plain_square_saw(const __grid_constant__ VoiceConst vc, int batch, const float* mixc,
                                 const float* phase, const float* kappa, float* osc) {
  const int64_t N = vc.n_samples;
  const size_t total = (size_t)batch * N;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t v = i / N;
    const int64_t n = (int64_t)(i - v * N);
    const int k = (int)(n / vc.R);
    osc[(v * 3 + 1) * N + n] =
        square_saw(phase[(v * 2 + 1) * N + n], kappa[(v * 2 + 0) * vc.K + k],
                   kappa[(v * 2 + 1) * vc.K + k], mixc[v * 5 + 3], mixc[v * 5 + 4]);
  }
}

__global__ void plain_noise(const __grid_constant__ VoiceConst vc, uint64_t seed,
                            uint64_t batch_index, int batch, float* osc) {
  const int64_t N = vc.n_samples;
  const int64_t nq = (N + 3) / 4;
  const size_t total = (size_t)batch * nq;
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t v = i / nq;
    const int64_t q = (int64_t)(i - v * nq);
    const uint64_t g = batch_index * (uint64_t)batch + v;
    const uint4 r = philox4x32_10(
        make_uint4((uint32_t)g, (uint32_t)(g >> 32), (uint32_t)q, kStreamNoise), key);
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
    for (int t = 0; t < 4; ++t)
      if (4 * q + t < N) osc[(v * 3 + 2) * N + 4 * q + t] = fmaf(2.f, u01f(w[t]), -1.f);
  }
}

__global__ void plain_vca_mix(const __grid_constant__ VoiceConst vc, int batch, const float* mixc,
                              const float* amp, const float* osc, float* audio) {
  const int64_t N = vc.n_samples;
  const size_t total = (size_t)batch * N;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t v = i / N;
    const int64_t n = (int64_t)(i - v * N);
    float acc = 0.f;
    for (int c = 0; c < 3; ++c)
      acc += mixc[v * 5 + c] * amp[(v * 3 + c) * N + n] * osc[(v * 3 + c) * N + n];
    audio[v * N + n] = acc;
  }
}

int grid_for(size_t total) {
  size_t b = (total + kPT - 1) / kPT;
  return (int)(b < 152 * 32 ? b : 152 * 32);
}

}  // namespace

size_t control_bytes(const VoiceConst& vc, int B) {
  const size_t P = (size_t)vc.K + 1, K = (size_t)vc.K;
  size_t o = 0;
  auto take = [&](size_t bytes) { o = align256(o + bytes); };
  take(sizeof(double) * B * kNumParams);
  take(sizeof(VoiceFF) * B);
  take(sizeof(ff) * B * 6 * P);
  take(sizeof(double) * B * 2 * P);
  take(sizeof(double) * B * 2 * P);
  take(sizeof(ff) * B * 5 * P);
  take(sizeof(SegVco) * B * 2 * K);
  take(sizeof(double) * B * 2 * K);
  take(sizeof(double) * B * 2 * K);
  take(sizeof(float) * B * 2 * K);
  take(sizeof(float) * B * 5);
  return o;
}

ControlBuffers control_carve(const VoiceConst& vc, int B, void* ws) {
  const size_t P = (size_t)vc.K + 1, K = (size_t)vc.K;
  char* base = static_cast<char*>(ws);
  size_t o = 0;
  auto take = [&](size_t bytes) { char* at = base + o; o = align256(o + bytes); return at; };
  ControlBuffers cb;
  cb.y = reinterpret_cast<double*>(take(sizeof(double) * B * kNumParams));
  cb.vff = reinterpret_cast<VoiceFF*>(take(sizeof(VoiceFF) * B));
  cb.env = reinterpret_cast<ff*>(take(sizeof(ff) * B * 6 * P));
  cb.lfo_inc = reinterpret_cast<double*>(take(sizeof(double) * B * 2 * P));
  cb.lfo_phase = reinterpret_cast<double*>(take(sizeof(double) * B * 2 * P));
  cb.dest = reinterpret_cast<ff*>(take(sizeof(ff) * B * 5 * P));
  cb.seg = reinterpret_cast<SegVco*>(take(sizeof(SegVco) * B * 2 * K));
  cb.seg_sum = reinterpret_cast<double*>(take(sizeof(double) * B * 2 * K));
  cb.seg_start = reinterpret_cast<double*>(take(sizeof(double) * B * 2 * K));
  cb.kappa = reinterpret_cast<float*>(take(sizeof(float) * B * 2 * K));
  cb.mixc = reinterpret_cast<float*>(take(sizeof(float) * B * 5));
  return cb;
}

void launch_control_pipeline(const VoiceConst& vc, uint64_t seed, uint64_t batch_index, int batch,
                             const float* params_in, float* params_out, const ControlBuffers& cb,
                             cudaStream_t st) {
  const int P = vc.K + 1, K = vc.K;
  dim3 gp((P + kPT - 1) / kPT, batch), gk((K + kPT - 1) / kPT, batch);
  dim3 g6((6 * P + kPT - 1) / kPT, batch);
  plain_params<<<batch, 128, 0, st>>>(vc, seed, batch_index, batch, params_in, params_out, cb.y);
  plain_voice_consts<<<batch, 96, 0, st>>>(vc, cb.y, cb.vff, cb.mixc);
  plain_adsr<<<g6, kPT, 0, st>>>(vc, cb.vff, cb.env);
  plain_lfo_rate<<<gp, kPT, 0, st>>>(vc, cb.vff, cb.env, cb.lfo_inc);
  plain_phase_scan<<<batch, kPT, 0, st>>>(cb.lfo_inc, cb.lfo_phase, P, P, cb.y, kLfo + 2,
                                          kLfo + 8 + 2);
  plain_modmix<<<gp, kPT, 0, st>>>(vc, cb.vff, cb.env, cb.lfo_phase, cb.dest);
  plain_vco_intervals<<<gk, kPT, 0, st>>>(vc, cb.vff, cb.dest, cb.seg, cb.seg_sum, cb.kappa);
  plain_phase_scan<<<batch, kPT, 0, st>>>(cb.seg_sum, cb.seg_start, K, K, cb.y, kSine + 2,
                                          kSqr + 2);
  plain_seg_phase<<<(int)(((size_t)batch * 2 * K + kPT - 1) / kPT), kPT, 0, st>>>(
      vc, cb.seg_start, cb.seg, batch);
}

void launch_control_fused(const VoiceConst& vc, uint64_t seed, uint64_t batch_index, int batch,
                          const float* params_in, float* params_out, const ControlBuffers& cb,
                          ScratchHeader* hdr, cudaStream_t st) {
  control_fused_kernel<<<batch, kFusedCtl, 0, st>>>(vc, seed, batch_index, batch, params_in,
                                                    params_out, cb, hdr);
}

size_t plain_workspace_bytes(const VoiceConst& vc, int batch) {
  return audio_layout(vc, batch, control_bytes(vc, batch)).total;
}

cudaError_t launch_render_plain(const VoiceConst& vc, uint64_t seed, uint64_t batch_index,
                                int batch, const float* params_in, float* audio,
                                float* params_out, void* workspace, ScratchHeader*, TileState*,
                                cudaStream_t st) {
  const ControlBuffers cb = control_carve(vc, batch, workspace);
  const AudioLayout L = audio_layout(vc, batch, control_bytes(vc, batch));
  char* ws = static_cast<char*>(workspace);
  float* amp = reinterpret_cast<float*>(ws + L.amp);
  float* phase = reinterpret_cast<float*>(ws + L.phase);
  float* osc = reinterpret_cast<float*>(ws + L.osc);
  const size_t NS = (size_t)batch * vc.n_samples;
  launch_control_pipeline(vc, seed, batch_index, batch, params_in, params_out, cb, st);
  plain_upsample_amp<<<grid_for(NS), kPT, 0, st>>>(vc, batch, cb.dest, amp);
  plain_vco_phase<<<grid_for(NS / 2), kPT, 0, st>>>(vc, batch, cb.seg, phase);
  plain_sine<<<grid_for(NS), kPT, 0, st>>>(vc, batch, phase, osc);
  plain_square_saw<<<grid_for(NS), kPT, 0, st>>>(vc, batch, cb.mixc, phase, cb.kappa, osc);
  plain_noise<<<grid_for(NS / 4), kPT, 0, st>>>(vc, seed, batch_index, batch, osc);
  plain_vca_mix<<<grid_for(NS), kPT, 0, st>>>(vc, batch, cb.mixc, amp, osc, audio);
  return cudaGetLastError();
}

}  // namespace synth
