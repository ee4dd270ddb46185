// render_fused.cu -- the fused persistent Voice render (one launch per batch).
//
// Work unit: a tile = (voice v, window w of kFusedTileSeg control intervals).
// Tiles are claimed from an atomic counter in window-major order (tile t ->
// v = t % batch, w = t / batch), so a tile's predecessors along its voice
// were claimed earlier by running CTAs.
//
// Each persistent CTA is warp-specialized:
//  * control warps (4 warps, one thread per control interval) claim the next
//    tile and compute everything that runs at the control rate (Sec. 3.1):
//    parameter draw (Philox, Sec. 2.1) and range map (Sec. 3.3); the 6 ADSRs,
//    the LFO rates, their phase scan with a look-back carry from earlier
//    windows, LFO shapes, modulation mixer, pitch and amplitudes (float-float,
//    control_ff.cuh); per control interval and VCO the phase advanced over the
//    interval (closed-form geometric sum of the upsampled pitch's increments)
//    and its scan with a second look-back carry (FP64; FP32 in the
//    precision-study mode). The result -- one SegVco per interval and VCO, the
//    amplitudes at the control points, the mixer gains -- goes into one of two
//    shared-memory hand-off buffers;
//  * audio warps (8 warps) take filled buffers in order and render the tile
//    (Sec. 3.2): each thread takes quads of 4 consecutive samples -- VCO
//    phases from the interval description, sine, square-saw, Philox noise,
//    VCAs, mixer -- and writes them with one 16-byte streaming store.
// The two groups hand buffers over through shared-memory mbarriers, so the
// audio warps never wait on the control group's internal barriers and the
// control work of tile i+1 overlaps the audio of tile i. Nothing but the
// audio, the parameters and a 48-byte look-back record per tile is written
// to device memory.

#include "control_ff.cuh"
#include "internal.h"
#include "render_common.cuh"

namespace synth {

namespace {

constexpr int TS = kFusedTileSeg;       // control intervals per tile
constexpr int kCtrl = TS;               // control threads: one per interval
constexpr int kAudio = 256;             // audio threads
constexpr int NT = kCtrl + kAudio;
static_assert(NT == kFusedThreads, "thread count shared with the launcher");
constexpr int kCtrlWarps = kCtrl / 32;
constexpr int kAudioWarps = kAudio / 32;
constexpr long long kHandoffSpinLimit = 1ll << 26;

// Control -> audio hand-off of one tile.
struct __align__(16) TileOut {
  SegVco seg[2][TS];
  float kappa[TS];
  float inv_tanh_kappa[TS];
  float amp[3][TS + 1];      // sine, square-saw, noise amplitudes at the control points
  float gain[3];
  float shape, inv_1p_shape;
  unsigned long long g;      // global voice index
  int v, k0, nseg, valid;
};

struct __align__(16) CtrlSmem {
  double y[kNumParams];
  VoiceFF V;
  FFTables T;
  ff env[6][TS + 1];
  ff m[2][TS + 1];           // VCO pitch (midi) at the window's control points
  double lfo_ex[2][TS + 1];  // exclusive LFO phase sums within the window
  double sums[2][TS];
  double warp_tot[2 * kCtrlWarps];
  float warp_tot_f[2 * kCtrlWarps];
  double prefix[2];
  double lfo_p0[2], vco_p0[2];  // initial phases in cycles, wrapped
  float u[80];
  ff inv_cr, inv_R, ln2_12R, m_nyq, log2_440_over_sr;
  int tile;
  unsigned int epoch;
};

struct __align__(16) FusedSmem {
  CtrlSmem c;
  TileOut out[2];
  unsigned long long full[2];   // mbarrier: control -> audio (1 arrival)
  unsigned long long empty[2];  // mbarrier: audio -> control (one arrival per audio warp)
};

__device__ __forceinline__ void ctrl_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kCtrl) : "memory"); }

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}
// Bounded wait for the phase of the given parity; false if it gave up.
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, uint32_t parity) {
  const uint32_t a = smem_addr(b);
  for (long long i = 0; i < kHandoffSpinLimit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Exclusive scan of two values over the control group's threads.
template <class T>
__device__ __forceinline__ void ctrl_exclusive_scan2(T& a, T& b, T* warp_tot, T& tot_a, T& tot_b) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T ia = a, ib = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T na = __shfl_up_sync(0xffffffffu, ia, o);
    const T nb = __shfl_up_sync(0xffffffffu, ib, o);
    if (lane >= o) { ia += na; ib += nb; }
  }
  if (lane == 31) { warp_tot[warp] = ia; warp_tot[kCtrlWarps + warp] = ib; }
  ctrl_sync();
  T pa = T(0), pb = T(0), ta = T(0), tb = T(0);
#pragma unroll
  for (int w = 0; w < kCtrlWarps; ++w) {  // fixed order: deterministic
    if (w < warp) { pa += warp_tot[w]; pb += warp_tot[kCtrlWarps + w]; }
    ta += warp_tot[w];
    tb += warp_tot[kCtrlWarps + w];
  }
  T ea = __shfl_up_sync(0xffffffffu, ia, 1);
  T eb = __shfl_up_sync(0xffffffffu, ib, 1);
  if (lane == 0) { ea = T(0); eb = T(0); }
  a = pa + ea;
  b = pb + eb;
  tot_a = ta;
  tot_b = tb;
  ctrl_sync();
}

template <class CarryT>
__device__ __forceinline__ CarryT* warp_buf(CtrlSmem& c);
template <> __device__ __forceinline__ double* warp_buf<double>(CtrlSmem& c) { return c.warp_tot; }
template <> __device__ __forceinline__ float* warp_buf<float>(CtrlSmem& c) { return c.warp_tot_f; }

// ----------------------------------------------------------- control group
template <class CarryT>
__device__ void control_loop(FusedSmem& sm, const VoiceConst& vc, uint64_t seed,
                             uint64_t batch_index, int batch, const float* __restrict__ params_in,
                             float* __restrict__ params_out, ScratchHeader* hdr, TileState* tiles,
                             int n_windows) {
  CtrlSmem& c = sm.c;
  const int tid = threadIdx.x;  // 0 .. kCtrl-1
  const int total_tiles = batch * n_windows;
  const int R = vc.R;
  const int64_t N = vc.n_samples;
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  const double two_pi = 6.28318530717958647692;
  const unsigned int epoch = c.epoch;
  for (int it = 0;; ++it) {
    const int b = it & 1;
    TileOut& o = sm.out[b];
    if (tid == 0) {
      // buffer b is free once the audio warps released its previous tile
      if (!mbar_wait(&sm.empty[b], (((uint32_t)it >> 1) & 1u) ^ 1u))
        atomicOr(&hdr->error, kErrLookbackTimeout);
      c.tile = (int)atomicAdd(&hdr->work, 1u);
    }
    ctrl_sync();
    const int t = c.tile;
    if (t >= total_tiles) {
      if (tid == 0) {
        o.valid = 0;
        mbar_arrive(&sm.full[b]);
      }
      break;
    }
    const int v = t % batch, w = t / batch;
    const uint64_t g = batch_index * (uint64_t)batch + (uint64_t)v;
    const int k0 = w * TS;
    const int nseg = min(TS, vc.K - k0);
    TileState* vt = tiles + (size_t)v * n_windows;

    // ---- parameters (Sec. 2.1 draw, Sec. 3.3 range map) ----------------
    if (params_in == nullptr) {
      if (tid < 20) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)g, (uint32_t)(g >> 32), (uint32_t)tid,
                                                 kStreamParam), key);
        c.u[4 * tid + 0] = u01f(r.x);
        c.u[4 * tid + 1] = u01f(r.y);
        c.u[4 * tid + 2] = u01f(r.z);
        c.u[4 * tid + 3] = u01f(r.w);
      }
    } else if (tid < kNumParams) {
      c.u[tid] = fminf(fmaxf(params_in[(size_t)v * kNumParams + tid], 0.f), 1.f);
    }
    ctrl_sync();
    if (tid < kNumParams) {
      const float u = c.u[tid];
      if (w == 0 && params_out) params_out[(size_t)v * kNumParams + tid] = u;
      c.y[tid] = range_map((double)u, vc.lo[tid], vc.hi[tid], vc.curve[tid], vc.sym[tid]);
    }
    ctrl_sync();
    const double* y = c.y;
    if (tid < 16) {
      voice_ff_fill(c.V, y, tid);
    } else if (tid == 32) {
      const double l0 = y[kMix], l1 = y[kMix + 1], l2 = y[kMix + 2];
      const double norm = fmax(1.0, l0 + l1 + l2);
      o.gain[0] = (float)(l0 / norm);
      o.gain[1] = (float)(l1 / norm);
      o.gain[2] = (float)(l2 / norm);
      o.shape = (float)y[kSqr + 3];
      o.inv_1p_shape = (float)(1.0 / (1.0 + y[kSqr + 3]));
      o.g = g;
      o.v = v;
      o.k0 = k0;
      o.nseg = nseg;
    } else if (tid == 64) {
      c.lfo_p0[0] = wrap01(y[kLfo + 2] / two_pi);
      c.lfo_p0[1] = wrap01(y[kLfo + 8 + 2] / two_pi);
      c.vco_p0[0] = wrap01(y[kSine + 2] / two_pi);
      c.vco_p0[1] = wrap01(y[kSqr + 2] / two_pi);
    }
    ctrl_sync();
    const VoiceFF& V = c.V;
    if (tid < 6) c.V.level_d[tid] = gate_level_ff(tid, V, c.T);
    ctrl_sync();

    // ---- envelopes at control points k0 .. k0 + nseg (one (point, ADSR) per item)
    for (int i = tid; i < 6 * (nseg + 1); i += kCtrl) {
      const int pt = i / 6, a = i - 6 * pt;
      c.env[a][pt] = adsr_ff(ff_mul_f(c.inv_cr, (float)(k0 + pt)), a, V, c.T);
    }
    ctrl_sync();

    // ---- LFO phase increments rate_k / CR at points k0 .. k0 + nseg - 1, scanned (FP64)
    double r0 = 0.0, r1 = 0.0;
    if (tid < nseg) {
      const ff lim = ff_make((float)kLfoMaxHz), z = ff_make(0.f);
      r0 = ff_to_double(ff_mul(ff_min(ff_max(ff_add(V.lfo_freq[0], ff_mul(V.lfo_depth[0], c.env[2][tid])), z), lim), c.inv_cr));
      r1 = ff_to_double(ff_mul(ff_min(ff_max(ff_add(V.lfo_freq[1], ff_mul(V.lfo_depth[1], c.env[4][tid])), z), lim), c.inv_cr));
    }
    double tot0, tot1;
    ctrl_exclusive_scan2<double>(r0, r1, c.warp_tot, tot0, tot1);
    if (tid < nseg) {
      c.lfo_ex[0][tid] = r0;
      c.lfo_ex[1][tid] = r1;
    }
    if (tid == 0) {
      c.lfo_ex[0][nseg] = tot0;
      c.lfo_ex[1][nseg] = tot1;
    }
    if (tid < 32) {
      double e0, e1;
      lookback<double>(vt, w, 0, epoch, wrap01(tot0), wrap01(tot1), e0, e1, hdr);
      if (tid == 0) {
        c.prefix[0] = e0;
        c.prefix[1] = e1;
      }
    }
    ctrl_sync();

    // ---- LFOs, modulation mixer, pitch and amplitudes at each control point
    for (int i = tid; i <= nseg; i += kCtrl) {
      ff lfo[2];
#pragma unroll
      for (int l = 0; l < 2; ++l) {
        const double theta = wrap01(c.lfo_p0[l] + c.prefix[l] + c.lfo_ex[l][i]);
        lfo[l] = lfo_ff(ff_from_double(theta), l, c.env[3 + 2 * l][i], V, c.T);
      }
      const ff src[4] = {c.env[0][i], c.env[1][i], lfo[0], lfo[1]};
      ff dest[5];
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        ff acc = ff_mul(V.mod_w[0][j], src[0]);
#pragma unroll
        for (int s = 1; s < 4; ++s) acc = ff_add(acc, ff_mul(V.mod_w[s][j], src[s]));
        dest[j] = ff_mul(acc, V.inv_norm[j]);
      }
      c.m[0][i] = ff_add(V.pitch_base[0], ff_mul(V.depth[0], dest[0]));
      c.m[1][i] = ff_add(V.pitch_base[1], ff_mul(V.depth[1], dest[2]));
      o.amp[0][i] = ff_to_float(dest[1]);
      o.amp[1][i] = ff_to_float(dest[3]);
      o.amp[2][i] = ff_to_float(dest[4]);
    }
    ctrl_sync();

    // ---- VCO phase over each control interval, scanned ---------------------
    CarryT s0 = CarryT(0), s1 = CarryT(0);
    if (tid < nseg) {
      const int k = k0 + tid;
      const int64_t rem = N - (int64_t)k * R;
      const int Rk = rem < R ? (int)rem : R;
      s0 = (CarryT)vco_interval_ff(c.m[0][tid], c.m[0][tid + 1], R, Rk, c.inv_R, c.ln2_12R, c.m_nyq,
                                   c.log2_440_over_sr, c.T, &o.seg[0][tid]);
      s1 = (CarryT)vco_interval_ff(c.m[1][tid], c.m[1][tid + 1], R, Rk, c.inv_R, c.ln2_12R, c.m_nyq,
                                   c.log2_440_over_sr, c.T, &o.seg[1][tid]);
      const ff mk = ff_min(c.m[1][tid], c.m_nyq);
      const float fk = (float)vc.sample_rate * ff_to_float(inc_at_ff(mk, c.log2_440_over_sr, c.T));
      const float kap = fminf((float)kBrightnessMax, 1.f + (float)vc.sample_rate / (8.f * fk));
      o.kappa[tid] = kap;
      o.inv_tanh_kappa[tid] = 1.f / tanhf(kap);
    }
    CarryT t0, t1;
    ctrl_exclusive_scan2<CarryT>(s0, s1, warp_buf<CarryT>(c), t0, t1);
    if (tid < 32) {
      CarryT e0, e1;
      lookback<CarryT>(vt, w, 1, epoch, wrap01(t0), wrap01(t1), e0, e1, hdr);
      if (tid == 0) {
        c.prefix[0] = (double)e0;
        c.prefix[1] = (double)e1;
      }
    }
    ctrl_sync();
    if (tid < nseg) {
      o.seg[0][tid].phase0 = (float)wrap01((CarryT)c.vco_p0[0] + (CarryT)c.prefix[0] + s0);
      o.seg[1][tid].phase0 = (float)wrap01((CarryT)c.vco_p0[1] + (CarryT)c.prefix[1] + s1);
    }
    ctrl_sync();
    if (tid == 0) {
      o.valid = 1;
      mbar_arrive(&sm.full[b]);  // release: the tile's description is complete
    }
  }
}

// ------------------------------------------------------------- audio group
__device__ void audio_loop(FusedSmem& sm, const VoiceConst& vc, uint64_t seed,
                           float* __restrict__ audio, ScratchHeader* hdr) {
  const int atid = threadIdx.x - kCtrl;  // 0 .. kAudio-1
  const int lane = threadIdx.x & 31;
  const int R = vc.R;
  const int qps = R >> 2;  // quads per control interval
  const int64_t N = vc.n_samples;
  const bool vec_ok = (N & 3) == 0;
  const float invR = 1.0f / (float)R;
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  for (int it = 0;; ++it) {
    const int b = it & 1;
    if (!mbar_wait(&sm.full[b], ((uint32_t)it >> 1) & 1u)) {
      if (atid == 0) atomicOr(&hdr->error, kErrLookbackTimeout);
      break;
    }
    const TileOut& o = sm.out[b];
    if (!o.valid) break;
    const float g0 = o.gain[0], g1 = o.gain[1], g2 = o.gain[2];
    const float shape = o.shape, inv_1p_shape = o.inv_1p_shape;
    const uint64_t g = o.g;
    const int k0 = o.k0;
    float* out_v = audio + (size_t)o.v * (size_t)N;
    const int nq = o.nseg * qps;
    for (int q = atid; q < nq; q += kAudio) {
      const int s = q / qps;
      const int j0 = (q - s * qps) << 2;
      const int64_t n0 = (int64_t)(k0 + s) * R + j0;
      if (n0 >= N) continue;
      float ps[4], pq[4];
      vco_quad(o.seg[0][s], j0, ps);
      vco_quad(o.seg[1][s], j0, pq);
      const float kap = o.kappa[s], itk = o.inv_tanh_kappa[s];
      const uint4 nz = philox4x32_10(
          make_uint4((uint32_t)g, (uint32_t)(g >> 32), (uint32_t)(n0 >> 2), kStreamNoise), key);
      const uint32_t nw[4] = {nz.x, nz.y, nz.z, nz.w};
      const float a00 = o.amp[0][s], a10 = o.amp[1][s], a20 = o.amp[2][s];
      const float d0 = o.amp[0][s + 1] - a00, d1 = o.amp[1][s + 1] - a10,
                  d2 = o.amp[2][s + 1] - a20;
      float out4[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float fj = (float)(j0 + i) * invR;
        const float x_sin = __sinf(kTwoPiF * ps[i]);
        const float x_sq = square_saw(pq[i], kap, itk, shape, inv_1p_shape);
        const float x_nz = fmaf(2.f, u01f(nw[i]), -1.f);
        out4[i] = g0 * fmaf(fj, d0, a00) * x_sin + g1 * fmaf(fj, d1, a10) * x_sq +
                  g2 * fmaf(fj, d2, a20) * x_nz;
      }
      if (vec_ok && n0 + 3 < N) {
        __stcs(reinterpret_cast<float4*>(out_v + n0), make_float4(out4[0], out4[1], out4[2], out4[3]));
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (n0 + i < N) out_v[n0 + i] = out4[i];
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&sm.empty[b]);
  }
}

template <class CarryT>
__global__ void __launch_bounds__(NT, 2) render_fused_kernel(
    const __grid_constant__ VoiceConst vc, uint64_t seed, uint64_t batch_index, int batch,
    const float* __restrict__ params_in, float* __restrict__ audio, float* __restrict__ params_out,
    ScratchHeader* hdr, TileState* tiles, int n_windows) {
  __shared__ FusedSmem sm;
  const int tid = threadIdx.x;
  if (tid == 0) {
    sm.c.epoch = *(volatile unsigned int*)&hdr->epoch;
    sm.c.inv_cr = ff_from_double(1.0 / vc.control_rate);
    sm.c.inv_R = ff_from_double(1.0 / (double)vc.R);
    sm.c.ln2_12R = ff_from_double(kLn2 / (12.0 * (double)vc.R));
    sm.c.m_nyq = ff_from_double(vc.m_nyq);
    sm.c.log2_440_over_sr = ff_from_double(log2(440.0 / vc.sample_rate));
    mbar_init(&sm.full[0], 1);
    mbar_init(&sm.full[1], 1);
    mbar_init(&sm.empty[0], kAudioWarps);
    mbar_init(&sm.empty[1], kAudioWarps);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 33) ff_tables_fill_entry(sm.c.T, tid);
  __syncthreads();
  if (tid < kCtrl)
    control_loop<CarryT>(sm, vc, seed, batch_index, batch, params_in, params_out, hdr, tiles,
                         n_windows);
  else
    audio_loop(sm, vc, seed, audio, hdr);
  __syncthreads();
  persistent_finish(hdr);
}

}  // namespace

int fused_max_active_blocks_per_sm() {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, render_fused_kernel<double>, NT, 0);
  return n;
}

cudaError_t launch_render_fused(const VoiceConst& vc, uint64_t seed, uint64_t batch_index,
                                int batch, const float* params_in, float* audio,
                                float* params_out, ScratchHeader* hdr, TileState* tiles,
                                int grid, cudaStream_t stream) {
  const int n_windows = windows_per_voice(vc.K);
  const int total = batch * n_windows;
  grid = grid < total ? grid : total;
  if (vc.carry_fp32)
    render_fused_kernel<float><<<grid, NT, 0, stream>>>(vc, seed, batch_index, batch, params_in,
                                                        audio, params_out, hdr, tiles, n_windows);
  else
    render_fused_kernel<double><<<grid, NT, 0, stream>>>(vc, seed, batch_index, batch, params_in,
                                                         audio, params_out, hdr, tiles, n_windows);
  return cudaGetLastError();
}

}  // namespace synth
