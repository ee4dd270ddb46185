// render_fused.cu -- the fused persistent Voice render (one launch per batch).
//
// Work unit: a tile = (voice v, window w of kFusedTileSeg control intervals).
// CTAs are persistent and claim tiles from an atomic counter in window-major
// order (tile t -> v = t % batch, w = t / batch), so a tile's predecessors
// along its voice were claimed earlier by running CTAs. Per tile:
//  1. draw (Philox, Sec. 2.1) and range-map (Sec. 3.3) the 78 parameters;
//  2. control rate (Sec. 3.1): 6 ADSRs at the window's control points, the
//     LFO rates, an exclusive block scan of the LFO phase increments and a
//     decoupled look-back for the LFO phase carry from earlier windows;
//     LFO shapes, modulation mixer, VCO pitch, amplitudes -- in float-float
//     (control_ff.cuh), with FP64 running sums;
//  3. per control interval and VCO, the phase advanced over the interval
//     (closed-form geometric sum of the upsampled pitch's increments,
//     float-float),
//     an exclusive block scan of those sums and a second look-back for the
//     VCO phase carry (FP64; FP32 in the precision-study mode);
//  4. audio rate (Sec. 3.2): each thread renders quads of 4 consecutive
//     samples -- VCO phases from the interval description, sine, square-saw,
//     Philox noise, VCAs, mixer -- and writes them with one 16-byte store.
// Nothing but the audio and the parameters is written to device memory apart
// from the 80-byte look-back record per tile.

#include "internal.h"
#include "control_ff.cuh"
#include "render_common.cuh"

namespace synth {

namespace {

constexpr int NT = kFusedThreads;
constexpr int TS = kFusedTileSeg;
static_assert(NT == 2 * TS, "one thread per (control interval, VCO) pair");

struct __align__(16) FusedSmem {
  double y[kNumParams];
  VoiceFF V;
  FFTables T;
  ff env[6][TS + 1];
  ff m[2][TS + 1];           // VCO pitch (midi) at the window's control points
  float amp[3][TS + 1];      // sine, square-saw, noise amplitudes
  SegVco seg[2][TS];
  float kappa[TS];
  float inv_tanh_kappa[TS];
  double warp_tot[2 * (NT / 32)];
  float warp_tot_f[2 * (NT / 32)];
  double prefix[2];
  float u[80];
  float gain[3];
  float shape, inv_1p_shape;
  ff inv_cr, inv_R, ln2_12R, m_nyq, log2_440_over_sr;
  int tile;
  unsigned int epoch;
};

template <class CarryT>
__device__ __forceinline__ CarryT* warp_buf(FusedSmem& sm);
template <> __device__ __forceinline__ double* warp_buf<double>(FusedSmem& sm) { return sm.warp_tot; }
template <> __device__ __forceinline__ float* warp_buf<float>(FusedSmem& sm) { return sm.warp_tot_f; }

template <class CarryT>
__global__ void __launch_bounds__(NT) render_fused_kernel(
    const __grid_constant__ VoiceConst vc, uint64_t seed, uint64_t batch_index, int batch,
    const float* __restrict__ params_in, float* __restrict__ audio, float* __restrict__ params_out,
    ScratchHeader* hdr, TileState* tiles, int n_windows) {
  __shared__ FusedSmem sm;
  const int tid = threadIdx.x;
  const int total_tiles = batch * n_windows;
  const int R = vc.R;
  const int qps = R >> 2;  // quads per control interval
  const int64_t N = vc.n_samples;
  const bool vec_ok = (N & 3) == 0;
  const float invR = 1.0f / (float)R;
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  const double two_pi = 6.28318530717958647692;
  if (tid == 0) {
    sm.epoch = *(volatile unsigned int*)&hdr->epoch;
    sm.inv_cr = ff_from_double(1.0 / vc.control_rate);
    sm.inv_R = ff_from_double(1.0 / (double)R);
    sm.ln2_12R = ff_from_double(kLn2 / (12.0 * (double)R));
    sm.m_nyq = ff_from_double(vc.m_nyq);
    sm.log2_440_over_sr = ff_from_double(log2(440.0 / vc.sample_rate));
  }
  if (tid < 33) ff_tables_fill_entry(sm.T, tid);

  for (;;) {
    if (tid == 0) sm.tile = (int)atomicAdd(&hdr->work, 1u);
    __syncthreads();
    const int t = sm.tile;
    const unsigned int epoch = sm.epoch;
    if (t >= total_tiles) break;
    const int v = t % batch, w = t / batch;
    const uint64_t g = batch_index * (uint64_t)batch + (uint64_t)v;
    const int k0 = w * TS;
    const int nseg = min(TS, vc.K - k0);
    TileState* vt = tiles + (size_t)v * n_windows;

    // ---- 1. parameters (Sec. 2.1 draw, Sec. 3.3 range map) --------------
    if (params_in == nullptr) {
      if (tid < 20) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)g, (uint32_t)(g >> 32), (uint32_t)tid,
                                                 kStreamParam), key);
        sm.u[4 * tid + 0] = u01f(r.x);
        sm.u[4 * tid + 1] = u01f(r.y);
        sm.u[4 * tid + 2] = u01f(r.z);
        sm.u[4 * tid + 3] = u01f(r.w);
      }
    } else if (tid < kNumParams) {
      sm.u[tid] = fminf(fmaxf(params_in[(size_t)v * kNumParams + tid], 0.f), 1.f);
    }
    __syncthreads();
    if (tid < kNumParams) {
      const float u = sm.u[tid];
      if (w == 0 && params_out) params_out[(size_t)v * kNumParams + tid] = u;
      sm.y[tid] = range_map((double)u, vc.lo[tid], vc.hi[tid], vc.curve[tid], vc.sym[tid]);
    }
    __syncthreads();
    const double* y = sm.y;
    if (tid < 16) {
      voice_ff_fill(sm.V, y, tid);
    } else if (tid == 32) {
      const double l0 = y[kMix], l1 = y[kMix + 1], l2 = y[kMix + 2];
      const double norm = fmax(1.0, l0 + l1 + l2);
      sm.gain[0] = (float)(l0 / norm);
      sm.gain[1] = (float)(l1 / norm);
      sm.gain[2] = (float)(l2 / norm);
      sm.shape = (float)y[kSqr + 3];
      sm.inv_1p_shape = (float)(1.0 / (1.0 + y[kSqr + 3]));
    }
    __syncthreads();
    const VoiceFF& V = sm.V;
    if (tid < 6) sm.V.level_d[tid] = gate_level_ff(tid, V, sm.T);
    __syncthreads();

    // ---- 2. envelopes at control points k0 .. k0 + nseg -------------------
    // (one thread per (point, ADSR) pair keeps the threads busy)
    for (int i = tid; i < 6 * (nseg + 1); i += NT) {
      const int pt = i / 6, a = i - 6 * pt;
      const ff tk = ff_mul_f(sm.inv_cr, (float)(k0 + pt));
      sm.env[a][pt] = adsr_ff(tk, a, V, sm.T);
    }
    __syncthreads();

    // LFO phase increments rate_k / CR at points k0 .. k0 + nseg - 1, scanned
    // in FP64.
    double r0 = 0.0, r1 = 0.0;
    if (tid < nseg) {
      const ff lim = ff_make((float)kLfoMaxHz);
      const ff z = ff_make(0.f);
      r0 = ff_to_double(ff_mul(ff_min(ff_max(ff_add(V.lfo_freq[0], ff_mul(V.lfo_depth[0], sm.env[2][tid])), z), lim), sm.inv_cr));
      r1 = ff_to_double(ff_mul(ff_min(ff_max(ff_add(V.lfo_freq[1], ff_mul(V.lfo_depth[1], sm.env[4][tid])), z), lim), sm.inv_cr));
    }
    double tot0, tot1;
    block_exclusive_scan2<double, NT>(r0, r1, sm.warp_tot, tot0, tot1);
    if (tid < 32) {
      double e0, e1;
      lookback<double>(vt, w, 0, epoch, wrap01(tot0), wrap01(tot1), e0, e1, hdr);
      if (tid == 0) {
        sm.prefix[0] = e0;
        sm.prefix[1] = e1;
      }
    }
    __syncthreads();

    // LFOs, modulation mixer, pitch and amplitudes at each control point.
    if (tid <= nseg) {
      ff lfo[2];
#pragma unroll
      for (int l = 0; l < 2; ++l) {
        const double theta = wrap01(wrap01(y[kLfo + 8 * l + 2] / two_pi) + sm.prefix[l] + (l == 0 ? r0 : r1));
        lfo[l] = lfo_ff(ff_from_double(theta), l, sm.env[3 + 2 * l][tid], V, sm.T);
      }
      const ff src[4] = {sm.env[0][tid], sm.env[1][tid], lfo[0], lfo[1]};
      ff dest[5];
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        ff acc = ff_mul(V.mod_w[0][j], src[0]);
#pragma unroll
        for (int i = 1; i < 4; ++i) acc = ff_add(acc, ff_mul(V.mod_w[i][j], src[i]));
        dest[j] = ff_mul(acc, V.inv_norm[j]);
      }
      sm.m[0][tid] = ff_add(V.pitch_base[0], ff_mul(V.depth[0], dest[0]));
      sm.m[1][tid] = ff_add(V.pitch_base[1], ff_mul(V.depth[1], dest[2]));
      sm.amp[0][tid] = dest[1].hi + dest[1].lo;
      sm.amp[1][tid] = dest[3].hi + dest[3].lo;
      sm.amp[2][tid] = dest[4].hi + dest[4].lo;
    }
    __syncthreads();

    // ---- 3. VCO phase over each control interval, scanned -----------------
    // (threads 0..nseg-1 take the sine VCO, threads 128.. the square-saw)
    double s_own = 0.0;
    {
      const int o = tid >= TS ? 1 : 0;
      const int si = tid - o * TS;
      if (si < nseg) {
        const int k = k0 + si;
        const int64_t rem = N - (int64_t)k * R;
        const int Rk = rem < R ? (int)rem : R;
        s_own = vco_interval_ff(sm.m[o][si], sm.m[o][si + 1], R, Rk, sm.inv_R, sm.ln2_12R, sm.m_nyq,
                                sm.log2_440_over_sr, sm.T, &sm.seg[o][si]);
        if (o == 1) {
          const ff mk = ff_min(sm.m[1][si], sm.m_nyq);
          const float fk = (float)vc.sample_rate * ff_to_float(inc_at_ff(mk, sm.log2_440_over_sr, sm.T));
          const float kap = fminf((float)kBrightnessMax, 1.f + (float)vc.sample_rate / (8.f * fk));
          sm.kappa[si] = kap;
          sm.inv_tanh_kappa[si] = 1.f / tanhf(kap);
        }
      }
    }
    __syncthreads();
    // gather the two VCOs' sums onto the scan threads 0..nseg-1
    CarryT s0 = CarryT(0), s1 = CarryT(0);
    {
      __shared__ double sums[2][TS];
      const int o = tid >= TS ? 1 : 0;
      const int si = tid - o * TS;
      if (si < nseg) sums[o][si] = s_own;
      __syncthreads();
      if (tid < nseg) {
        s0 = (CarryT)sums[0][tid];
        s1 = (CarryT)sums[1][tid];
      }
    }
    CarryT t0, t1;
    block_exclusive_scan2<CarryT, NT>(s0, s1, warp_buf<CarryT>(sm), t0, t1);
    if (tid < 32) {
      CarryT e0, e1;
      lookback<CarryT>(vt, w, 1, epoch, wrap01(t0), wrap01(t1), e0, e1, hdr);
      if (tid == 0) {
        sm.prefix[0] = (double)e0;
        sm.prefix[1] = (double)e1;
      }
    }
    __syncthreads();
    if (tid < nseg) {
      const CarryT p0 = (CarryT)wrap01(y[kSine + 2] / two_pi);
      const CarryT p1 = (CarryT)wrap01(y[kSqr + 2] / two_pi);
      sm.seg[0][tid].phase0 = (float)wrap01(p0 + (CarryT)sm.prefix[0] + s0);
      sm.seg[1][tid].phase0 = (float)wrap01(p1 + (CarryT)sm.prefix[1] + s1);
    }
    __syncthreads();

    // ---- 4. audio rate ----------------------------------------------------
    const float g0 = sm.gain[0], g1 = sm.gain[1], g2 = sm.gain[2];
    const float shape = sm.shape, inv_1p_shape = sm.inv_1p_shape;
    float* out_v = audio + (size_t)v * (size_t)N;
    const int nq = nseg * qps;
    for (int q = tid; q < nq; q += NT) {
      const int s = q / qps;
      const int j0 = (q - s * qps) << 2;
      const int64_t n0 = (int64_t)(k0 + s) * R + j0;
      if (n0 >= N) continue;
      float ps[4], pq[4];
      vco_quad(sm.seg[0][s], j0, ps);
      vco_quad(sm.seg[1][s], j0, pq);
      const float kap = sm.kappa[s], itk = sm.inv_tanh_kappa[s];
      const uint4 nz = philox4x32_10(
          make_uint4((uint32_t)g, (uint32_t)(g >> 32), (uint32_t)(n0 >> 2), kStreamNoise), key);
      const uint32_t nw[4] = {nz.x, nz.y, nz.z, nz.w};
      float o[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float fj = (float)(j0 + i) * invR;
        const float a0 = fmaf(fj, sm.amp[0][s + 1] - sm.amp[0][s], sm.amp[0][s]);
        const float a1 = fmaf(fj, sm.amp[1][s + 1] - sm.amp[1][s], sm.amp[1][s]);
        const float a2 = fmaf(fj, sm.amp[2][s + 1] - sm.amp[2][s], sm.amp[2][s]);
        const float x_sin = __sinf(kTwoPiF * ps[i]);
        const float x_sq = square_saw(pq[i], kap, itk, shape, inv_1p_shape);
        const float x_nz = fmaf(2.f, u01f(nw[i]), -1.f);
        o[i] = g0 * a0 * x_sin + g1 * a1 * x_sq + g2 * a2 * x_nz;
      }
      if (vec_ok && n0 + 3 < N) {
        __stcs(reinterpret_cast<float4*>(out_v + n0), make_float4(o[0], o[1], o[2], o[3]));
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (n0 + i < N) out_v[n0 + i] = o[i];
      }
    }
    __syncthreads();
  }
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
