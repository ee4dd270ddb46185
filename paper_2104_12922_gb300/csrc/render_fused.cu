// render_fused.cu -- the fused persistent Voice render (one launch per batch
// or per several consecutive batches).
//
// Work unit: a tile = (voice v, window w) of kFusedTilePoints = 256 control
// points, i.e. the 255 control intervals between them; window w starts at
// control point 255 w, so consecutive windows share their boundary point.
// Tiles are claimed from an atomic counter in window-major order (tile t ->
// v = t % batch, w = t / batch), so a tile's predecessors along its voice
// were claimed earlier by running CTAs.
//
// One CTA of 256 threads takes a tile through these steps, one thread per
// control point (Sec. 3.1 control rate) and then all threads on the audio:
//  1. parameters: Philox draw (Sec. 2.1) or the caller's values, Sec. 3.3
//     range map (float-float), the per-voice constants -- derived by the
//     voice's first window and published, copied by its later windows;
//  2. the 6 ADSRs at the thread's control point, the two LFO rates and their
//     phase increments over the interval that starts there;
//  3. a block scan of those increments plus a look-back over the voice's
//     earlier windows gives each point's LFO phases; LFO shapes, modulation
//     mixer, pitch of both VCOs and the three amplitudes at the point;
//  4. per interval and VCO the closed-form description of the phase (SegVco)
//     and the phase advanced over it; a second scan + look-back gives each
//     interval's starting phase;
//  5. the audio (Sec. 3.2): each thread takes runs of quads of 4 consecutive
//     samples of one interval -- VCO phases from the interval description,
//     stepped from quad to quad, sine, square-saw, Philox noise, VCAs,
//     mixer -- each quad written with one 16-byte streaming store.
// The control chain is float-float (control_ff.cuh); running phase sums are
// 64-bit fixed point, exact and order-independent (FP32 in the precision-study
// mode). Nothing but the audio, the parameters, a 48-byte look-back record
// per tile and a set-up record per voice is written to device memory, and no
// FP64 arithmetic runs. Consecutive launches on a stream may overlap (see
// release_next_launch and the launch record at the end of this file).

#include <mutex>
#include <unordered_map>

#include "control_ff.cuh"
#include "internal.h"
#include "philox_noise.cuh"
#include "render_common.cuh"

namespace synth {

namespace {

constexpr int NT = kFusedThreads;
constexpr int P = kFusedTilePoints;
constexpr int TI = kFusedTileSeg;
constexpr int kWarps = NT / 32;
static_assert(NT == P, "one thread per control point");

using u64 = unsigned long long;

// What a tile derives from its voice's parameters before its control points
// (step 1): the same for every window of the voice.
struct __align__(16) VoiceSetup {
  VoiceFF V;
  u64 lfo_p0[2], vco_p0[2];    // initial phases
  float gain[3];               // mixer gains (sine, square-saw, noise)
  float shape, inv_1p_shape;   // square-saw shape and 1 / (1 + shape)
};
static_assert(sizeof(VoiceSetup) % 16 == 0, "voice set-up copies as 16-byte vectors");

// A voice's set-up as its first window published it: windows after the
// first copy it instead of deriving it again when it is there (flag = this
// launch's epoch tag); when it is not yet, they derive it themselves, with
// the same arithmetic, so the result does not depend on which happened.
struct __align__(16) VoiceSetupRecord {
  unsigned int flag;  // (epoch << 2) | 1 once vs is written in this launch
  unsigned int pad[3];
  VoiceSetup vs;
};

struct __align__(16) Smem {
  FFTables T;
  union {
    ff env[6][P];            // the 6 ADSRs at the control points (steps 2-3)
    struct {
      SegVco seg[2][TI];     // VCO interval descriptions (steps 4-5)
      union {
        float4 aslope[TI];   // R a multiple of 4: amplitude change per sample over each
                             // interval, (ampv[k + 1] - ampv[k]) / R
        struct {
          int sst[P];        // fractional R: first sample of each interval (tile-relative),
                             // sst[nseg] = the tile's sample count
          float u0f[TI];     // fractional R: fraction of each interval's first sample
        };
      };
    };
  };
  float4 sq[TI];             // square-saw constants per interval: k2, c1, c2 (square_saw_sc)
  float4 ampv[P];            // gain x amplitude at the control points: sine, square-saw (gain
                             // folded into sq), noise
  ff m[2][P];                // VCO pitch (midi) at the control points
  ff y[kNumParams];          // human-range parameters
  VoiceSetup vs;
  float u[80];
  u64 warp_tot[2][2][kWarps];  // [scan][chain][warp]
  float warp_tot_f[2][kWarps];
  float warp_max[kWarps];      // peak variant: per-warp largest |sample|
  u64 prefix[2][2];            // [scan][chain]: phase carried in from earlier windows
  float prefix_f[2];
  int tile;
  int setup_ready;             // this tile copies its voice's published set-up
  unsigned int epoch;
};
// static shared memory is capped at 48 KB per block; 4 blocks per SM fit
static_assert(sizeof(Smem) <= 48 * 1024, "shared-memory layout exceeds the static limit");

// Exclusive block scan of two fixed-point values (exact, any order). After
// the barrier inside, warp 0 receives the block totals in tot0/tot1 (all
// lanes) for its look-back; the caller then writes s.prefix and syncs.
__device__ __forceinline__ void block_scan2_fix(u64& a, u64& b, u64 (*buf)[kWarps], u64& tot0,
                                                u64& tot1) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u64 ia = a, ib = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u64 na = __shfl_up_sync(0xffffffffu, ia, o);
    const u64 nb = __shfl_up_sync(0xffffffffu, ib, o);
    if (lane >= o) { ia += na; ib += nb; }
  }
  if (lane == 31) { buf[0][warp] = ia; buf[1][warp] = ib; }
  __syncthreads();
  u64 pa = 0, pb = 0, ta = 0, tb = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    const u64 wa = buf[0][w], wb = buf[1][w];
    if (w < warp) { pa += wa; pb += wb; }
    ta += wa;
    tb += wb;
  }
  a = pa + ia - a;
  b = pb + ib - b;
  tot0 = ta;
  tot1 = tb;
}

// The same for two float values (FP32-carry mode): the warp-level inclusive
// sums, then the earlier warps' totals added in a fixed order.
__device__ __forceinline__ void block_scan2_f32(float& a, float& b, float (*buf)[kWarps],
                                                float& tot0, float& tot1) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float ia = a, ib = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float na = __shfl_up_sync(0xffffffffu, ia, o);
    const float nb = __shfl_up_sync(0xffffffffu, ib, o);
    if (lane >= o) { ia += na; ib += nb; }
  }
  if (lane == 31) { buf[0][warp] = ia; buf[1][warp] = ib; }
  __syncthreads();
  float pa = 0.f, pb = 0.f, ta = 0.f, tb = 0.f;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    if (w < warp) { pa += buf[0][w]; pb += buf[1][w]; }
    ta += buf[0][w];
    tb += buf[1][w];
  }
  float ea = __shfl_up_sync(0xffffffffu, ia, 1);
  float eb = __shfl_up_sync(0xffffffffu, ib, 1);
  if (lane == 0) { ea = 0.f; eb = 0.f; }
  a = pa + ea;
  b = pb + eb;
  tot0 = ta;
  tot1 = tb;
}

// The tile's peak (a block maximum of the threads' largest |sample|),
// published in its tile record behind a done flag once every thread's
// stores are visible at device scope.
__device__ __forceinline__ void publish_tile_peak(Smem& s, TileState* me, float vmax,
                                                  unsigned int epoch) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  if ((tid & 31) == 0) s.warp_max[tid >> 5] = vmax;
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    float m = s.warp_max[0];
#pragma unroll
    for (int i = 1; i < kWarps; ++i) m = fmaxf(m, s.warp_max[i]);
    me->peak = __float_as_uint(m);
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> f(me->done);
    f.store(((epoch & 0x3fffffffu) << 2) | 3u, cuda::memory_order_release);
  }
}

// One normalisation work item: chunk c (kNormChunkSamples samples) of voice
// v. Waits, with a spin limit, for the done flags of the voice's render
// tiles, takes the largest of their peaks, and scales the chunk by 1 / peak
// when the peak reaches the threshold; chunk 0 also writes the voice's peak
// and silence flag. Every tile it waits for was claimed earlier from the
// same counter by a running CTA, and render tiles never wait for these
// items, so the wait ends.
__device__ __noinline__ void normalize_chunk(Smem& s, float* __restrict__ audio, int64_t N,
                                             TileState* vt, int n_windows, int v, int c,
                                             bool vec_ok, const PeakNormArgs& norm,
                                             ScratchHeader* hdr, unsigned int epoch) {
  const int tid = threadIdx.x;
  const unsigned int tag = ((epoch & 0x3fffffffu) << 2) | 3u;
  float m = 0.f;
  for (int w = tid; w < n_windows; w += NT) {
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> f(vt[w].done);
    bool ready = false;
    for (int spins = 0; spins < kLookbackSpinLimit; ++spins) {
      if (f.load(cuda::memory_order_acquire) == tag) { ready = true; break; }
      if (*(volatile unsigned int*)&hdr->error) break;
      __nanosleep(128);
    }
    if (!ready) {
      atomicOr(&hdr->error, kErrTileWaitTimeout);
      break;
    }
    m = fmaxf(m, __uint_as_float(__ldcg(&vt[w].peak)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((tid & 31) == 0) s.warp_max[tid >> 5] = m;
  __syncthreads();
  float peak = s.warp_max[0];
#pragma unroll
  for (int i = 1; i < kWarps; ++i) peak = fmaxf(peak, s.warp_max[i]);
  const bool failed = *(volatile unsigned int*)&hdr->error & kErrTileWaitTimeout;
  const bool loud = peak >= norm.threshold && peak > 0.f && !failed;
  if (c == 0 && tid == 0) {
    if (norm.peak_out) norm.peak_out[v] = peak;
    if (norm.silent_out) norm.silent_out[v] = loud ? 0 : 1;
  }
  if (!loud) return;
  const float g = 1.0f / peak;
  const int64_t a0 = (int64_t)c * kNormChunkSamples;
  const int n = (int)min((int64_t)kNormChunkSamples, N - a0);
  // the chunk's samples lie in the voice's [0, N)
  if (!in_bounds(hdr, a0, N) || !in_bounds(hdr, a0 + n - 1, N)) return;
  float* x = audio + (size_t)v * N + a0;
  if (vec_ok) {  // N % 4 == 0 and a 16-byte aligned buffer: whole quads
    float4* x4 = reinterpret_cast<float4*>(x);
    constexpr int kPer = 4;  // quads in flight per thread
#pragma unroll 1
    for (int q0 = tid; 4 * q0 < n; q0 += kPer * NT) {
      float4 r[kPer];
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const int q = q0 + i * NT;
        if (4 * q < n) r[i] = __ldcg(x4 + q);
      }
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const int q = q0 + i * NT;
        if (4 * q < n) __stcs(x4 + q, make_float4(r[i].x * g, r[i].y * g, r[i].z * g, r[i].w * g));
      }
    }
  } else {
    for (int i = tid; i < n; i += NT) x[i] = __ldcg(x + i) * g;
  }
}

// Programmatic dependent launch. When a CTA takes a render tile that is
// likely its last (fewer items remain after it than the grid has CTAs), and
// after a scaling item that is, it waits for the previous grid on the stream
// to complete (a no-op unless this launch may overlap it) and then releases
// the next launch on the stream: when every CTA has done so, the next
// launch's CTAs start in the SM slots that this launch's last wave leaves
// idle. Releasing before the last tile rather than after it lets the next
// launch in while that tile runs. The wait comes first, so launch N + 2,
// which uses launch N's scratch, can never overlap launch N. Neither grid
// ever waits on the other's work.
__device__ __forceinline__ void release_next_launch(bool& released) {
  if (released) return;
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  released = true;
}

template <bool kCarryF32, bool kPeak, bool kGenR>
__global__ void __launch_bounds__(NT, 4) render_fused_kernel(
    const __grid_constant__ VoiceConst vc, uint64_t seed, uint64_t first, int split, int batch,
    const float* __restrict__ params_in, float* __restrict__ audio, float* __restrict__ params_out,
    ScratchHeader* hdr, TileState* tiles, int n_windows, const PeakNormArgs norm,
    uint64_t seed_step, int sub_batch, VoiceSetupRecord* setups) {
  __shared__ Smem s;
  const int tid = threadIdx.x;
  const int total_tiles = batch * n_windows;
  const int R = vc.R, K = vc.K;
  const int64_t N = vc.n_samples;
  const int qps = R >> 2;             // quads per control interval
  const bool vec_ok = (N & 3) == 0 && (reinterpret_cast<uintptr_t>(audio) & 15) == 0;
  const float invR = 1.0f / (float)R;
  load_tables(s.T, vc.T);
  if (tid == 0) s.epoch = *(volatile unsigned int*)&hdr->epoch;
  // all work items of the launch: render tiles, then (peak variant) scaling chunks
  const int total_items =
      total_tiles + (kPeak ? (int)((N + kNormChunkSamples - 1) / kNormChunkSamples) * batch : 0);
  bool released = false;

  for (;;) {
    if (tid == 0) {
      const int tc = (int)atomicAdd(&hdr->work, 1u);
      s.tile = tc;
      // a later window of a voice whose first window has published its set-up
      int ready = 0;
      if (setups && tc < total_tiles && tc >= batch && in_bounds(hdr, tc % batch, batch)) {
        cuda::atomic_ref<unsigned int, cuda::thread_scope_device> f(setups[tc % batch].flag);
        ready = f.load(cuda::memory_order_acquire) == (((s.epoch & 0x3fffffffu) << 2) | 1u);
      }
      s.setup_ready = ready;
    }
    __syncthreads();  // also: the previous tile's audio is done with the shared buffers
    const int t = s.tile;
    if (t >= total_tiles) {
      // peak variant: the scaling chunks follow the render tiles, voice by
      // voice (window-major tiles finish their voices in that order)
      if (!kPeak) { release_next_launch(released); break; }
      const int chunks = (int)((N + kNormChunkSamples - 1) / kNormChunkSamples);
      const int j = t - total_tiles;
      if (j >= chunks * batch) { release_next_launch(released); break; }
      if (!in_bounds(hdr, j / chunks, batch)) continue;
      normalize_chunk(s, audio, N, tiles + (size_t)(j / chunks) * n_windows, n_windows,
                      j / chunks, j % chunks, vec_ok, norm, hdr, s.epoch);
      if (t + (int)gridDim.x >= total_items) release_next_launch(released);
      continue;
    }
    if (t + (int)gridDim.x >= total_items) release_next_launch(released);  // likely the last tile
    const int v = t % batch, w = t / batch;
    // the tile's voice and window address its set-up, tile and output records
    if (!in_bounds(hdr, v, batch) || !in_bounds(hdr, w, n_windows)) continue;
    const uint64_t g = split_voice(split, first + (uint64_t)v);
    // consecutive sub-batches of sub_batch voices may each have their own
    // seed: seed + (v / sub_batch) seed_step
    const uint64_t sd = seed + (uint64_t)(v / sub_batch) * seed_step;
    const uint2 key = make_uint2((uint32_t)sd, (uint32_t)(sd >> 32));
    const int k0 = w * TI;
    const int nseg = min(TI, K - k0);
    // 1 <= nseg <= TI: every per-interval index below (tid, si < nseg; the
    // point after an interval, <= nseg < P) stays inside the shared arrays
    if (!in_bounds(hdr, nseg - 1, TI)) continue;
    TileState* vt = tiles + (size_t)v * n_windows;
    const unsigned int epoch = s.epoch;

    // ---- 1. parameters (Sec. 2.1 draw, Sec. 3.3 range map) ---------------
    const VoiceFF& V = s.vs.V;
    constexpr int kSetupVec = (int)(sizeof(VoiceSetup) / 16);
    static_assert(kSetupVec <= NT, "one 16-byte vector of the set-up per thread");
    if (s.setup_ready) {
      // a later window: the set-up its voice's first window published
      const float4* src = reinterpret_cast<const float4*>(&setups[v].vs);
      float4* dst = reinterpret_cast<float4*>(&s.vs);
      for (int i = tid; i < kSetupVec; i += NT) dst[i] = __ldcg(src + i);
      __syncthreads();
    } else {
      if (params_in == nullptr) {
        if (tid < 20) {
          const uint4 r = philox4x32_10(make_uint4((uint32_t)g, (uint32_t)(g >> 32), (uint32_t)tid,
                                                   kStreamParam), key);
          s.u[4 * tid + 0] = u01f(r.x);
          s.u[4 * tid + 1] = u01f(r.y);
          s.u[4 * tid + 2] = u01f(r.z);
          s.u[4 * tid + 3] = u01f(r.w);
        }
      } else if (tid < kNumParams &&
                 in_bounds(hdr, (long long)v * kNumParams + tid, (long long)batch * kNumParams)) {
        s.u[tid] = fminf(fmaxf(params_in[(size_t)v * kNumParams + tid], 0.f), 1.f);
      }
      __syncthreads();
      if (tid < kNumParams) {
        const float u = s.u[tid];
        if (w == 0 && params_out &&
            in_bounds(hdr, (long long)v * kNumParams + tid, (long long)batch * kNumParams))
          params_out[(size_t)v * kNumParams + tid] = u;
        s.y[tid] = range_map_ff(u, vc.map_base[tid], vc.map_scale[tid], vc.map_curve[tid],
                                vc.map_code[tid], vc.sym[tid], s.T);
      }
      __syncthreads();
      if (tid < 16) {
        voice_ff_fill(s.vs.V, s.y, tid);
      } else if (tid == 32) {
        const float l0 = ff_to_float(s.y[kMix]), l1 = ff_to_float(s.y[kMix + 1]),
                    l2 = ff_to_float(s.y[kMix + 2]);
        const float inv = 1.f / fmaxf(1.f, l0 + l1 + l2);
        s.vs.gain[0] = l0 * inv;
        s.vs.gain[1] = l1 * inv;
        s.vs.gain[2] = l2 * inv;
        const float sh = ff_to_float(s.y[kSqr + 3]);
        s.vs.shape = sh;
        s.vs.inv_1p_shape = 1.f / (1.f + sh);
      } else if (tid == 64) {
        s.vs.lfo_p0[0] = ff_to_fix64(ff_mul(s.y[kLfo + 2], vc.inv_2pi));
        s.vs.lfo_p0[1] = ff_to_fix64(ff_mul(s.y[kLfo + 8 + 2], vc.inv_2pi));
        s.vs.vco_p0[0] = ff_to_fix64(ff_mul(s.y[kSine + 2], vc.inv_2pi));
        s.vs.vco_p0[1] = ff_to_fix64(ff_mul(s.y[kSqr + 2], vc.inv_2pi));
      }
      __syncthreads();
      if (tid < 6) s.vs.V.level_d[tid] = gate_level_ff(tid, V, s.T);
      __syncthreads();
      if (w == 0 && setups && n_windows > 1 && tid < kSetupVec) {
        // published for the voice's later windows; the flag follows after
        // the barrier that ends step 3
        reinterpret_cast<float4*>(&setups[v].vs)[tid] = reinterpret_cast<const float4*>(&s.vs)[tid];
        __threadfence();
      }
    }

    // ---- 2. rate envelopes at point k0 + tid; LFO increments over interval tid
    const bool has_pt = tid <= nseg;
    const ff tk = ff_mul_f(vc.inv_cr, (float)(k0 + tid));
    if (has_pt) {
#pragma unroll 1
      for (int a = 2; a <= 4; a += 2) s.env[a][tid] = adsr_ff(tk, a, V, s.T);
    }
    u64 r0 = 0, r1 = 0;
    if (tid < nseg) {
      const ff lim = ff_make((float)kLfoMaxHz), z = ff_make(0.f);
#pragma unroll 1
      for (int l = 0; l < 2; ++l) {
        const ff rate = ff_min(
            ff_max(ff_add(V.lfo_freq[l], ff_mul(V.lfo_depth[l], s.env[2 + 2 * l][tid])), z), lim);
        const u64 r = ff_to_fix64(ff_mul(rate, vc.inv_cr));
        if (l == 0) r0 = r; else r1 = r;
      }
    }

    // ---- 3. LFO phases: scan, publish this window's aggregate, the other
    // four envelopes, then the look-back (the predecessors have had the time
    // of four envelopes to publish theirs); LFOs, mixer, pitch, amplitudes --
    {
      u64 t0, t1;
      block_scan2_fix(r0, r1, s.warp_tot[0], t0, t1);
      if (tid == 0) lookback_publish<u64>(vt, w, 0, epoch, t0, t1);
      if (has_pt) {
#pragma unroll 1
        for (int i = 0; i < 4; ++i) {  // envelopes 0, 1, 3, 5
          const int a = i < 2 ? i : 2 * i - 1;
          s.env[a][tid] = adsr_ff(tk, a, V, s.T);
        }
      }
      if (tid < 32) {
        u64 e0, e1;
        lookback_consume<u64>(vt, w, 0, epoch, e0, e1, hdr);
        if (tid == 0) { s.prefix[0][0] = e0; s.prefix[0][1] = e1; }
      }
      __syncthreads();
    }
    if (has_pt) {
      ff lfo0, lfo1;
#pragma unroll 1
      for (int l = 0; l < 2; ++l) {
        const ff th = fix64_to_ff(s.vs.lfo_p0[l] + s.prefix[0][l] + (l == 0 ? r0 : r1));
        const ff val = lfo_ff(th, l, s.env[3 + 2 * l][tid], V, s.T);
        if (l == 0) lfo0 = val; else lfo1 = val;
      }
      const ff src[4] = {s.env[0][tid], s.env[1][tid], lfo0, lfo1};
#pragma unroll
      for (int o = 0; o < 2; ++o) {
        ff acc = V.pitch_base[o];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc = ff_add(acc, ff_mul(V.pitch_w[o][q], src[q]));
        s.m[o][tid] = acc;
      }
      float srcf[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) srcf[q] = ff_to_float(src[q]);
      float amp[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        float acc = V.amp_w[k][0] * srcf[0];
#pragma unroll
        for (int q = 1; q < 4; ++q) acc = fmaf(V.amp_w[k][q], srcf[q], acc);
        amp[k] = acc;
      }
      s.ampv[tid] = make_float4(s.vs.gain[0] * amp[0], amp[1], s.vs.gain[2] * amp[2], 0.f);
    }
    __syncthreads();
    if (w == 0 && setups && n_windows > 1 && tid == 0) {
      // every part of the voice's set-up record is stored and fenced
      cuda::atomic_ref<unsigned int, cuda::thread_scope_device> f(setups[v].flag);
      f.store(((epoch & 0x3fffffffu) << 2) | 1u, cuda::memory_order_release);
    }

    // ---- 4. VCO phase over each control interval, scanned -----------------
    ff tot[2] = {ff_make(0.f), ff_make(0.f)};
    // the tile's first sample: interval k starts at sample ceil(k a / b)
    const int64_t s_tile =
        kGenR ? ((int64_t)k0 * vc.rate_a + vc.rate_b - 1) / vc.rate_b : (int64_t)k0 * R;
    if (tid < nseg) {
      float inc1 = 0.5f;
      if constexpr (kGenR) {
        const int64_t k = k0 + tid;
        const int64_t sk = (k * vc.rate_a + vc.rate_b - 1) / vc.rate_b;
        const int64_t sk1 = min(((k + 1) * vc.rate_a + vc.rate_b - 1) / vc.rate_b, N);
        const int Rk = (int)(sk1 - sk);
        // fraction of the way from point k to point k + 1: (s_k b - k a) / a
        const ff u0 = ff_mul_f(vc.inv_a, (float)(sk * vc.rate_b - k * vc.rate_a));
        s.sst[tid] = (int)(sk - s_tile);
        s.u0f[tid] = ff_to_float(u0);
        if (tid == nseg - 1) s.sst[nseg] = (int)(sk1 - s_tile);
        // the pitch at the interval's first sample, and the end point that
        // keeps the slope (m_(k+1) - m_k) / R per sample
#pragma unroll 1
        for (int o = 0; o < 2; ++o) {
          const ff dm = ff_sub(s.m[o][tid + 1], s.m[o][tid]);
          const ff mf = ff_add(s.m[o][tid], ff_mul(dm, u0));
          float inc;
          const ff t_o = vco_interval_ff(mf, ff_add(mf, dm), vc.r_f, Rk, vc.inv_R, vc.ln2_12R,
                                         vc.m_nyq_ff, vc.log2_440_over_sr, s.T, &s.seg[o][tid],
                                         &inc);
          if (o == 0) tot[0] = t_o; else tot[1] = t_o;
        }
      } else {
        const int64_t rem = N - (int64_t)(k0 + tid) * R;
        const int Rk = rem < R ? (int)rem : R;
        {  // the amplitudes' change per sample over this interval (linear upsampling)
          const float4 a = s.ampv[tid], b = s.ampv[tid + 1];
          s.aslope[tid] = make_float4((b.x - a.x) * invR, (b.y - a.y) * invR, (b.z - a.z) * invR, 0.f);
        }
#pragma unroll 1
        for (int o = 0; o < 2; ++o) {
          float inc;
          const ff t_o = vco_interval_ff(s.m[o][tid], s.m[o][tid + 1], (float)R, Rk, vc.inv_R,
                                         vc.ln2_12R, vc.m_nyq_ff, vc.log2_440_over_sr, s.T,
                                         &s.seg[o][tid], &inc);
          if (o == 0) tot[0] = t_o; else { tot[1] = t_o; inc1 = inc; }
        }
      }
      if constexpr (kGenR)  // kappa follows the (capped) frequency at the control point
        inc1 = ff_gt(s.m[1][tid], vc.m_nyq_ff)
                   ? 0.5f
                   : ff_to_float(inc_at_ff(s.m[1][tid], vc.log2_440_over_sr, s.T));
      // square-saw drive from the (capped) frequency at the interval start:
      // kappa = 1 + SR / (8 f) = 1 + 1 / (8 inc), at most 50
      const float kap = fminf((float)kBrightnessMax, 1.f + 0.125f / inc1);
      const float c1 = s.vs.gain[1] * s.vs.inv_1p_shape / tanhf(kap);
      s.sq[tid] = make_float4(kTwoLog2e * kap, c1, c1 * s.vs.shape, 0.f);
    }
    if constexpr (!kCarryF32) {
      u64 c0 = tid < nseg ? ff_to_fix64(tot[0]) : 0ull;
      u64 c1 = tid < nseg ? ff_to_fix64(tot[1]) : 0ull;
      u64 t0, t1;
      block_scan2_fix(c0, c1, s.warp_tot[1], t0, t1);
      if (tid < 32) {
        u64 e0, e1;
        lookback<u64>(vt, w, 1, epoch, t0, t1, e0, e1, hdr);
        if (tid == 0) { s.prefix[1][0] = e0; s.prefix[1][1] = e1; }
      }
      __syncthreads();
      if (tid < nseg) {
        s.seg[0][tid].phase0 = fix64_to_float(s.vs.vco_p0[0] + s.prefix[1][0] + c0);
        s.seg[1][tid].phase0 = fix64_to_float(s.vs.vco_p0[1] + s.prefix[1][1] + c1);
      }
    } else {
      // FP32 carries (precision study): the interval phases are summed in
      // float within the window and carried across windows in float.
      float c0 = tid < nseg ? ff_to_float(tot[0]) : 0.f;
      float c1 = tid < nseg ? ff_to_float(tot[1]) : 0.f;
      float t0, t1;
      block_scan2_f32(c0, c1, s.warp_tot_f, t0, t1);
      if (tid < 32) {
        float e0, e1;
        lookback<float>(vt, w, 1, epoch, carry_wrap(t0), carry_wrap(t1), e0, e1, hdr);
        if (tid == 0) { s.prefix_f[0] = e0; s.prefix_f[1] = e1; }
      }
      __syncthreads();
      if (tid < nseg) {
        s.seg[0][tid].phase0 = carry_wrap(fix64_to_float(s.vs.vco_p0[0]) + s.prefix_f[0] + c0);
        s.seg[1][tid].phase0 = carry_wrap(fix64_to_float(s.vs.vco_p0[1]) + s.prefix_f[1] + c1);
      }
    }
    __syncthreads();

    // ---- 5. audio ----------------------------------------------------------
    if constexpr (kGenR) {
      // fractional R: quads of the voice's own 4-sample grid. A work item is
      // (interval, chunk): the quad that straddles the interval's start is
      // evaluated on its own (each sample in the interval whose start it has
      // passed; a quad meets at most two intervals since R >= 4), the quads
      // inside the interval in runs of kGenG, their VCO phases stepped from
      // quad to quad as on the default path. The tile writes only its own
      // samples.
      const int n_t = s.sst[nseg];
      float* out_v = audio + (size_t)v * (size_t)N;
      const float invRg = ff_to_float(vc.inv_R);
      float vmax = 0.f;
      // a quad's four samples at tile-relative sample rel0: 16-byte stores
      // inside the tile, else the samples in [0, n_t) one by one
      auto store_quad = [&](int rel0, const float out4[4]) {
        const int64_t n0 = s_tile + rel0;
        if (vec_ok && rel0 >= 0 && rel0 + 3 < n_t) {
          if (!in_bounds(hdr, n0, N) || !in_bounds(hdr, n0 + 3, N)) return;
          if (kPeak) {
            *reinterpret_cast<float4*>(out_v + n0) = make_float4(out4[0], out4[1], out4[2], out4[3]);
            vmax = fmaxf(fmaxf(vmax, fmaxf(fabsf(out4[0]), fabsf(out4[1]))),
                         fmaxf(fabsf(out4[2]), fabsf(out4[3])));
          } else {
            __stcs(reinterpret_cast<float4*>(out_v + n0),
                   make_float4(out4[0], out4[1], out4[2], out4[3]));
          }
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (rel0 + i >= 0 && rel0 + i < n_t && in_bounds(hdr, n0 + i, N)) {
              out_v[n0 + i] = out4[i];
              if (kPeak) vmax = fmaxf(vmax, fabsf(out4[i]));
            }
        }
      };
      // the noise generator's key schedule and the products the voice fixes,
      // once per tile (the peak variant keeps the wide-product form)
      const PhiloxNoise pn =
          philox_noise_setup((uint32_t)g, (uint32_t)(g >> 32), kStreamNoise, key.x, key.y);
      auto noise_quad = [&](int rel0) {
        const uint32_t q = (uint32_t)((s_tile + rel0) >> 2);
        if constexpr (kPeak) {
          return philox4x32_10_wide(make_uint4((uint32_t)g, (uint32_t)(g >> 32), q, kStreamNoise), key);
        } else {
          uint32_t o[4];
          philox_noise(pn, q, o);
          return make_uint4(o[0], o[1], o[2], o[3]);
        }
      };
      // a quad on its own, its interval found from a float estimate
      auto single_quad = [&](int rel0) {
        const int r0 = max(rel0, 0);
        int si = min((int)((float)r0 * invRg), nseg - 1);
        while (si + 1 < nseg && s.sst[si + 1] <= r0) ++si;
        while (si > 0 && s.sst[si] > r0) --si;
        const int b1 = s.sst[si + 1];
        const bool two = si + 1 < nseg && rel0 + 3 >= b1;
        float psA[4], pqA[4], psB[4], pqB[4];
        vco_quad<false, false>(s.seg[0][si], rel0 - s.sst[si], psA);
        vco_quad<false, false>(s.seg[1][si], rel0 - s.sst[si], pqA);
        if (two) {
          vco_quad<false, false>(s.seg[0][si + 1], rel0 - b1, psB);
          vco_quad<false, false>(s.seg[1][si + 1], rel0 - b1, pqB);
        }
        const uint4 nz = noise_quad(rel0);
        const uint32_t nw[4] = {nz.x, nz.y, nz.z, nz.w};
        float out4[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int rel = rel0 + i;
          const bool in_b = two && rel >= b1;
          const int ii = in_b ? si + 1 : si;
          const float ps = in_b ? psB[i] : psA[i], pq = in_b ? pqB[i] : pqA[i];
          const float4 sq = s.sq[ii];
          const float4 A = s.ampv[ii], Bn = s.ampv[ii + 1];
          const float fj = fmaf((float)(rel - s.sst[ii]), invRg, s.u0f[ii]);
          const float x_sin = __sinf(kTwoPiF * ps);
          float sn, cs;
          __sincosf(kTwoPiF * pq, &sn, &cs);
          const float x_sq = square_saw_sc(sn, cs, sq.x, sq.y, sq.z);
          const float x_nz = fmaf((float)(nw[i] >> 8), 0x1p-23f, -1.f);
          out4[i] = fmaf(fmaf(fj, Bn.x - A.x, A.x), x_sin,
                         fmaf(fmaf(fj, Bn.y - A.y, A.y), x_sq, fmaf(fj, Bn.z - A.z, A.z) * x_nz));
        }
        store_quad(rel0, out4);
      };
      // first the quads that straddle an interval's start (or the tile's
      // start or end), one loop of their own so that the run loop below
      // carries none of their state
      for (int si = tid; si < nseg; si += NT) {
        const int a = s.sst[si], b = s.sst[si + 1];
        const int f = a + (int)((-(s_tile + a)) & 3);  // first grid quad at or after a
        const int nf = b - f >= 4 ? (b - f) >> 2 : 0;   // quads wholly inside [a, b)
        const int tail = f + 4 * nf;
        const int n_single = (f > a ? 1 : 0) + (si == nseg - 1 && tail < b ? 1 : 0);
#pragma unroll 1
        for (int k = 0; k < n_single; ++k) single_quad(k == 0 && f > a ? f - 4 : tail);
      }
      // then the whole quads: work items of kGenG quads of one interval
      constexpr int kGenG = 5;
      const int full_max = (int)(vc.r_f * 0.25f) + 2;  // bound on an interval's whole quads
      const int cpi = (full_max + kGenG - 1) / kGenG;   // chunks per interval
      for (int it = tid; it < nseg * cpi; it += NT) {
        const int si = it / cpi, c = it - si * cpi;
        const int a = s.sst[si], b = s.sst[si + 1];
        const int f = a + (int)((-(s_tile + a)) & 3);
        const int nf = b - f >= 4 ? (b - f) >> 2 : 0;
        const int q0 = c * kGenG, q1 = min(nf, q0 + kGenG);
        if (q0 >= q1) continue;
        const SegVco& sv0 = s.seg[0][si];
        const SegVco& sv1 = s.seg[1][si];
        // one whole quad from its VCO phases (radians)
        auto emit = [&](int rel0, const float ps[4], const float pq[4]) {
          const float4 sq = s.sq[si];
          const float4 A = s.ampv[si], Bn = s.ampv[si + 1];
          const float u0 = s.u0f[si];
          // amplitudes: A + (Bn - A) ((rel - a) / R + u0), linear in rel
          const float dx = (Bn.x - A.x) * invRg, dy = (Bn.y - A.y) * invRg, dz = (Bn.z - A.z) * invRg;
          const float fj0 = (float)(rel0 - a);
          const float a0x = fmaf(fj0, dx, fmaf(u0, Bn.x - A.x, A.x));
          const float a0y = fmaf(fj0, dy, fmaf(u0, Bn.y - A.y, A.y));
          const float a0z = fmaf(fj0, dz, fmaf(u0, Bn.z - A.z, A.z));
          const uint4 nz = noise_quad(rel0);
          const uint32_t nw[4] = {nz.x, nz.y, nz.z, nz.w};
          float out4[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float x_sin = __sinf(ps[i]);
            float sn, cs;
            __sincosf(pq[i], &sn, &cs);
            const float x_sq = square_saw_sc(sn, cs, sq.x, sq.y, sq.z);
            const float x_nz = fmaf((float)(nw[i] >> 8), 0x1p-23f, -1.f);  // 2u - 1, exact
            const float fi = (float)i;
            out4[i] = fmaf(fmaf(fi, dx, a0x), x_sin,
                           fmaf(fmaf(fi, dy, a0y), x_sq, fmaf(fi, dz, a0z) * x_nz));
          }
          store_quad(rel0, out4);
        };
        VcoRun r0, r1;
        const int j0 = f + 4 * q0 - a;  // the chunk's first sample in its interval
        if (vco_run_start(sv0, j0, 4 * (q1 - q0), r0) & vco_run_start(sv1, j0, 4 * (q1 - q0), r1)) {
#pragma unroll 1
          for (int q = q0; q < q1; ++q) {
            float ps[4], pq[4];
            vco_run_quad(sv0, r0, ps);
            vco_run_quad(sv1, r1, pq);
            emit(f + 4 * q, ps, pq);
          }
        } else {
          // a chunk that meets a Nyquist-cap boundary evaluates each quad on its own
#pragma unroll 1
          for (int q = q0; q < q1; ++q) {
            float ps[4], pq[4];
            vco_quad<false, true>(sv0, f + 4 * q - a, ps);
            vco_quad<false, true>(sv1, f + 4 * q - a, pq);
#pragma unroll
            for (int i = 0; i < 4; ++i) { ps[i] *= kTwoPiF; pq[i] *= kTwoPiF; }
            emit(f + 4 * q, ps, pq);
          }
        }
      }
      if (kPeak) publish_tile_peak(s, vt + w, vmax, epoch);
    } else {
      const int64_t t0 = (int64_t)k0 * R;                     // first sample of the tile
      float* out_t = audio + (size_t)v * (size_t)N + (size_t)t0;
      const int n_t = (int)min((int64_t)nseg * R, N - t0);   // samples in the tile
      const uint32_t q_t = (uint32_t)(t0 >> 2);               // its first quad (R % 4 == 0)
      // A work item is a run of G consecutive quads of one interval (G
      // divides the interval's quads): the VCO phase description is
      // evaluated for the run's first quad and stepped from quad to quad, in
      // radians. The interval's audio constants are read from shared memory
      // at each quad (holding them across the run costs registers the loop
      // has not got).
      const int G = qps % 5 == 0 ? 5 : qps % 4 == 0 ? 4 : qps % 3 == 0 ? 3 : qps % 2 == 0 ? 2 : 1;
      const int gpi = qps / G;
      const int ngr = nseg * gpi;
      float vmax = 0.f;  // largest |sample| this thread wrote (kPeak)
      for (int gi = tid; gi < ngr; gi += NT) {
        const int si = gi / gpi;
        const int j0 = (gi - si * gpi) * (4 * G);  // the run's first sample in its interval
        const int off0 = si * R + j0;
        if (off0 >= n_t) continue;
        const SegVco& sv0 = s.seg[0][si];
        const SegVco& sv1 = s.seg[1][si];
        // one quad of audio from its VCO phases (radians)
        auto emit = [&](int q, const float ps[4], const float pq[4]) {
          const float4 sq = s.sq[si];
          const float4 A = s.ampv[si], D = s.aslope[si];
          const int jq = j0 + 4 * q;
          const int off = off0 + 4 * q;
          const uint4 nc =
              make_uint4((uint32_t)g, (uint32_t)(g >> 32), q_t + (uint32_t)(off >> 2), kStreamNoise);
          // the peak variant: the wide-product form, which leaves it no spills
          const uint4 nz = kPeak ? philox4x32_10_wide(nc, key) : philox4x32_10(nc, key);
          const uint32_t nw[4] = {nz.x, nz.y, nz.z, nz.w};
          // amplitudes at the quad's first sample, then one step of the slope per sample
          const float fj0 = (float)jq;
          const float a0x = fmaf(fj0, D.x, A.x), a0y = fmaf(fj0, D.y, A.y), a0z = fmaf(fj0, D.z, A.z);
          float out4[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float x_sin = __sinf(ps[i]);
            float sn, cs;
            __sincosf(pq[i], &sn, &cs);
            const float x_sq = square_saw_sc(sn, cs, sq.x, sq.y, sq.z);
            const float x_nz = fmaf((float)(nw[i] >> 8), 0x1p-23f, -1.f);  // 2u - 1, exact
            const float fi = (float)i;
            out4[i] = fmaf(fmaf(fi, D.x, a0x), x_sin,
                           fmaf(fmaf(fi, D.y, a0y), x_sq, fmaf(fi, D.z, a0z) * x_nz));
          }
          if (vec_ok && off + 3 < n_t &&
              in_bounds(hdr, t0 + off, N) && in_bounds(hdr, t0 + off + 3, N)) {
            // streaming stores, except when the scaling pass reads the audio
            // back: then it stays in L2 for that pass
            if (kPeak)
              *reinterpret_cast<float4*>(out_t + off) = make_float4(out4[0], out4[1], out4[2], out4[3]);
            else
              __stcs(reinterpret_cast<float4*>(out_t + off),
                     make_float4(out4[0], out4[1], out4[2], out4[3]));
            if (kPeak)
              vmax = fmaxf(fmaxf(vmax, fmaxf(fabsf(out4[0]), fabsf(out4[1]))),
                           fmaxf(fabsf(out4[2]), fabsf(out4[3])));
          } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)
              if (off + i < n_t && in_bounds(hdr, t0 + off + i, N)) {
                out_t[off + i] = out4[i];
                if (kPeak) vmax = fmaxf(vmax, fabsf(out4[i]));
              }
          }
        };
        const int gq = min(G, (n_t - off0 + 3) >> 2);  // quads of the run inside the tile
        VcoRun r0, r1;
        // a run that meets a Nyquist-cap boundary evaluates each quad on its own
        const bool run = vco_run_start(sv0, j0, 4 * G, r0) & vco_run_start(sv1, j0, 4 * G, r1);
        if (kPeak) {
          // one loop for both cases (the peak variant's extra state leaves no
          // registers for two)
#pragma unroll 1
          for (int q = 0; q < gq; ++q) {
            float ps[4], pq[4];
            if (run) {
              vco_run_quad(sv0, r0, ps);
              vco_run_quad(sv1, r1, pq);
            } else {
              vco_quad<false, true>(sv0, j0 + 4 * q, ps);
              vco_quad<false, true>(sv1, j0 + 4 * q, pq);
#pragma unroll
              for (int i = 0; i < 4; ++i) { ps[i] *= kTwoPiF; pq[i] *= kTwoPiF; }
            }
            emit(q, ps, pq);
          }
        } else if (run) {
          // two loops: the stepped one carries no state of the other
#pragma unroll 1
          for (int q = 0; q < gq; ++q) {
            float ps[4], pq[4];
            vco_run_quad(sv0, r0, ps);
            vco_run_quad(sv1, r1, pq);
            emit(q, ps, pq);
          }
        } else {
#pragma unroll 1
          for (int q = 0; q < gq; ++q) {
            float ps[4], pq[4];
            vco_quad<false, true>(sv0, j0 + 4 * q, ps);
            vco_quad<false, true>(sv1, j0 + 4 * q, pq);
#pragma unroll
            for (int i = 0; i < 4; ++i) { ps[i] *= kTwoPiF; pq[i] *= kTwoPiF; }
            emit(q, ps, pq);
          }
        }
      }
      if (kPeak) publish_tile_peak(s, vt + w, vmax, epoch);
    }
  }
  persistent_finish(hdr);
}

}  // namespace

namespace {

// The buffers and scratch of one fused launch, for the overlap check: the
// CTAs of a launch that overlaps its predecessor run their work items while
// the predecessor's last wave is still running (they wait for it only before
// releasing their own dependents), so the two must share no scratch and no
// buffer that either of them writes.
struct FusedLaunchRecord {
  const void* hdr = nullptr;
  uintptr_t lo[5] = {}, hi[5] = {};  // params_in, audio, params_out, peak, silent
  bool writes[5] = {};
  bool other = false;  // the last launch was another kernel that releases its successor early
};

bool launches_conflict(const FusedLaunchRecord& a, const FusedLaunchRecord& b) {
  if (a.other || b.other || a.hdr == b.hdr) return true;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j)
      if ((a.writes[i] || b.writes[j]) && a.lo[i] < a.hi[i] && b.lo[j] < b.hi[j] &&
          a.lo[i] < b.hi[j] && b.lo[j] < a.hi[i])
        return true;
  return false;
}

std::mutex g_fused_launch_mu;
std::unordered_map<cudaStream_t, FusedLaunchRecord> g_last_fused_launch;  // per stream

void set_range(FusedLaunchRecord& r, int k, const void* p, size_t bytes, bool writes) {
  if (!p || bytes == 0) return;
  r.lo[k] = reinterpret_cast<uintptr_t>(p);
  r.hi[k] = r.lo[k] + bytes;
  r.writes[k] = writes;
}

}  // namespace

size_t fused_voice_setup_bytes() { return sizeof(VoiceSetupRecord); }

void note_early_release_launch(cudaStream_t st) {
  FusedLaunchRecord rec;
  rec.other = true;
  std::lock_guard<std::mutex> lock(g_fused_launch_mu);
  g_last_fused_launch[st] = rec;
}

int fused_max_active_blocks_per_sm() {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, render_fused_kernel<false, false, false>, NT, 0);
  return n;
}

cudaError_t launch_render_fused(const VoiceConst& vc, uint64_t seed, uint64_t first, int split,
                                int batch, const float* params_in, float* audio,
                                float* params_out, ScratchHeader* hdr, TileState* tiles,
                                int grid, cudaStream_t stream, const PeakNormArgs* norm,
                                uint64_t seed_step, int sub_batch, bool overlap_previous,
                                void* voice_setups) {
  const int n_windows = windows_per_voice(vc.K);
  const int total = batch * n_windows;
  grid = grid < total ? grid : total;
  const PeakNormArgs nz = norm ? *norm : PeakNormArgs{0.f, nullptr, nullptr};
  if (sub_batch <= 0) sub_batch = batch;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  FusedLaunchRecord rec;
  rec.hdr = hdr;
  const size_t nv = (size_t)batch;
  set_range(rec, 0, params_in, nv * kNumParams * sizeof(float), false);
  set_range(rec, 1, audio, nv * (size_t)vc.n_samples * sizeof(float), true);
  set_range(rec, 2, params_out, nv * kNumParams * sizeof(float), true);
  set_range(rec, 3, nz.peak_out, nv * sizeof(float), true);
  set_range(rec, 4, nz.silent_out, nv * sizeof(int32_t), true);
  bool overlap = false;
  {
    std::lock_guard<std::mutex> lock(g_fused_launch_mu);
    auto it = g_last_fused_launch.find(stream);
    overlap = overlap_previous &&
              (it == g_last_fused_launch.end() || !launches_conflict(it->second, rec));
    g_last_fused_launch[stream] = rec;
  }
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = overlap ? 1 : 0;
  VoiceSetupRecord* setups = static_cast<VoiceSetupRecord*>(voice_setups);
#define SYNTH_FUSED_ARGS vc, seed, first, split, batch, params_in, audio, params_out, hdr, tiles, \
                         n_windows, nz, seed_step, sub_batch, setups
  cudaError_t e;
  if (vc.general_r) {  // fractional R (never with FP32 carries)
    if (norm) e = cudaLaunchKernelEx(&cfg, render_fused_kernel<false, true, true>, SYNTH_FUSED_ARGS);
    else e = cudaLaunchKernelEx(&cfg, render_fused_kernel<false, false, true>, SYNTH_FUSED_ARGS);
  } else if (vc.carry_fp32) {
    if (norm) e = cudaLaunchKernelEx(&cfg, render_fused_kernel<true, true, false>, SYNTH_FUSED_ARGS);
    else e = cudaLaunchKernelEx(&cfg, render_fused_kernel<true, false, false>, SYNTH_FUSED_ARGS);
  } else {
    if (norm) e = cudaLaunchKernelEx(&cfg, render_fused_kernel<false, true, false>, SYNTH_FUSED_ARGS);
    else e = cudaLaunchKernelEx(&cfg, render_fused_kernel<false, false, false>, SYNTH_FUSED_ARGS);
  }
#undef SYNTH_FUSED_ARGS
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace synth
