// spectral.cu -- the multi-resolution log-magnitude STFT distance (the
// paper's multi-scale spectrogram distance, Sec. 4, Table 2) and its gradient with
// respect to the audio, on warp-level FP32 FFTs (fft_warp.cuh): periodic Hann
// window, hop n/4, centred frames with reflect padding;
// L_v = sum_n mean_(bins, frames) |log(|X| + eps) - log(|Y| + eps)|.
//
// One kernel per resolution and pass. A CTA takes a voice and a group of
// frames, stages the padded audio the group covers in shared memory, and
// each warp transforms 32 / R frames at a time (n = 64 R). The target pass
// stores log(|Y| + eps) per bin; the loss pass forms d = log(|X| + eps) -
// log(|Y| + eps), sums |d| per voice and, for the gradient, the spectrum
// G_k = sign(d_k) / ((|X_k| + eps) |X_k|) X_k / (F bins), whose inverse real
// DFT times the window is the gradient of the frame:
//   dframe[t] = w[t] sum_(k = 0 .. n/2) Re(G_k e^(2 pi i k t / n)).
// It runs the forward decomposition in reverse (a 32-point inverse DFT per
// lane, twiddles, the transpose back, the R-point inverse DFTs) on the
// packed sequence z[m] = dframe[2m] + i dframe[2m+1] / w. The CTA sums its
// frames' gradients into the padded segment they cover (in shared memory)
// and writes that partial; one gather over all resolutions then adds the
// partials of the (at most two) segments covering each padded position and
// folds the reflect padding back. Also here: the Slaney mel filterbank of
// the log-mel features.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "fft_warp.cuh"
#include "launch_config.h"
#include "mbarrier.cuh"
#include "spectral.h"

namespace synth {

namespace {

using fftw::bitrev;

constexpr int kWarpsMr = 8;
constexpr int kThreadsMr = 32 * kWarpsMr;
constexpr int kLdMr = 33;  // padded row of the per-warp transpose buffer

template <int R>
struct MrCfg {
  static constexpr int M = 32 * R;            // complex points per frame
  static constexpr int n = 2 * M;             // n_fft
  static constexpr int hop = n / 4;
  static constexpr int ldl = M + 4;  // row stride of the target log-magnitudes (bins M + 1,
                                     // padded to a 16-byte multiple for bulk copies)
  static constexpr int FPW = 32 / R;          // frames per warp pass
  static constexpr int G = kWarpsMr * FPW;    // frames per work item: one pass per warp
  static constexpr int seg = (G - 1) * hop + n;
};

template <int R>
struct __align__(16) MrSmem {
  float seg[2][MrCfg<R>::seg];  // this item's padded audio and the next one's (prefetched)
  float buf[kWarpsMr][32 * kLdMr];
  float2 win[MrCfg<R>::M];     // window at samples (2m, 2m + 1)
  float2 tw[R * 32];           // e^(-2 pi i b k1 / M) at [k1][b]
  float2 twi[32 * R];          // e^(+2 pi i b k1 / M) at [b][k1]
  float2 post[MrCfg<R>::M];    // e^(-2 pi i k / n)
  float red[kWarpsMr];
  uint64_t mbar[kWarpsMr];     // per warp: its frames' target rows have arrived
};

constexpr long long kMrWaitLimit = 1ll << 24;

struct MrTables {
  const float2* win;
  const float2* tw;
  const float2* twi;
  const float2* post;
};

enum MrMode { kMrTarget = 0, kMrLoss = 1, kMrLossGrad = 2 };

// Conditional move of the upper half of a lane's 32 values one slot down
// (slot s holds k2 = s in register bitrev<32>(s)): slot 16..30 <- 17..31,
// slot 31 <- 16, or back. On lanes with k1 = 0 this makes the partner of the
// value in slot j (k2' = 32 - k2 mod 32) sit in slot 31 - j, as it does on
// every other lane (k2' = 31 - k2).
__device__ __forceinline__ void rotate_upper(float (&x)[32], bool on, bool back) {
  if (!back) {
    const float t = x[bitrev<32>(16)];
#pragma unroll
    for (int s = 16; s < 31; ++s) x[bitrev<32>(s)] = on ? x[bitrev<32>(s + 1)] : x[bitrev<32>(s)];
    x[bitrev<32>(31)] = on ? t : x[bitrev<32>(31)];
  } else {
    const float t = x[bitrev<32>(31)];
#pragma unroll
    for (int s = 30; s >= 16; --s) x[bitrev<32>(s + 1)] = on ? x[bitrev<32>(s)] : x[bitrev<32>(s + 1)];
    x[bitrev<32>(16)] = on ? t : x[bitrev<32>(16)];
  }
}

// Stages the padded samples base .. base + len - 1 of signal x (sample j of
// the segment = x[reflect(base + j)]) in dst: 16-byte cp.async copies where a
// 4-sample run lies inside the signal, plain loads where it is reflected;
// the copies form one commit group.
__device__ __forceinline__ void stage_segment(float* dst, const float* __restrict__ x, int N,
                                              bool vec, int base, int len) {
  for (int j = 4 * threadIdx.x; j < len; j += 4 * kThreadsMr) {
    const int i0 = base + j;
    if (vec && i0 >= 0 && i0 + 3 < N) {
      const unsigned int d = (unsigned int)__cvta_generic_to_shared(dst + j);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(x + i0) : "memory");
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int i = i0 + q;
        i = i < 0 ? -i : i;
        i = i >= N ? 2 * (N - 1) - i : i;
        dst[j + q] = __ldg(x + i);
      }
    }
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int R>
__global__ void __launch_bounds__(kThreadsMr, 2)
    mr_fft_kernel(const float* __restrict__ sig, int N, int F, int batch, MrTables t, float eps,
                  float scale, int mode, float* __restrict__ logy, double* __restrict__ loss_item,
                  float* __restrict__ part, unsigned int* __restrict__ err) {
  using C = MrCfg<R>;
  extern __shared__ __align__(16) unsigned char mr_raw[];
  MrSmem<R>& S = *reinterpret_cast<MrSmem<R>*>(mr_raw);
  for (int j = threadIdx.x; j < C::M; j += kThreadsMr) {
    S.win[j] = __ldg(t.win + j);
    S.post[j] = __ldg(t.post + j);
  }
  for (int j = threadIdx.x; j < 32 * R; j += kThreadsMr) {
    S.tw[j] = __ldg(t.tw + j);
    S.twi[j] = __ldg(t.twi + j);
  }
  if ((threadIdx.x & 31) == 0) mbar::init(&S.mbar[threadIdx.x >> 5], 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  uint32_t mb_phase = 0;
  const bool vec = (N & 3) == 0 && (reinterpret_cast<uintptr_t>(sig) & 15) == 0;
  const int groups = (F + C::G - 1) / C::G;
  const int items = groups * batch;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int phi = lane / R, k1 = lane % R;            // this lane's frame and k1 after the transpose
  const int src = phi * R + ((R - k1) & (R - 1));     // the lane holding Z[M - k]
  const bool self = k1 == 0;
  float* B = S.buf[warp];

  auto stage = [&](int it, float* dst) {
    const int vv = it / groups, ff = (it - vv * groups) * C::G;
    stage_segment(dst, sig + (size_t)vv * N, N, vec, ff * C::hop - C::n / 2,
                  (min(C::G, F - ff) - 1) * C::hop + C::n);
  };
  if ((int)blockIdx.x < items) stage(blockIdx.x, S.seg[0]);
  int cur = 0;
  for (int item = blockIdx.x; item < items; item += gridDim.x, cur ^= 1) {
    const int v = item / groups, f0 = (item - v * groups) * C::G;
    const int Gi = min(C::G, F - f0);
    const int len = (Gi - 1) * C::hop + C::n;
    float* sg = S.seg[cur];
    __syncthreads();  // the previous item is done with the other buffer and S.red
    // prefetch the next item's segment, then wait for this one's copies
    if (item + (int)gridDim.x < items) {
      stage(item + gridDim.x, S.seg[cur ^ 1]);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();

    float acc = 0.f;  // sum of |d| over this warp's bins
    // one pass per warp: frames lf0 .. lf0 + FPW - 1 of the item
    const int lf0 = warp * C::FPW;
    float re[32], im[32];
    if (lf0 < Gi) {
      // ---- forward: z[32 a + lane] of frames lf0 .. lf0 + FPW - 1, windowed
#pragma unroll
      for (int fr = 0; fr < C::FPW; ++fr) {
        const int lf = min(lf0 + fr, Gi - 1);
        const float2* s2 = reinterpret_cast<const float2*>(sg + lf * C::hop);
#pragma unroll
        for (int a = 0; a < R; ++a) {
          const float2 sv = s2[32 * a + lane];
          const float2 wv = S.win[32 * a + lane];
          re[fr * R + a] = sv.x * wv.x;
          im[fr * R + a] = sv.y * wv.y;
        }
      }
      fftw::dft_frames<R>(re, im);
#pragma unroll
      for (int fr = 0; fr < C::FPW; ++fr)
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int kk = bitrev<R>(r);
          if (kk != 0) {
            const float2 w = S.tw[32 * kk + lane];
            const float yr = re[fr * R + r], yi = im[fr * R + r];
            re[fr * R + r] = fmaf(yr, w.x, -yi * w.y);
            im[fr * R + r] = fmaf(yr, w.y, yi * w.x);
          }
        }
#pragma unroll
      for (int fr = 0; fr < C::FPW; ++fr)
#pragma unroll
        for (int r = 0; r < R; ++r) B[(fr * R + bitrev<R>(r)) * kLdMr + lane] = re[fr * R + r];
      __syncwarp();
#pragma unroll
      for (int b = 0; b < 32; ++b) re[b] = B[lane * kLdMr + b];
      __syncwarp();
#pragma unroll
      for (int fr = 0; fr < C::FPW; ++fr)
#pragma unroll
        for (int r = 0; r < R; ++r) B[(fr * R + bitrev<R>(r)) * kLdMr + lane] = im[fr * R + r];
      __syncwarp();
#pragma unroll
      for (int b = 0; b < 32; ++b) im[b] = B[lane * kLdMr + b];
      __syncwarp();
      // the target rows of this warp's frames into B (free until the inverse
      // transposes) by one bulk copy, in flight during the 32-point DFTs
      if (mode != kMrTarget && lane == 0) {
        const int rows = min(C::FPW, Gi - lf0);
        const uint32_t bytes = (uint32_t)(rows * C::ldl * sizeof(float));
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar::expect_tx(&S.mbar[warp], bytes);
        mbar::bulk_g2s(B, logy + ((size_t)v * F + f0 + lf0) * C::ldl, bytes, &S.mbar[warp]);
      }
      fftw::dft<32, 0>(re, im);  // Z[k1 + R k2] of frame phi in register bitrev<32>(k2)
      if (mode != kMrTarget) {
        if (!mbar::wait(&S.mbar[warp], mb_phase, kMrWaitLimit) && lane == 0) atomicOr(err, 1u);
        mb_phase ^= 1;
      }
      const float* ly = B + phi * C::ldl;  // this lane's frame's target row

      const int lf = lf0 + phi;
      const bool valid = lf < Gi;
      const size_t row = (size_t)v * F + f0 + (valid ? lf : 0);
      rotate_upper(re, self, false);
      rotate_upper(im, self, false);
      // slot pairs (j, 31 - j): their values are partners of the partner
      // lane's slots (31 - j, j); on k1 = 0 lanes slots j and 31 - j are
      // partners of each other (slot 0: k = 0 with the Nyquist bin; slot 31
      // after the rotation: k = M / 2, its own partner)
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int ra = bitrev<32>(j), rb = bitrev<32>(31 - j);
        const int k2a = j, k2b = self ? (j == 0 ? 16 : 32 - j) : 31 - j;
        float par = __shfl_sync(0xffffffffu, re[rb], src), pai = __shfl_sync(0xffffffffu, im[rb], src);
        float pbr = __shfl_sync(0xffffffffu, re[ra], src), pbi = __shfl_sync(0xffffffffu, im[ra], src);
        if (self) {
          par = j == 0 ? re[ra] : re[rb];
          pai = j == 0 ? im[ra] : im[rb];
          pbr = j == 0 ? re[rb] : re[ra];
          pbi = j == 0 ? im[rb] : im[ra];
        }
        float gr[2], gi[2];
        float nyq_g = 0.f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int rr = h == 0 ? ra : rb;
          const int k2 = h == 0 ? k2a : k2b;
          const int k = k1 + R * k2;
          const float zr = re[rr], zi = im[rr];
          const float pr = h == 0 ? par : pbr, pi = h == 0 ? pai : pbi;
          const float ar = zr + pr, ai = zi - pi;  // Z + conj(P)
          const float cr = zi + pi, ci = pr - zr;  // -i (Z - conj(P))
          const float2 w = S.post[k];
          const float xr = 0.5f * (ar + fmaf(w.x, cr, -w.y * ci));
          const float xi = 0.5f * (ai + fmaf(w.x, ci, w.y * cr));
          // |X| by the reciprocal square root, log by the SFU: both well
          // inside the distance's and the gradient's tolerances
          const float p2 = fmaf(xr, xr, xi * xi);
          const float mag = p2 > 0.f ? p2 * rsqrtf(p2) : 0.f;
          const float lm = __logf(mag + eps);
          gr[h] = 0.f;
          gi[h] = 0.f;
          if (mode == kMrTarget) {
            if (valid) logy[row * C::ldl + k] = lm;
          } else {
            const float d = lm - (valid ? ly[k] : lm);
            acc += fabsf(d);
            if (mag > 0.f && d != 0.f) {
              const float g = __fdividef(d > 0.f ? scale : -scale, (mag + eps) * mag);
              gr[h] = g * xr;
              gi[h] = g * xi;
            }
          }
          if (k == 0) {  // the Nyquist bin X[M] = Re Z[0] - Im Z[0] (real)
            const float xn = zr - zi, mn = fabsf(xn), ln = __logf(mn + eps);
            if (mode == kMrTarget) {
              if (valid) logy[row * C::ldl + C::M] = ln;
            } else {
              const float d = ln - (valid ? ly[C::M] : ln);
              acc += fabsf(d);
              if (mn > 0.f && d != 0.f) nyq_g = __fdividef(d > 0.f ? scale : -scale, (mn + eps) * mn) * xn;
            }
          }
        }
        if (mode == kMrLossGrad) {
          // inverse packing: Zp_k = A_k + i B_k with A_k = (G_k + conj G_(M-k)) / 2,
          // B_k = (G_k - conj G_(M-k)) / 2 e^(2 pi i k / n); k = 0 pairs with
          // the Nyquist bin: A_0 = Re G_0 + G_M, B_0 = Re G_0 - G_M
          float qar = __shfl_sync(0xffffffffu, gr[1], src), qai = __shfl_sync(0xffffffffu, gi[1], src);
          float qbr = __shfl_sync(0xffffffffu, gr[0], src), qbi = __shfl_sync(0xffffffffu, gi[0], src);
          if (self) {
            qar = j == 0 ? gr[0] : gr[1];
            qai = j == 0 ? gi[0] : gi[1];
            qbr = j == 0 ? gr[1] : gr[0];
            qbi = j == 0 ? gi[1] : gi[0];
          }
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int rr = h == 0 ? ra : rb;
            const int k2 = h == 0 ? k2a : k2b;
            const int k = k1 + R * k2;
            const float g_r = gr[h], g_i = gi[h];
            const float q_r = h == 0 ? qar : qbr, q_i = h == 0 ? qai : qbi;
            float Ar = 0.5f * (g_r + q_r), Ai = 0.5f * (g_i - q_i);
            const float Dr = 0.5f * (g_r - q_r), Di = 0.5f * (g_i + q_i);
            const float2 w = S.post[k];  // e^(2 pi i k / n) = conj(w)
            float Br = fmaf(Dr, w.x, Di * w.y), Bi = fmaf(Di, w.x, -Dr * w.y);
            if (k == 0) {
              Ar = g_r + nyq_g;
              Ai = 0.f;
              Br = g_r - nyq_g;
              Bi = 0.f;
            }
            re[rr] = Ar - Bi;  // A + i B
            im[rr] = Ai + Br;
          }
        }
      }
      if (mode == kMrLossGrad) {
      // ---- inverse: z[m] = sum_k Zp_k e^(2 pi i k m / M), m = 32 a + b
      rotate_upper(re, self, true);
      rotate_upper(im, self, true);
      // 32-point inverse DFT over k2 (the swap of real and imaginary parts
      // turns the forward transform into the inverse one)
      {
        float tr[32], ti[32];
#pragma unroll
        for (int k2 = 0; k2 < 32; ++k2) {
          tr[k2] = re[bitrev<32>(k2)];
          ti[k2] = im[bitrev<32>(k2)];
        }
        fftw::dft<32, 0>(ti, tr);  // T[b] in register bitrev<32>(b)
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          const int b = bitrev<32>(r);
          float yr = tr[r], yi = ti[r];
          if (b != 0 && k1 != 0) {
            const float2 w = S.twi[b * R + k1];
            const float t0 = fmaf(yr, w.x, -yi * w.y);
            yi = fmaf(yr, w.y, yi * w.x);
            yr = t0;
          }
          re[b] = yr;
          im[b] = yi;
        }
      }
      // transpose back: lane (phi, k1) row, column b
#pragma unroll
      for (int b = 0; b < 32; ++b) B[lane * kLdMr + b] = re[b];
      __syncwarp();
#pragma unroll
      for (int fr = 0; fr < C::FPW; ++fr)
#pragma unroll
        for (int q = 0; q < R; ++q) re[fr * R + q] = B[(fr * R + q) * kLdMr + lane];
      __syncwarp();
#pragma unroll
      for (int b = 0; b < 32; ++b) B[lane * kLdMr + b] = im[b];
      __syncwarp();
#pragma unroll
      for (int fr = 0; fr < C::FPW; ++fr)
#pragma unroll
        for (int q = 0; q < R; ++q) im[fr * R + q] = B[(fr * R + q) * kLdMr + lane];
      __syncwarp();
      fftw::dft_frames<R>(im, re);  // z[32 a + lane] of frame fr in register fr R + bitrev<R>(a)
      }
    }
    if (mode == kMrLossGrad) {
      // the item's frame gradients (times the window) summed into its padded
      // segment, over the audio it no longer needs; frames four hops apart do
      // not overlap, so the four residue classes of the frame index add in
      // turn (a fixed order: the sums are deterministic)
      __syncthreads();
      for (int j = 4 * threadIdx.x; j < len; j += 4 * kThreadsMr)
        *reinterpret_cast<float4*>(sg + j) = make_float4(0.f, 0.f, 0.f, 0.f);
      __syncthreads();
#pragma unroll
      for (int c = 0; c < 4; ++c) {
#pragma unroll
        for (int fr = 0; fr < C::FPW; ++fr) {
          const int lf = lf0 + fr;
          if (lf < Gi && (lf & 3) == c) {
            float2* a = reinterpret_cast<float2*>(sg + lf * C::hop);
#pragma unroll
            for (int r = 0; r < R; ++r) {
              const int m = 32 * bitrev<R>(r) + lane;
              const float2 wv = S.win[m];
              float2 o = a[m];
              o.x = fmaf(re[fr * R + r], wv.x, o.x);
              o.y = fmaf(im[fr * R + r], wv.y, o.y);
              a[m] = o;
            }
          }
        }
        __syncthreads();
      }
      float4* dst = reinterpret_cast<float4*>(part + (size_t)item * C::seg);
      for (int j = threadIdx.x; 4 * j < len; j += kThreadsMr)
        dst[j] = reinterpret_cast<const float4*>(sg)[j];
    }
    if (mode != kMrTarget) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) S.red[warp] = acc;
      __syncthreads();
      if (threadIdx.x == 0) {
        double tot = 0.0;
#pragma unroll
        for (int w = 0; w < kWarpsMr; ++w) tot += (double)S.red[w];
        loss_item[item] = tot * (double)scale;  // summed per voice in item order later
      }
    }
  }
}

// The audio gradient from the items' segment partials of every resolution:
// grad[v][s] = sum over resolutions, over the padded positions p with
// reflect(p - n/2) = s (one, or two near the ends), over the items whose
// segment covers p (one or two: segments of (G + 3) hops start every G hops)
// of the partial at p. One thread per sample, a fixed summation order.
struct OlaRes {
  const float* part;  // [batch][groups][seg]
  int n, hop, G, groups, seg, F;
};
struct OlaArgs {
  OlaRes r[8];
  int n_res;
};

__device__ __forceinline__ float ola_sample(const OlaArgs& a, int N, int v, int s) {
  float acc = 0.f;
  for (int k = 0; k < a.n_res; ++k) {
    const OlaRes& R = a.r[k];
    const int pad = R.n / 2, stride = R.G * R.hop;
    const float* pv = R.part + (size_t)v * R.groups * R.seg;
    int pre[3];
    int np = 0;
    pre[np++] = s + pad;
    if (s >= 1 && s <= pad) pre[np++] = pad - s;
    if (s <= N - 2 && 2 * (N - 1) - s + pad < N + 2 * pad && 2 * (N - 1) - s >= N)
      pre[np++] = 2 * (N - 1) - s + pad;
    for (int j = 0; j < np; ++j) {
      const int p = pre[j];
      const int i = min(p / stride, R.groups - 1);
      for (int q = i; q >= 0 && q >= i - 1; --q) {
        const int off = p - q * stride;
        const int len = (min(R.G, R.F - q * R.G) - 1) * R.hop + R.n;
        if (off >= 0 && off < len) acc += pv[(size_t)q * R.seg + off];
      }
    }
  }
  return acc;
}

// Four samples per thread: away from the ends (no reflected positions) the
// four padded positions s + n/2 share their items and segment bounds (all
// multiples of 4), so each covering segment contributes one 16-byte load.
__global__ void mr_ola_gather(OlaArgs a, int N, int pad_max, float* __restrict__ grad) {
  const int v = blockIdx.y;
  const int n4 = (N + 3) / 4;
  const bool vec = (N & 3) == 0 && (reinterpret_cast<uintptr_t>(grad) & 15) == 0;
  for (int i4 = blockIdx.x * blockDim.x + threadIdx.x; i4 < n4; i4 += gridDim.x * blockDim.x) {
    const int s0 = 4 * i4;
    if (vec && s0 > pad_max && s0 + 3 <= N - 2 - pad_max) {
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int k = 0; k < a.n_res; ++k) {
        const OlaRes& R = a.r[k];
        const int stride = R.G * R.hop, p0 = s0 + R.n / 2;
        const float* pv = R.part + (size_t)v * R.groups * R.seg;
        const int i = min(p0 / stride, R.groups - 1);
        for (int q = i; q >= 0 && q >= i - 1; --q) {
          const int off = p0 - q * stride;
          const int len = (min(R.G, R.F - q * R.G) - 1) * R.hop + R.n;
          if (off >= 0 && off < len) {
            const float4 t = *reinterpret_cast<const float4*>(pv + (size_t)q * R.seg + off);
            acc.x += t.x;
            acc.y += t.y;
            acc.z += t.z;
            acc.w += t.w;
          }
        }
      }
      *reinterpret_cast<float4*>(grad + (size_t)v * N + s0) = acc;
    } else {
      for (int s = s0; s < min(s0 + 4, N); ++s) grad[(size_t)v * N + s] = ola_sample(a, N, v, s);
    }
  }
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// FFT tables of one resolution (n = 64 R), built on the host in FP64.
size_t mr_table_bytes(int R) {
  const int M = 32 * R;
  return al256(sizeof(float2) * M) * 2 + al256(sizeof(float2) * 32 * R) * 2;
}

MrTables mr_tables(int R, const char* p) {
  const int M = 32 * R;
  MrTables t;
  t.win = reinterpret_cast<const float2*>(p);
  t.post = reinterpret_cast<const float2*>(p + al256(sizeof(float2) * M));
  t.tw = reinterpret_cast<const float2*>(p + 2 * al256(sizeof(float2) * M));
  t.twi = reinterpret_cast<const float2*>(p + 2 * al256(sizeof(float2) * M) +
                                          al256(sizeof(float2) * 32 * R));
  return t;
}

cudaError_t mr_tables_fill(int R, void* dst, cudaStream_t st) {
  const double pi = 3.14159265358979323846;
  const int M = 32 * R, n = 2 * M;
  std::vector<char> host(mr_table_bytes(R), 0);
  const MrTables t = mr_tables(R, host.data());
  float2* win = const_cast<float2*>(t.win);
  float2* post = const_cast<float2*>(t.post);
  float2* tw = const_cast<float2*>(t.tw);
  float2* twi = const_cast<float2*>(t.twi);
  for (int m = 0; m < M; ++m) {
    win[m] = make_float2((float)(0.5 - 0.5 * std::cos(2.0 * pi * (2 * m) / n)),
                         (float)(0.5 - 0.5 * std::cos(2.0 * pi * (2 * m + 1) / n)));
    const double a = -2.0 * pi * m / n;
    post[m] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  for (int k1 = 0; k1 < R; ++k1)
    for (int b = 0; b < 32; ++b) {
      const double a = 2.0 * pi * (double)((b * k1) % M) / M;
      tw[32 * k1 + b] = make_float2((float)std::cos(a), (float)-std::sin(a));
      twi[b * R + k1] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
  return cudaMemcpyAsync(dst, host.data(), host.size(), cudaMemcpyHostToDevice, st);
}

int r_of(int n_fft) { return n_fft == 512 ? 8 : n_fft == 1024 ? 16 : n_fft == 2048 ? 32 : 0; }

template <int R>
cudaError_t mr_launch(const float* sig, int N, int F, int batch, const char* tables, float eps,
                      float scale, int mode, float* logy, double* loss_item, float* part,
                      unsigned int* err, cudaStream_t st) {
  const int smem = (int)sizeof(MrSmem<R>);
  int grid_cap = 0;  // resident CTAs on the current device
  const cudaError_t ge =
      resident_grid(reinterpret_cast<const void*>(mr_fft_kernel<R>), kThreadsMr, smem, &grid_cap);
  if (ge != cudaSuccess) return ge;
  const int64_t items = (int64_t)((F + MrCfg<R>::G - 1) / MrCfg<R>::G) * batch;
  if (items >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
  const int grid = (int)std::min<int64_t>(items, grid_cap);
  mr_fft_kernel<R><<<grid, kThreadsMr, smem, st>>>(sig, N, F, batch, mr_tables(R, tables), eps,
                                                   scale, mode, logy, loss_item, part, err);
  return cudaGetLastError();
}

cudaError_t mr_pass(int n_fft, const float* sig, int N, int F, int batch, const char* tables,
                    float eps, float scale, int mode, float* logy, double* loss_item, float* part,
                    unsigned int* err, cudaStream_t st) {
#define SYNTH_MR_ARGS sig, N, F, batch, tables, eps, scale, mode, logy, loss_item, part, err, st
  switch (r_of(n_fft)) {
    case 8: return mr_launch<8>(SYNTH_MR_ARGS);
    case 16: return mr_launch<16>(SYNTH_MR_ARGS);
    case 32: return mr_launch<32>(SYNTH_MR_ARGS);
    default: return cudaErrorInvalidValue;
  }
#undef SYNTH_MR_ARGS
}

// frames per work item and padded segment length of a resolution
int mr_group(int n_fft) { return kWarpsMr * (32 / std::max(1, r_of(n_fft))); }
int mr_seg(int n_fft) { return (mr_group(n_fft) - 1) * (n_fft / 4) + n_fft; }

}  // namespace

int stft_frames(int64_t N, int n_fft) { return 1 + (int)(N / (n_fft / 4)); }

// Slaney mel band edges in Hz: n_mels + 2 points equally spaced on the mel
// scale (linear below 1 kHz, logarithmic above) from 0 to sr / 2.
std::vector<double> mel_edges_host(int n_mels, double sr) {
  auto hz_to_mel = [](double f) {
    return f < 1000.0 ? 3.0 * f / 200.0 : 15.0 + 27.0 * std::log(f / 1000.0) / std::log(6.4);
  };
  auto mel_to_hz = [](double m) {
    return m < 15.0 ? 200.0 * m / 3.0 : 1000.0 * std::exp((m - 15.0) * std::log(6.4) / 27.0);
  };
  std::vector<double> edges(n_mels + 2);
  const double m_hi = hz_to_mel(sr / 2.0);
  for (int i = 0; i < n_mels + 2; ++i) edges[i] = mel_to_hz(m_hi * i / (n_mels + 1));
  return edges;
}

// Slaney mel filterbank [n_mels][ld], built on the host in FP64: triangles
// between the mel-spaced edges, unit area in Hz.
std::vector<float> mel_filterbank_host(int n_fft, int n_mels, double sr, int ld) {
  const int nb = n_fft / 2 + 1;
  const std::vector<double> edges = mel_edges_host(n_mels, sr);
  std::vector<float> fb((size_t)n_mels * ld, 0.f);
  for (int i = 0; i < n_mels; ++i) {
    const double lo = edges[i], c = edges[i + 1], hi = edges[i + 2];
    for (int k = 0; k < nb; ++k) {
      const double f = k * sr / n_fft;
      const double w = std::fmax(0.0, std::fmin((f - lo) / (c - lo), (hi - f) / (hi - c)));
      fb[(size_t)i * ld + k] = (float)(w * 2.0 / (hi - lo));
    }
  }
  return fb;
}

// ---------------------------------------------------------------- MR-STFT
namespace {
struct MrLayout {
  char* tables[8];
  float* part[8];
  float* logy[8];
  double* loss_item[8];  // per work item (voice, frame group) of each resolution
  int groups[8];
  double* loss_voice;
  size_t total;
};

// Per-voice loss: the work items' partial sums added in a fixed order
// (resolution, then frame group), so the total does not depend on which
// CTA finished first.
struct MrLossItems {
  const double* item[8];
  int groups[8];
  int n_res;
};

__global__ void mr_loss_reduce(MrLossItems li, int batch, double* __restrict__ loss_voice) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= batch) return;
  double s = 0.0;
  for (int r = 0; r < li.n_res; ++r)
    for (int g = 0; g < li.groups[r]; ++g) s += li.item[r][(size_t)v * li.groups[r] + g];
  loss_voice[v] = s;
}

MrLayout mr_layout(int64_t N, int batch, const int* n_ffts, int n_res, void* ws) {
  MrLayout L;
  char* base = static_cast<char*>(ws);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += al256(bytes);
    return p;
  };
  for (int r = 0; r < n_res; ++r) {
    const int n = n_ffts[r], F = stft_frames(N, n);
    L.tables[r] = take(mr_table_bytes(std::max(1, r_of(n))));
    L.logy[r] = reinterpret_cast<float*>(take(sizeof(float) * batch * F * (n / 2 + 4)));
    const int64_t groups = (F + mr_group(n) - 1) / mr_group(n);
    L.part[r] = reinterpret_cast<float*>(take(sizeof(float) * batch * groups * mr_seg(n)));
    L.loss_item[r] = reinterpret_cast<double*>(take(sizeof(double) * batch * groups));
    L.groups[r] = (int)groups;
  }
  L.loss_voice = reinterpret_cast<double*>(take(sizeof(double) * batch));
  L.total = off;
  return L;
}
}  // namespace

size_t mrstft_workspace_bytes(int64_t N, int batch, const int* n_ffts, int n_res) {
  return mr_layout(N, batch, n_ffts, n_res, nullptr).total;
}

cudaError_t mrstft_loss_grad(const float* x, const float* y, int64_t N, int batch,
                             const int* n_ffts, int n_res, float eps, bool target_ready,
                             double* loss_voice_out, float* grad_x, void* ws, unsigned int* err,
                             cudaStream_t st) {
  if (n_res < 1 || n_res > 8) return cudaErrorInvalidValue;
  for (int r = 0; r < n_res; ++r)  // reflect padding needs more samples than half a frame
    if (r_of(n_ffts[r]) == 0 || N <= n_ffts[r] / 2 || N >= (int64_t)1 << 31)
      return cudaErrorInvalidValue;
  if (batch <= 0) return cudaSuccess;
  MrLayout L = mr_layout(N, batch, n_ffts, n_res, ws);
  cudaError_t e;
  if (!target_ready) {
    for (int r = 0; r < n_res; ++r) {
      const int n = n_ffts[r];
      if ((e = mr_tables_fill(r_of(n), L.tables[r], st)) != cudaSuccess) return e;
      if ((e = mr_pass(n, y, (int)N, stft_frames(N, n), batch, L.tables[r], eps, 0.f, kMrTarget,
                       L.logy[r], nullptr, nullptr, err, st)) != cudaSuccess)
        return e;
    }
  }
  OlaArgs ola;
  MrLossItems li;
  li.n_res = n_res;
  ola.n_res = n_res;
  for (int r = 0; r < n_res; ++r) {
    const int n = n_ffts[r], F = stft_frames(N, n);
    const float scale = 1.0f / (float)((int64_t)F * (n / 2 + 1));
    if ((e = mr_pass(n, x, (int)N, F, batch, L.tables[r], eps, scale,
                     grad_x ? kMrLossGrad : kMrLoss, L.logy[r], L.loss_item[r], L.part[r], err,
                     st)) != cudaSuccess)
      return e;
    li.item[r] = L.loss_item[r];
    li.groups[r] = L.groups[r];
    ola.r[r] = OlaRes{L.part[r], n, n / 4, mr_group(n), (F + mr_group(n) - 1) / mr_group(n),
                      mr_seg(n), F};
  }
  if (grad_x) {
    int pad_max = 0;
    for (int r = 0; r < n_res; ++r) pad_max = std::max(pad_max, n_ffts[r] / 2);
    dim3 go((unsigned)std::min<int64_t>((N / 4 + 255) / 256 + 1, 1024), (unsigned)batch);
    mr_ola_gather<<<go, 256, 0, st>>>(ola, (int)N, pad_max, grad_x);
  }
  mr_loss_reduce<<<(batch + 127) / 128, 128, 0, st>>>(li, batch,
                                                     loss_voice_out ? loss_voice_out : L.loss_voice);
  return cudaGetLastError();
}

}  // namespace synth
