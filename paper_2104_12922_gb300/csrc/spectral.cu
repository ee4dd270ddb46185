// spectral.cu -- STFT-as-GEMM front ends on the tcgen05 tensor cores.
//
// * Multi-resolution log-magnitude STFT distance (the paper's "multi-scale
//   spectrogram" distance, Sec. 4.4) and its gradient with respect to the
//   audio: periodic Hann window, hop n/4, centred frames with reflect
//   padding; L = sum_n mean_(bins, frames) |log(|X| + eps) - log(|Y| + eps)|,
//   summed over voices.
// * Log-mel features for the learned proposal: |X|^2 (n 2048, hop 512),
//   128 Slaney-scale triangular bands, log(. + 1e-6).
//
// Framing: audio (FP32) -> frames (bf16, reflect-padded) -> GEMM with a
// window-folded DFT matrix whose rows interleave cos and -sin of each bin, so
// accumulator columns (2b, 2b+1) are (Re, Im) of bin b. The gradient runs the
// transposed GEMM (dSpec x DFT) and an overlap-add gather that also folds the
// reflect padding back.

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "gemm_tc.h"
#include "spectral.h"

namespace synth {

namespace {

// Split-bf16 products: a value a is carried as a_hi = bf16(a) and
// a_lo = bf16(a - a_hi); a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi keeps about
// 16 significant bits where a single bf16 product keeps 8. Laying the
// operand A out as [hi | hi | lo] along K and B as [hi | lo | hi] makes one
// tensor-core GEMM over 3K sum exactly those three products in FP32.
__device__ __forceinline__ void split_bf16(float a, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16(a);
  lo = __float2bfloat16(a - __bfloat162float(hi));
}

__device__ __forceinline__ int reflect32(int q, int N) {
  if (q < 0) q = -q;
  if (q >= N) q = 2 * (N - 1) - q;
  return q;
}

// frames[row][seg * n_fft]: row = (voice, frame), one block per row; seg = 1
// plain bf16, seg = 3 the [hi | hi | lo] split layout. Two samples per
// thread and store (n_fft is even).
__global__ void frame_reflect_bf16(const float* __restrict__ audio, int N, int n_fft, int hop,
                                   int F, int seg, __nv_bfloat16* __restrict__ frames) {
  const int row = blockIdx.x;
  const int f = row % F, b = row / F;
  const float* a = audio + (size_t)b * N;
  const int start = f * hop - n_fft / 2;
  __nv_bfloat16* dst = frames + (size_t)row * seg * n_fft;
  for (int t = 2 * (int)threadIdx.x; t < n_fft; t += 2 * (int)blockDim.x) {
    const float a0 = a[reflect32(start + t, N)], a1 = a[reflect32(start + t + 1, N)];
    if (seg == 1) {
      *reinterpret_cast<__nv_bfloat162*>(dst + t) = __floats2bfloat162_rn(a0, a1);
    } else {
      __nv_bfloat16 h0, l0, h1, l1;
      split_bf16(a0, h0, l0);
      split_bf16(a1, h1, l1);
      const __nv_bfloat162 hh = __halves2bfloat162(h0, h1), ll = __halves2bfloat162(l0, l1);
      *reinterpret_cast<__nv_bfloat162*>(dst + t) = hh;
      *reinterpret_cast<__nv_bfloat162*>(dst + n_fft + t) = hh;
      *reinterpret_cast<__nv_bfloat162*>(dst + 2 * n_fft + t) = ll;
    }
  }
}

// fwd[2b][t] = w(t) cos(2 pi b t / n), fwd[2b+1][t] = -w(t) sin(2 pi b t / n)
// (bins b < n/2 + 1), row stride seg * n_fft ([hi | lo | hi] when seg = 3);
// bwd[t][2b], bwd[t][2b+1] the same values transposed, row stride seg * ld_bwd
// with segments of ld_bwd columns (zero-padded).
__global__ void dft_tables(int n_fft, int rows_fwd, int seg, __nv_bfloat16* fwd, int ld_bwd,
                           __nv_bfloat16* bwd) {
  const int nb = n_fft / 2 + 1;
  const int64_t total = (int64_t)rows_fwd * n_fft;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i / n_fft), t = (int)(i % n_fft);
    const int b = r >> 1;
    double val = 0.0;
    if (b < nb) {
      const double w = 0.5 - 0.5 * cospi(2.0 * (double)t / (double)n_fft);
      const int64_t bt = ((int64_t)b * t) % n_fft;  // exact argument reduction
      double s, c;
      sincospi(2.0 * (double)bt / (double)n_fft, &s, &c);
      val = (r & 1) ? -w * s : w * c;
    }
    __nv_bfloat16 hi, lo;
    split_bf16((float)val, hi, lo);
    __nv_bfloat16* f = fwd + (int64_t)r * seg * n_fft + t;
    f[0] = hi;
    if (seg == 3) {
      f[n_fft] = lo;
      f[2 * n_fft] = hi;
    }
    if (bwd && r < ld_bwd) {
      __nv_bfloat16* g = bwd + (int64_t)t * seg * ld_bwd + r;
      g[0] = hi;
      if (seg == 3) {
        g[ld_bwd] = lo;
        g[2 * ld_bwd] = hi;
      }
    }
  }
}

// log-magnitude of the target: logy[row][b] = log(|Y_b| + eps)
__global__ void spec_logmag(const float* __restrict__ spec, int ld_spec, int64_t M, int nb,
                            float eps, float* __restrict__ logy) {
  const int64_t total = M * nb;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / nb;
    const int b = (int)(i % nb);
    const float re = spec[row * ld_spec + 2 * b], im = spec[row * ld_spec + 2 * b + 1];
    logy[i] = logf(sqrtf(re * re + im * im) + eps);
  }
}

// |log(|X| + eps) - logy| summed per voice, and the gradient w.r.t. (Re, Im)
// of X for the loss mean over (bins, frames) of one resolution. Block
// (v, c) takes a slice of voice v's frames and adds one partial sum. The
// gradient goes out in the split layout [hi | hi | lo] with segments of
// ld_dspec columns; the padding columns of each segment are written as 0.
__global__ void spec_l1_logmag_grad(const float* __restrict__ spec, int ld_spec,
                                    const float* __restrict__ logy, int nb, int F, float eps,
                                    float scale, double* __restrict__ loss_voice,
                                    __nv_bfloat16* __restrict__ dspec, int ld_dspec) {
  __shared__ float red[32];
  const int v = blockIdx.x;
  const int total = F * nb;
  float local = 0.f;
  for (int i = (int)blockIdx.y * (int)blockDim.x + (int)threadIdx.x; i < total;
       i += (int)gridDim.y * (int)blockDim.x) {
    const int fr = i / nb, b = i - fr * nb;
    const size_t row = (size_t)v * F + fr;
    const float2 x = *reinterpret_cast<const float2*>(spec + row * ld_spec + 2 * b);
    const float mag = sqrtf(x.x * x.x + x.y * x.y);
    const float d = logf(mag + eps) - logy[row * nb + b];
    local += fabsf(d);
    float gre = 0.f, gim = 0.f;
    if (mag > 0.f && d != 0.f) {
      const float g = (d > 0.f ? scale : -scale) / ((mag + eps) * mag);
      gre = g * x.x;
      gim = g * x.y;
    }
    __nv_bfloat16* dst = dspec + row * 3 * (size_t)ld_dspec + 2 * b;
    __nv_bfloat16 h0, l0, h1, l1;
    split_bf16(gre, h0, l0);
    split_bf16(gim, h1, l1);
    const __nv_bfloat162 hh = __halves2bfloat162(h0, h1), ll = __halves2bfloat162(l0, l1);
    *reinterpret_cast<__nv_bfloat162*>(dst) = hh;
    *reinterpret_cast<__nv_bfloat162*>(dst + ld_dspec) = hh;
    *reinterpret_cast<__nv_bfloat162*>(dst + 2 * ld_dspec) = ll;
    if (b == 0) {
      __nv_bfloat16* prow = dspec + row * 3 * (size_t)ld_dspec;
      for (int c = 2 * nb; c < ld_dspec; ++c) {
        prow[c] = __float2bfloat16(0.f);
        prow[ld_dspec + c] = __float2bfloat16(0.f);
        prow[2 * ld_dspec + c] = __float2bfloat16(0.f);
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += (double)red[w];
    atomicAdd(&loss_voice[v], t * scale);
  }
}

// dAudio[b][s] (+)= sum over padded positions p with reflect(p - pad) == s of
// sum over frames f covering p of dframes[b F + f][p - f hop]. Grid
// (samples, voices); accumulate = 0 overwrites.
__global__ void overlap_add_reflect(const float* __restrict__ dframes, int N, int n_fft, int hop,
                                    int F, int accumulate, float* __restrict__ daudio) {
  const int pad = n_fft / 2;
  const int b = blockIdx.y;
  const float* dfv = dframes + (size_t)b * F * n_fft;
  float* out = daudio + (size_t)b * N;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
    int pre[3];
    int np = 0;
    pre[np++] = s + pad;
    if (s >= 1 && s <= pad) pre[np++] = pad - s;
    if (s <= N - 2 && 2 * (N - 1) - s + pad < N + 2 * pad && 2 * (N - 1) - s >= N)
      pre[np++] = 2 * (N - 1) - s + pad;
    float acc = 0.f;
    for (int j = 0; j < np; ++j) {
      const int p = pre[j];
      int f_hi = p / hop;
      if (f_hi > F - 1) f_hi = F - 1;
      int f_lo = (p - n_fft + hop) / hop;  // ceil((p - n_fft + 1) / hop)
      if (p - n_fft + 1 <= 0) f_lo = 0;
      for (int f = f_lo; f <= f_hi; ++f) {
        const int t = p - f * hop;
        if (t >= 0 && t < n_fft) acc += dfv[(size_t)f * n_fft + t];
      }
    }
    out[s] = accumulate ? out[s] + acc : acc;
  }
}

int grid_of(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 64 ? b : 152 * 64);
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

int stft_frames(int64_t N, int n_fft) { return 1 + (int)(N / (n_fft / 4)); }

// ------------------------------------------------------------------ tables
size_t dft_bytes(int n_fft, int seg) {
  const int nb = n_fft / 2 + 1;
  const int rows = 2 * nb;
  const int ld_bwd = (rows + 7) & ~7;
  return al256(sizeof(__nv_bfloat16) * (size_t)rows * seg * n_fft) +
         al256(sizeof(__nv_bfloat16) * (size_t)n_fft * seg * ld_bwd);
}

DftTables dft_carve(int n_fft, void* mem, int seg) {
  DftTables t;
  t.n_fft = n_fft;
  t.seg = seg;
  t.nb = n_fft / 2 + 1;
  t.rows = 2 * t.nb;
  t.ld_bwd = (t.rows + 7) & ~7;
  char* p = static_cast<char*>(mem);
  t.fwd = reinterpret_cast<__nv_bfloat16*>(p);
  t.bwd = reinterpret_cast<__nv_bfloat16*>(
      p + al256(sizeof(__nv_bfloat16) * (size_t)t.rows * seg * n_fft));
  return t;
}

cudaError_t dft_fill(const DftTables& t, cudaStream_t st) {
  cudaMemsetAsync(t.bwd, 0, sizeof(__nv_bfloat16) * (size_t)t.n_fft * t.seg * t.ld_bwd, st);
  dft_tables<<<grid_of((int64_t)t.rows * t.n_fft), 256, 0, st>>>(t.n_fft, t.rows, t.seg, t.fwd,
                                                                 t.ld_bwd, t.bwd);
  return cudaGetLastError();
}

// Slaney mel filterbank [n_mels][ld] (bf16, zero-padded), built on the host in
// FP64: triangles between mel-spaced edges from 0 to SR/2, unit area in Hz.
std::vector<float> mel_filterbank_host(int n_fft, int n_mels, double sr, int ld) {
  auto hz_to_mel = [](double f) {
    return f < 1000.0 ? 3.0 * f / 200.0 : 15.0 + 27.0 * std::log(f / 1000.0) / std::log(6.4);
  };
  auto mel_to_hz = [](double m) {
    return m < 15.0 ? 200.0 * m / 3.0 : 1000.0 * std::exp((m - 15.0) * std::log(6.4) / 27.0);
  };
  const int nb = n_fft / 2 + 1;
  std::vector<double> edges(n_mels + 2);
  const double m_hi = hz_to_mel(sr / 2.0);
  for (int i = 0; i < n_mels + 2; ++i) edges[i] = mel_to_hz(m_hi * i / (n_mels + 1));
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
// The distance and its gradient use split-bf16 operands (3 products, about
// 16 significant bits): d log(|X| + eps) / d|X| = 1/(|X| + eps) weights the
// quiet bins heavily, and a single bf16 rounding of frames and DFT weights
// leaves those bins with noise only.
namespace {
constexpr int kSplit = 3;

struct MrLayout {
  DftTables tabs[8];
  __nv_bfloat16* frames;
  float* spec;
  __nv_bfloat16* dspec;
  float* dframes;
  float* logy[8];
  double* loss_voice;
  size_t total;
};

MrLayout mr_layout(int64_t N, int batch, const int* n_ffts, int n_res, void* ws) {
  MrLayout L;
  char* base = static_cast<char*>(ws);
  size_t off = 0;
  int64_t max_frames = 0, max_spec = 0, max_dspec = 0, max_dfr = 0, max_nb = 0;
  for (int r = 0; r < n_res; ++r) {
    const int n = n_ffts[r];
    L.tabs[r] = dft_carve(n, base ? base + off : nullptr, kSplit);
    off += dft_bytes(n, kSplit);
    const int64_t M = (int64_t)batch * stft_frames(N, n);
    max_frames = std::max<int64_t>(max_frames, M * kSplit * n);
    max_spec = std::max<int64_t>(max_spec, M * L.tabs[r].ld_bwd);
    max_dspec = std::max<int64_t>(max_dspec, M * kSplit * L.tabs[r].ld_bwd);
    max_dfr = std::max<int64_t>(max_dfr, M * n);
    max_nb = std::max<int64_t>(max_nb, M * L.tabs[r].nb);
  }
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += al256(bytes);
    return p;
  };
  L.frames = reinterpret_cast<__nv_bfloat16*>(take(sizeof(__nv_bfloat16) * max_frames));
  L.spec = reinterpret_cast<float*>(take(sizeof(float) * max_spec));
  L.dspec = reinterpret_cast<__nv_bfloat16*>(take(sizeof(__nv_bfloat16) * max_dspec));
  L.dframes = reinterpret_cast<float*>(take(sizeof(float) * max_dfr));
  for (int r = 0; r < n_res; ++r) L.logy[r] = reinterpret_cast<float*>(take(sizeof(float) * max_nb));
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
    if (N <= n_ffts[r] / 2 || N >= (int64_t)1 << 31) return cudaErrorInvalidValue;
  MrLayout L = mr_layout(N, batch, n_ffts, n_res, ws);
  cudaError_t e;
  auto spectrum = [&](const float* sig, int r) -> cudaError_t {
    const int n = n_ffts[r], F = stft_frames(N, n);
    const int64_t M = (int64_t)batch * F;
    frame_reflect_bf16<<<(unsigned)M, 256, 0, st>>>(sig, (int)N, n, n / 4, F, kSplit, L.frames);
    GemmEpilogue ep;
    ep.kind = kEpiStoreF32;
    ep.out_f32 = L.spec;
    ep.ldc = L.tabs[r].ld_bwd;
    return gemm_bf16(L.frames, kSplit * n, L.tabs[r].fwd, kSplit * n, (int)M, L.tabs[r].rows,
                     kSplit * n, ep, err, st);
  };
  if (!target_ready) {
    for (int r = 0; r < n_res; ++r) {
      if ((e = dft_fill(L.tabs[r], st)) != cudaSuccess) return e;
      if ((e = spectrum(y, r)) != cudaSuccess) return e;
      const int64_t M = (int64_t)batch * stft_frames(N, n_ffts[r]);
      spec_logmag<<<grid_of(M * L.tabs[r].nb), 256, 0, st>>>(L.spec, L.tabs[r].ld_bwd, M,
                                                            L.tabs[r].nb, eps, L.logy[r]);
    }
  }
  cudaMemsetAsync(L.loss_voice, 0, sizeof(double) * batch, st);
  for (int r = 0; r < n_res; ++r) {
    const int n = n_ffts[r], F = stft_frames(N, n);
    const int64_t M = (int64_t)batch * F;
    const int ld = L.tabs[r].ld_bwd;
    if ((e = spectrum(x, r)) != cudaSuccess) return e;
    const float scale = 1.0f / (float)((int64_t)F * L.tabs[r].nb);
    const int64_t per_voice = (int64_t)F * L.tabs[r].nb;
    dim3 gl(batch, (unsigned)std::min<int64_t>(64, (per_voice + 255) / 256));
    spec_l1_logmag_grad<<<gl, 256, 0, st>>>(L.spec, ld, L.logy[r], L.tabs[r].nb, F, eps, scale,
                                            L.loss_voice, L.dspec, ld);
    if (grad_x) {
      // dFrames[M][n] = dSpec[M][3 ld] * bwd[n][3 ld]^T
      GemmEpilogue eb;
      eb.kind = kEpiStoreF32;
      eb.out_f32 = L.dframes;
      eb.ldc = n;
      if ((e = gemm_bf16(L.dspec, kSplit * ld, L.tabs[r].bwd, kSplit * ld, (int)M, n, kSplit * ld,
                         eb, err, st)) != cudaSuccess)
        return e;
      dim3 go((unsigned)std::min<int64_t>((N + 255) / 256, 1024), (unsigned)batch);
      overlap_add_reflect<<<go, 256, 0, st>>>(L.dframes, (int)N, n, n / 4, F, r > 0 ? 1 : 0,
                                              grad_x);
    }
  }
  if (loss_voice_out)
    cudaMemcpyAsync(loss_voice_out, L.loss_voice, sizeof(double) * batch, cudaMemcpyDeviceToDevice,
                    st);
  return cudaGetLastError();
}

}  // namespace synth
