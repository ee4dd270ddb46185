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

__device__ __forceinline__ int64_t reflect_index(int64_t q, int64_t N) {
  if (q < 0) q = -q;
  if (q >= N) q = 2 * (N - 1) - q;
  return q;
}

__global__ void frame_reflect_bf16(const float* __restrict__ audio, int64_t N, int n_fft, int hop,
                                   int F, int batch, __nv_bfloat16* __restrict__ frames) {
  const int64_t total = (int64_t)batch * F * n_fft;
  const int pad = n_fft / 2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(i % n_fft);
    const int64_t row = i / n_fft;
    const int f = (int)(row % F);
    const int64_t b = row / F;
    const int64_t q = reflect_index((int64_t)f * hop + t - pad, N);
    frames[i] = __float2bfloat16(audio[b * N + q]);
  }
}

// fwd[2b][t] = w(t) cos(2 pi b t / n), fwd[2b+1][t] = -w(t) sin(2 pi b t / n)
// (bins b < n/2 + 1, rows up to rows_fwd zero-padded);
// bwd[t][2b], bwd[t][2b+1] the same values transposed (columns up to ld_bwd).
__global__ void dft_tables(int n_fft, int rows_fwd, __nv_bfloat16* fwd, int ld_bwd,
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
    const __nv_bfloat16 v = __float2bfloat16((float)val);
    fwd[i] = v;
    if (bwd && r < ld_bwd) bwd[(int64_t)t * ld_bwd + r] = v;
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
// (v, c) takes a slice of voice v's frames and adds one partial sum.
__global__ void spec_l1_logmag_grad(const float* __restrict__ spec, int ld_spec,
                                    const float* __restrict__ logy, int nb, int F, float eps,
                                    float scale, double* __restrict__ loss_voice,
                                    __nv_bfloat16* __restrict__ dspec, int ld_dspec) {
  __shared__ double red[32];
  const int v = blockIdx.x;
  const int64_t row0 = (int64_t)v * F;
  const int64_t total = (int64_t)F * nb;
  double local = 0.0;
  for (int64_t i = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.y * blockDim.x) {
    const int64_t row = row0 + i / nb;
    const int b = (int)(i % nb);
    const float re = spec[row * ld_spec + 2 * b], im = spec[row * ld_spec + 2 * b + 1];
    const float mag = sqrtf(re * re + im * im);
    const float d = logf(mag + eps) - logy[row * nb + b];
    local += fabsf(d);
    float gre = 0.f, gim = 0.f;
    if (mag > 0.f && d != 0.f) {
      const float g = (d > 0.f ? scale : -scale) / ((mag + eps) * mag);
      gre = g * re;
      gim = g * im;
    }
    dspec[row * ld_dspec + 2 * b] = __float2bfloat16(gre);
    dspec[row * ld_dspec + 2 * b + 1] = __float2bfloat16(gim);
  }
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    atomicAdd(&loss_voice[v], t * scale);
  }
}

// dAudio[b][i] (+)= sum over padded positions p with reflect(p - pad) == i of
// sum over frames f covering p of dframes[b F + f][p - f hop].
__global__ void overlap_add_reflect(const float* __restrict__ dframes, int64_t N, int n_fft, int hop,
                                    int F, int batch, float* __restrict__ daudio) {
  const int pad = n_fft / 2;
  const int64_t total = (int64_t)batch * N;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i / N, s = i % N;
    int64_t pre[3];
    int np = 0;
    pre[np++] = s + pad;
    if (s >= 1 && s <= pad) pre[np++] = pad - s;
    if (s <= N - 2 && 2 * (N - 1) - s + pad < N + 2 * pad && 2 * (N - 1) - s >= N)
      pre[np++] = 2 * (N - 1) - s + pad;
    float acc = 0.f;
    for (int j = 0; j < np; ++j) {
      const int64_t p = pre[j];
      int64_t f_hi = p / hop;
      if (f_hi > F - 1) f_hi = F - 1;
      int64_t f_lo = (p - n_fft + hop) / hop;  // ceil((p - n_fft + 1) / hop)
      if (p - n_fft + 1 <= 0) f_lo = 0;
      for (int64_t f = f_lo; f <= f_hi; ++f) {
        const int64_t t = p - f * hop;
        if (t >= 0 && t < n_fft) acc += dframes[(b * F + f) * n_fft + t];
      }
    }
    daudio[i] += acc;
  }
}

__global__ void fill_zero_f(float* p, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 0.f;
}

int grid_of(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 64 ? b : 152 * 64);
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

int stft_frames(int64_t N, int n_fft) { return 1 + (int)(N / (n_fft / 4)); }

// ------------------------------------------------------------------ tables
size_t dft_bytes(int n_fft) {
  const int nb = n_fft / 2 + 1;
  const int rows = 2 * nb;
  const int ld_bwd = (rows + 7) & ~7;
  return al256(sizeof(__nv_bfloat16) * (size_t)rows * n_fft) +
         al256(sizeof(__nv_bfloat16) * (size_t)n_fft * ld_bwd);
}

DftTables dft_carve(int n_fft, void* mem) {
  DftTables t;
  t.n_fft = n_fft;
  t.nb = n_fft / 2 + 1;
  t.rows = 2 * t.nb;
  t.ld_bwd = (t.rows + 7) & ~7;
  char* p = static_cast<char*>(mem);
  t.fwd = reinterpret_cast<__nv_bfloat16*>(p);
  t.bwd = reinterpret_cast<__nv_bfloat16*>(p + al256(sizeof(__nv_bfloat16) * (size_t)t.rows * n_fft));
  return t;
}

cudaError_t dft_fill(const DftTables& t, cudaStream_t st) {
  cudaMemsetAsync(t.bwd, 0, sizeof(__nv_bfloat16) * (size_t)t.n_fft * t.ld_bwd, st);
  dft_tables<<<grid_of((int64_t)t.rows * t.n_fft), 256, 0, st>>>(t.n_fft, t.rows, t.fwd, t.ld_bwd,
                                                                 t.bwd);
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
size_t mrstft_workspace_bytes(int64_t N, int batch, const int* n_ffts, int n_res) {
  size_t total = 0;
  int64_t max_rows_n = 0, max_spec = 0, max_nb = 0;
  for (int r = 0; r < n_res; ++r) {
    const int n = n_ffts[r];
    total += dft_bytes(n);
    const int64_t M = (int64_t)batch * stft_frames(N, n);
    max_rows_n = std::max<int64_t>(max_rows_n, M * n);
    const int ld = ((2 * (n / 2 + 1)) + 7) & ~7;
    max_spec = std::max<int64_t>(max_spec, M * ld);
    max_nb = std::max<int64_t>(max_nb, M * (n / 2 + 1));
  }
  total += al256(sizeof(__nv_bfloat16) * max_rows_n);  // frames
  total += al256(sizeof(float) * max_spec);           // spectrum (f32)
  total += al256(sizeof(__nv_bfloat16) * max_spec);   // d spectrum (bf16)
  total += al256(sizeof(float) * max_rows_n);         // d frames
  total += al256(sizeof(float) * max_nb) * n_res;     // target log-magnitudes per resolution
  total += al256(sizeof(double) * batch);             // per-voice loss
  return total;
}

cudaError_t mrstft_loss_grad(const float* x, const float* y, int64_t N, int batch,
                             const int* n_ffts, int n_res, float eps, bool target_ready,
                             double* loss_voice_out, float* grad_x, void* ws, unsigned int* err,
                             cudaStream_t st) {
  char* base = static_cast<char*>(ws);
  size_t off = 0;
  DftTables tabs[8];
  for (int r = 0; r < n_res; ++r) {
    tabs[r] = dft_carve(n_ffts[r], base + off);
    off += dft_bytes(n_ffts[r]);
  }
  int64_t max_rows_n = 0, max_spec = 0, max_nb = 0;
  for (int r = 0; r < n_res; ++r) {
    const int n = n_ffts[r];
    const int64_t M = (int64_t)batch * stft_frames(N, n);
    max_rows_n = std::max<int64_t>(max_rows_n, M * n);
    max_spec = std::max<int64_t>(max_spec, M * tabs[r].ld_bwd);
    max_nb = std::max<int64_t>(max_nb, M * tabs[r].nb);
  }
  auto take = [&](size_t bytes) { char* p = base + off; off += al256(bytes); return p; };
  __nv_bfloat16* frames = reinterpret_cast<__nv_bfloat16*>(take(sizeof(__nv_bfloat16) * max_rows_n));
  float* spec = reinterpret_cast<float*>(take(sizeof(float) * max_spec));
  __nv_bfloat16* dspec = reinterpret_cast<__nv_bfloat16*>(take(sizeof(__nv_bfloat16) * max_spec));
  float* dframes = reinterpret_cast<float*>(take(sizeof(float) * max_rows_n));
  float* logy[8];
  for (int r = 0; r < n_res; ++r) logy[r] = reinterpret_cast<float*>(take(sizeof(float) * max_nb));
  double* loss_voice = reinterpret_cast<double*>(take(sizeof(double) * batch));

  cudaError_t e;
  if (!target_ready) {
    for (int r = 0; r < n_res; ++r) {
      if ((e = dft_fill(tabs[r], st)) != cudaSuccess) return e;
      const int n = n_ffts[r], F = stft_frames(N, n);
      const int64_t M = (int64_t)batch * F;
      frame_reflect_bf16<<<grid_of(M * n), 256, 0, st>>>(y, N, n, n / 4, F, batch, frames);
      GemmEpilogue ep;
      ep.kind = kEpiStoreF32;
      ep.out_f32 = spec;
      ep.ldc = tabs[r].ld_bwd;
      if ((e = gemm_bf16(frames, n, tabs[r].fwd, n, (int)M, tabs[r].rows, n, ep, err, st)) !=
          cudaSuccess)
        return e;
      spec_logmag<<<grid_of(M * tabs[r].nb), 256, 0, st>>>(spec, tabs[r].ld_bwd, M, tabs[r].nb,
                                                          eps, logy[r]);
    }
  }
  cudaMemsetAsync(loss_voice, 0, sizeof(double) * batch, st);
  if (grad_x) fill_zero_f<<<grid_of((int64_t)batch * N), 256, 0, st>>>(grad_x, (int64_t)batch * N);
  for (int r = 0; r < n_res; ++r) {
    const int n = n_ffts[r], F = stft_frames(N, n);
    const int64_t M = (int64_t)batch * F;
    frame_reflect_bf16<<<grid_of(M * n), 256, 0, st>>>(x, N, n, n / 4, F, batch, frames);
    GemmEpilogue ep;
    ep.kind = kEpiStoreF32;
    ep.out_f32 = spec;
    ep.ldc = tabs[r].ld_bwd;
    if ((e = gemm_bf16(frames, n, tabs[r].fwd, n, (int)M, tabs[r].rows, n, ep, err, st)) !=
        cudaSuccess)
      return e;
    cudaMemsetAsync(dspec, 0, sizeof(__nv_bfloat16) * M * tabs[r].ld_bwd, st);
    const float scale = 1.0f / (float)((int64_t)F * tabs[r].nb);
    const int64_t per_voice = (int64_t)F * tabs[r].nb;
    dim3 gl(batch, (unsigned)std::min<int64_t>(64, (per_voice + 255) / 256));
    spec_l1_logmag_grad<<<gl, 256, 0, st>>>(spec, tabs[r].ld_bwd, logy[r], tabs[r].nb, F, eps,
                                            scale, loss_voice, dspec, tabs[r].ld_bwd);
    if (grad_x) {
      // dFrames[M][n] = dSpec[M][K = ld] * bwd[n][K]^T
      GemmEpilogue eb;
      eb.kind = kEpiStoreF32;
      eb.out_f32 = dframes;
      eb.ldc = n;
      if ((e = gemm_bf16(dspec, tabs[r].ld_bwd, tabs[r].bwd, tabs[r].ld_bwd, (int)M, n,
                         tabs[r].ld_bwd, eb, err, st)) != cudaSuccess)
        return e;
      overlap_add_reflect<<<grid_of((int64_t)batch * N), 256, 0, st>>>(dframes, N, n, n / 4, F,
                                                                       batch, grad_x);
    }
  }
  if (loss_voice_out)
    cudaMemcpyAsync(loss_voice_out, loss_voice, sizeof(double) * batch, cudaMemcpyDeviceToDevice,
                    st);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- log-mel
size_t logmel_workspace_bytes(int64_t N, int batch) {
  const int n = kMelFFT, F = stft_frames(N, n);
  const int64_t M = (int64_t)batch * F;
  const int nb = n / 2 + 1, ldp = (nb + 7) & ~7;
  return dft_bytes(n) + al256(sizeof(__nv_bfloat16) * kMelBands * ldp) +
         al256(sizeof(__nv_bfloat16) * M * n) + al256(sizeof(__nv_bfloat16) * M * ldp);
}

cudaError_t logmel_init(int64_t N, int batch, double sample_rate, void* ws, cudaStream_t st) {
  const int n = kMelFFT;
  DftTables t = dft_carve(n, ws);
  cudaError_t e = dft_fill(t, st);
  if (e != cudaSuccess) return e;
  const int nb = n / 2 + 1, ldp = (nb + 7) & ~7;
  std::vector<float> fb = mel_filterbank_host(n, kMelBands, sample_rate, ldp);
  std::vector<__nv_bfloat16> fbb(fb.size());
  for (size_t i = 0; i < fb.size(); ++i) fbb[i] = __float2bfloat16(fb[i]);
  char* mel = static_cast<char*>(ws) + dft_bytes(n);
  e = cudaMemcpyAsync(mel, fbb.data(), fbb.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}

cudaError_t logmel_features(const float* audio, int64_t N, int batch, void* ws,
                            __nv_bfloat16* features, unsigned int* err, cudaStream_t st) {
  const int n = kMelFFT, F = stft_frames(N, n);
  const int64_t M = (int64_t)batch * F;
  const int nb = n / 2 + 1, ldp = (nb + 7) & ~7;
  char* base = static_cast<char*>(ws);
  DftTables t = dft_carve(n, base);
  size_t off = dft_bytes(n);
  __nv_bfloat16* melfb = reinterpret_cast<__nv_bfloat16*>(base + off);
  off += al256(sizeof(__nv_bfloat16) * kMelBands * ldp);
  __nv_bfloat16* frames = reinterpret_cast<__nv_bfloat16*>(base + off);
  off += al256(sizeof(__nv_bfloat16) * M * n);
  __nv_bfloat16* power = reinterpret_cast<__nv_bfloat16*>(base + off);
  frame_reflect_bf16<<<grid_of(M * n), 256, 0, st>>>(audio, N, n, n / 4, F, batch, frames);
  cudaMemsetAsync(power, 0, sizeof(__nv_bfloat16) * M * ldp, st);
  GemmEpilogue ep;
  ep.kind = kEpiPowerPairs;
  ep.out_bf16 = power;
  ep.ldc = ldp;
  ep.n_valid = nb;
  cudaError_t e = gemm_bf16(frames, n, t.fwd, n, (int)M, t.rows, n, ep, err, st);
  if (e != cudaSuccess) return e;
  GemmEpilogue em;
  em.kind = kEpiLogBF16;
  em.out_bf16 = features;
  em.ldc = kMelBands;
  em.n_valid = kMelBands;
  em.eps = 1e-6f;
  em.shift = kFeatureShift;
  em.alpha = 1.0f / kFeatureScale;
  return gemm_bf16(power, ldp, melfb, ldp, (int)M, kMelBands, ldp, em, err, st);
}

}  // namespace synth
