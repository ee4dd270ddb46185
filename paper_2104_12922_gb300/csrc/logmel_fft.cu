// logmel_fft.cu -- the proposal network's log-mel front end as a shared-memory
// FFT: periodic-Hann frames of 2048 samples at hop 512 with centred reflect
// padding, |X|^2 per bin, 128 Slaney mel bands, log(. + 1e-6) and the fixed
// affine map to the network input, in one kernel that reads the audio once
// and writes only the bf16 features.
//
// A CTA takes one voice and a group of up to kGroup frames: it stages the
// padded audio segment the group covers in shared memory, then each warp
// transforms whole frames. A 2048-point real frame is packed as a 1024-point
// complex sequence z[m] = x[2m] + i x[2m+1]; the 1024-point FFT is split as
// 32 x 32 (m = 32 a + b, k = k1 + 32 k2): lane b computes the 32-point DFT
// over a in registers, multiplies by W1024^(b k1), a padded shared-memory
// transpose hands column k1 to lane k1, which computes the 32-point DFT over
// b. The real spectrum follows from Z[k] and Z[1024 - k] (a lane shuffle):
// X[k] = E[k] + W2048^k O[k] with E = (Z[k] + conj Z[1024-k]) / 2 and
// O = (Z[k] - conj Z[1024-k]) / 2i. The 1/2 of E and O is folded into the
// mel weights (a factor 1/4 on |X|^2). The window is a shared-memory table
// each CTA fills once from the SFU cosine (evaluated per frame, the cosines
// competed with the transform for registers and spilled), and each mel
// weight comes from its band's two triangle lines.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "fft_warp.cuh"
#include "launch_config.h"
#include "pdl.cuh"
#include "spectral.h"

namespace synth {
namespace {

using fftw::bitrev;

constexpr int kHop = kMelFFT / 4;      // 512
constexpr int kHalf = kMelFFT / 2;     // 1024 complex points
constexpr int kBins = kHalf + 1;       // 1025
constexpr int kGroup = 16;             // frames per CTA
constexpr int kWarpsLm = 8;
constexpr int kThreadsLm = 32 * kWarpsLm;
constexpr int kLd = 33;                // padded row of the transpose buffer
constexpr int kBuf = 32 * kLd;         // floats per warp (>= kBins)
constexpr int kSegMax = (kGroup - 1) * kHop + kMelFFT;
static_assert(kBuf >= kBins, "power spectrum fits the transpose buffer");

struct LmTables {
  const float2* tw;     // [32][32]: e^(-2 pi i b k1 / 1024) at [k1][b]
  const float2* post;   // [1024]: e^(-2 pi i k / 2048)
  const int2* band;     // [128]: first non-zero bin, bin count
  const float4* line;   // [128]: mel weight x 1/4 of bin k = max(0, min(x k + y, z k + w))
};

struct __align__(16) LmSmem {
  float seg[kSegMax];           // the group's padded audio
  float buf[kWarpsLm][kBuf];    // per warp: transpose, then power spectrum, then bands
  float2 tw[32 * 32];
  float2 post[kHalf];
  float2 hann[kHalf];           // Hann window at samples 2m, 2m + 1
  int2 band[kMelBands];
  float4 line[kMelBands];
};

// Periodic Hann window at sample k of the 2048-point frame from the SFU
// cosine on [-pi, pi): 0.5 - 0.5 cos(2 pi k / n) = 0.5 + 0.5 cos(2 pi k / n - pi).
__device__ __forceinline__ float hann2048(int k) {
  return fmaf(0.5f, __cosf(fmaf((float)k, 0.0030679615757712823f, -3.14159265358979f)), 0.5f);
}

__global__ void __launch_bounds__(kThreadsLm, 2)
    logmel_fft_kernel(const float* __restrict__ audio, int N, int F, int batch, LmTables t,
                      float eps, float shift, float inv_scale,
                      __nv_bfloat16* __restrict__ features) {
  pdl_wait();     // earlier kernels' writes are visible
  pdl_release();  // the next kernel may be scheduled
  extern __shared__ __align__(16) unsigned char lm_raw[];
  LmSmem& S = *reinterpret_cast<LmSmem*>(lm_raw);
  for (int j = threadIdx.x; j < kHalf; j += kThreadsLm) {
    S.post[j] = __ldg(t.post + j);
    S.hann[j] = make_float2(hann2048(2 * j), hann2048(2 * j + 1));
  }
  for (int j = threadIdx.x; j < 32 * 32; j += kThreadsLm) S.tw[j] = __ldg(t.tw + j);
  for (int j = threadIdx.x; j < kMelBands; j += kThreadsLm) {
    S.band[j] = __ldg(t.band + j);
    S.line[j] = __ldg(t.line + j);
  }
  const bool vec = (N & 3) == 0 && (reinterpret_cast<uintptr_t>(audio) & 15) == 0;
  const int groups = (F + kGroup - 1) / kGroup;
  const int items = groups * batch;
  // persistent: items (voice, group of frames) strided over the grid
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int v = item / groups, f0 = (item - v * groups) * kGroup;
    const int G = min(kGroup, F - f0);
    const int len = (G - 1) * kHop + kMelFFT;
    const float* x = audio + (size_t)v * N;
    // padded sample j of the group = x[reflect(f0 * hop + j - n/2)]; base is a
    // multiple of 4, so with N % 4 == 0 every 4-sample run is either wholly
    // inside the signal (one 16-byte load) or wholly reflected
    const int base = f0 * kHop - kHalf;
    __syncthreads();  // the previous item's frames are done with the segment
    for (int j = 4 * threadIdx.x; j < len; j += 4 * kThreadsLm) {
      const int i0 = base + j;
      if (vec && i0 >= 0 && i0 + 3 < N) {
        // asynchronous 16-byte copy: all of the segment's copies are in
        // flight before the one wait below
        const unsigned int dst = (unsigned int)__cvta_generic_to_shared(S.seg + j);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(x + i0)
                     : "memory");
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int i = i0 + q;
          i = i < 0 ? -i : i;
          i = i >= N ? 2 * (N - 1) - i : i;
          S.seg[j + q] = __ldg(x + i);
        }
      }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* B = S.buf[warp];
    for (int lf = warp; lf < G; lf += kWarpsLm) {
      const float2* s2 = reinterpret_cast<const float2*>(S.seg + lf * kHop);
      float re[32], im[32];
      // z[32 a + lane], windowed
#pragma unroll
      for (int a = 0; a < 32; ++a) {
        const float2 sv = s2[32 * a + lane], w = S.hann[32 * a + lane];
        re[a] = sv.x * w.x;
        im[a] = sv.y * w.y;
      }
      fftw::dft<32, 0>(re, im);  // over a: Y[k1] in register bitrev<32>(k1)
      // twiddle W1024^(lane k1), then the transpose: real parts, then imaginary
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        const int k1 = bitrev<32>(r);
        if (k1 != 0) {
          const float2 w = S.tw[32 * k1 + lane];
          const float yr = re[r], yi = im[r];
          re[r] = fmaf(yr, w.x, -yi * w.y);
          im[r] = fmaf(yr, w.y, yi * w.x);
        }
      }
#pragma unroll
      for (int r = 0; r < 32; ++r) B[bitrev<32>(r) * kLd + lane] = re[r];
      __syncwarp();
#pragma unroll
      for (int b = 0; b < 32; ++b) re[b] = B[lane * kLd + b];
      __syncwarp();
#pragma unroll
      for (int r = 0; r < 32; ++r) B[bitrev<32>(r) * kLd + lane] = im[r];
      __syncwarp();
#pragma unroll
      for (int b = 0; b < 32; ++b) im[b] = B[lane * kLd + b];
      __syncwarp();
      fftw::dft<32, 0>(re, im);  // over b: Z[lane + 32 k2] in register bitrev<32>(k2)

      // real spectrum and power; the partner Z[1024 - k] of k = lane + 32 k2 is
      // Z[(32 - lane) + 32 (31 - k2)] on lane 32 - lane, or, on lane 0,
      // Z[32 ((32 - k2) mod 32)] on lane 0 itself
      const int src = (32 - lane) & 31;
#pragma unroll
      for (int k2 = 0; k2 < 32; ++k2) {
        const int r = bitrev<32>(k2);
        float pr = __shfl_sync(0xffffffffu, re[bitrev<32>(31 - k2)], src);
        float pi = __shfl_sync(0xffffffffu, im[bitrev<32>(31 - k2)], src);
        if (lane == 0) {
          pr = re[bitrev<32>((32 - k2) & 31)];
          pi = im[bitrev<32>((32 - k2) & 31)];
        }
        const int k = lane + 32 * k2;
        const float zr = re[r], zi = im[r];
        const float ar = zr + pr, ai = zi - pi;  // Z + conj(P)
        const float cr = zi + pi, ci = pr - zr;  // -i (Z - conj(P))
        const float2 w = S.post[k];
        const float xr = ar + fmaf(w.x, cr, -w.y * ci);  // 2 X[k]
        const float xi = ai + fmaf(w.x, ci, w.y * cr);
        B[k] = fmaf(xr, xr, xi * xi);
        if (k == 0) {
          const float ny = zr - zi;  // X[1024] = Re Z[0] - Im Z[0]; stored as (2 X)^2
          B[kHalf] = 4.f * ny * ny;
        }
      }
      __syncwarp();
      // mel bands {lane, 63 - lane, 64 + lane, 127 - lane}: narrow and wide
      // bands paired so the lanes' work is about even
      float mel[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = q == 0 ? lane : q == 1 ? 63 - lane : q == 2 ? 64 + lane : 127 - lane;
        const int2 br = S.band[m];
        const float4 ln = S.line[m];
        float acc = 0.f, kf = (float)br.x;
#pragma unroll 4
        for (int j = 0; j < br.y; ++j, kf += 1.f) {
          const float w = fmaxf(0.f, fminf(fmaf(kf, ln.x, ln.y), fmaf(kf, ln.z, ln.w)));
          acc = fmaf(w, B[br.x + j], acc);
        }
        mel[q] = (__logf(acc + eps) - shift) * inv_scale;
      }
      __syncwarp();
      B[lane] = mel[0];
      B[63 - lane] = mel[1];
      B[64 + lane] = mel[2];
      B[127 - lane] = mel[3];
      __syncwarp();
      const float4 o = reinterpret_cast<const float4*>(B)[lane];
      __nv_bfloat162 lo = __floats2bfloat162_rn(o.x, o.y), hi = __floats2bfloat162_rn(o.z, o.w);
      uint2 packed;
      packed.x = *reinterpret_cast<unsigned int*>(&lo);
      packed.y = *reinterpret_cast<unsigned int*>(&hi);
      reinterpret_cast<uint2*>(features + ((size_t)v * F + f0 + lf) * kMelBands)[lane] = packed;
      __syncwarp();
    }
  }
}

size_t al256b(size_t x) { return (x + 255) & ~size_t(255); }

struct LmLayout {
  size_t tw, post, band, line, total;
};

LmLayout lm_layout() {
  LmLayout L{};
  size_t o = 0;
  L.tw = o;   o += al256b(sizeof(float2) * 32 * 32);
  L.post = o; o += al256b(sizeof(float2) * kHalf);
  L.band = o; o += al256b(sizeof(int2) * kMelBands);
  L.line = o; o += al256b(sizeof(float4) * kMelBands);
  L.total = o;
  return L;
}

}  // namespace

size_t logmel_fft_table_bytes() { return lm_layout().total; }

cudaError_t logmel_fft_init(double sample_rate, void* tables, cudaStream_t st) {
  const double pi = 3.14159265358979323846;
  const LmLayout L = lm_layout();
  std::vector<char> host(L.total, 0);
  float2* tw = reinterpret_cast<float2*>(host.data() + L.tw);
  for (int k1 = 0; k1 < 32; ++k1)
    for (int b = 0; b < 32; ++b) {
      const double a = -2.0 * pi * (double)(b * k1) / kHalf;
      tw[32 * k1 + b] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
  float2* post = reinterpret_cast<float2*>(host.data() + L.post);
  for (int k = 0; k < kHalf; ++k) {
    const double a = -2.0 * pi * (double)k / kMelFFT;
    post[k] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  // each band: the bins where the FP64 bank is non-zero, and the two lines of
  // its triangle (rising edge, falling edge) in the bin index, with the unit
  // area normalisation and the 1/4 of the packed transform folded in
  const std::vector<float> fb = mel_filterbank_host(kMelFFT, kMelBands, sample_rate, kBins);
  const std::vector<double> edges = mel_edges_host(kMelBands, sample_rate);
  const double df = sample_rate / kMelFFT;
  int2* band = reinterpret_cast<int2*>(host.data() + L.band);
  float4* line = reinterpret_cast<float4*>(host.data() + L.line);
  for (int m = 0; m < kMelBands; ++m) {
    int lo = -1, hi = -1;
    for (int k = 0; k < kBins; ++k)
      if (fb[(size_t)m * kBins + k] != 0.f) {
        if (lo < 0) lo = k;
        hi = k;
      }
    band[m] = lo < 0 ? make_int2(0, 0) : make_int2(lo, hi - lo + 1);
    const double e0 = edges[m], c = edges[m + 1], e1 = edges[m + 2];
    const double norm = 0.25 * 2.0 / (e1 - e0);
    line[m] = make_float4((float)(norm * df / (c - e0)), (float)(-norm * e0 / (c - e0)),
                          (float)(-norm * df / (e1 - c)), (float)(norm * e1 / (e1 - c)));
  }
  cudaError_t e = cudaMemcpyAsync(tables, host.data(), L.total, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}

cudaError_t logmel_features_fft(const float* audio, int64_t N, int batch, const void* tables,
                                __nv_bfloat16* features, cudaStream_t st) {
  if (N <= kMelFFT / 2 || N >= (int64_t)1 << 31) return cudaErrorInvalidValue;
  if (batch <= 0) return cudaSuccess;
  const int F = stft_frames(N, kMelFFT);
  const LmLayout L = lm_layout();
  const char* b = static_cast<const char*>(tables);
  LmTables t;
  t.tw = reinterpret_cast<const float2*>(b + L.tw);
  t.post = reinterpret_cast<const float2*>(b + L.post);
  t.band = reinterpret_cast<const int2*>(b + L.band);
  t.line = reinterpret_cast<const float4*>(b + L.line);
  const int smem = (int)sizeof(LmSmem);
  int grid_cap = 0;  // resident CTAs on the current device
  const cudaError_t ge =
      resident_grid(reinterpret_cast<const void*>(logmel_fft_kernel), kThreadsLm, smem, &grid_cap);
  if (ge != cudaSuccess) return ge;
  const int64_t items = (int64_t)((F + kGroup - 1) / kGroup) * batch;
  if (items >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
  const int grid = (int)(items < grid_cap ? items : grid_cap);
  const cudaError_t le = launch_pdl(logmel_fft_kernel, dim3((unsigned)grid), dim3(kThreadsLm),
                                    (size_t)smem, st, audio, (int)N, F, batch, t, 1e-6f,
                                    kFeatureShift, 1.0f / kFeatureScale, features);
  if (le != cudaSuccess) return le;
  return cudaGetLastError();
}

}  // namespace synth
