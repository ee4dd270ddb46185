// fft_warp.cuh -- building blocks of the warp-level real FFTs of the spectral
// front ends (log-mel features, MR-STFT distance).
//
// A real frame of n = 2M samples is packed as the M-point complex sequence
// z[m] = x[2m] + i x[2m+1]. With M = 32 R (R = 8, 16, 32) a warp transforms
// 32 / R frames at once, split as m = 32 a + b (a < R, b < 32) and
// k = k1 + R k2 (k1 < R, k2 < 32):
//   Z[k1 + R k2] = sum_b W32^(b k2) W_M^(b k1) sum_a W_R^(a k1) z[32 a + b],
// with W_L = e^(-2 pi i / L). Lane b holds the R values z[32 a + b] of each of
// its frames and takes the R-point DFTs over a; after the twiddle W_M^(b k1)
// a padded shared-memory transpose gives lane (frame, k1) the 32 values over
// b, and a 32-point DFT over b finishes the transform. The DFTs run in
// registers; every register index is a compile-time constant after
// unrolling.
#pragma once

namespace synth {
namespace fftw {

// e^(-2 pi i j / 32), j = 0..15: the values of cos and -sin at 2 pi j / 32
__device__ __forceinline__ float w32_re(int j) {
  constexpr float c[16] = {1.000000000e+00f, 9.807852804e-01f, 9.238795325e-01f, 8.314696123e-01f,
                           7.071067812e-01f, 5.555702330e-01f, 3.826834324e-01f, 1.950903220e-01f,
                           0.0f, -1.950903220e-01f, -3.826834324e-01f, -5.555702330e-01f,
                           -7.071067812e-01f, -8.314696123e-01f, -9.238795325e-01f, -9.807852804e-01f};
  return c[j];
}
__device__ __forceinline__ float w32_im(int j) {
  constexpr float s[16] = {0.0f, -1.950903220e-01f, -3.826834324e-01f, -5.555702330e-01f,
                           -7.071067812e-01f, -8.314696123e-01f, -9.238795325e-01f, -9.807852804e-01f,
                           -1.000000000e+00f, -9.807852804e-01f, -9.238795325e-01f, -8.314696123e-01f,
                           -7.071067812e-01f, -5.555702330e-01f, -3.826834324e-01f, -1.950903220e-01f};
  return s[j];
}

// bit reversal of r in log2(L) bits (L = 8, 16, 32)
template <int L>
__host__ __device__ constexpr int bitrev(int r) {
  return L == 32 ? (((r & 1) << 4) | ((r & 2) << 2) | (r & 4) | ((r & 8) >> 2) | ((r & 16) >> 4))
       : L == 16 ? (((r & 1) << 3) | ((r & 2) << 1) | ((r & 4) >> 1) | ((r & 8) >> 3))
                 : (((r & 1) << 2) | (r & 2) | ((r & 4) >> 2));
}

// In-register radix-2 decimation-in-frequency L-point DFT (L = 8, 16, 32) of
// re/im[O .. O + L): X[k] = sum_n x[n] e^(-2 pi i n k / L) for natural-order
// input, X[k] left in register O + bitrev<L>(k). The twiddle of a butterfly
// of half-width h at offset j is e^(-2 pi i j / (2h)) = W32^(16 j / h); the
// trivial ones (1 and -i) cost no multiplications.
template <int L, int O>
__device__ __forceinline__ void dft(float (&re)[32], float (&im)[32]) {
#pragma unroll
  for (int half = L / 2; half >= 1; half >>= 1) {
#pragma unroll
    for (int g = 0; g < L; g += 2 * half) {
#pragma unroll
      for (int j = 0; j < half; ++j) {
        const int p = O + g + j, q = O + g + j + half;
        const float ur = re[p], ui = im[p], vr = re[q], vi = im[q];
        re[p] = ur + vr;
        im[p] = ui + vi;
        const float dr = ur - vr, di = ui - vi;
        const int tw = j * (16 / half);
        if (tw == 0) {
          re[q] = dr;
          im[q] = di;
        } else if (tw == 8) {  // -i
          re[q] = di;
          im[q] = -dr;
        } else {
          const float wr = w32_re(tw), wi = w32_im(tw);
          re[q] = fmaf(dr, wr, -di * wi);
          im[q] = fmaf(dr, wi, di * wr);
        }
      }
    }
  }
}

// The R-point DFTs of all 32 / R frames a lane holds (frame f in registers
// f R .. f R + R - 1).
template <int R>
__device__ __forceinline__ void dft_frames(float (&re)[32], float (&im)[32]) {
  dft<R, 0>(re, im);
  if constexpr (R <= 16) dft<R, R>(re, im);
  if constexpr (R <= 8) {
    dft<R, 2 * R>(re, im);
    dft<R, 3 * R>(re, im);
  }
}

}  // namespace fftw
}  // namespace synth
