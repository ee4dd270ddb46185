// spectral.h -- spectral front ends on warp-level FFTs: the MR-STFT distance
// and its gradient (spectral.cu) and the log-mel features (logmel_fft.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

namespace synth {

constexpr int kMelFFT = 2048;   // log-mel: n_fft 2048, hop 512
constexpr int kMelBands = 128;
// Network input = (log(mel + 1e-6) - shift) / scale: a fixed affine map that
// takes the log floor (-13.8) to about -1.9 and a full-scale tone's bands
// (about +9) to about +1.9.
constexpr float kFeatureShift = -2.5f;
constexpr float kFeatureScale = 6.0f;

// Centred frames of an N-sample signal at hop n/4.
int stft_frames(int64_t N, int n_fft);

// Multi-resolution log-magnitude distance between x and y ([batch][N] FP32,
// device) and its gradient w.r.t. x; n_ffts from {512, 1024, 2048}.
// loss_voice_out [batch] (device, FP64, may be NULL); grad_x [batch][N] or NULL. With target_ready the tables and
// the target log-magnitudes left in ws by an earlier call for the same y are
// reused. err: device word, bit 0 set if a bounded wait gave up.
size_t mrstft_workspace_bytes(int64_t N, int batch, const int* n_ffts, int n_res);
cudaError_t mrstft_loss_grad(const float* x, const float* y, int64_t N, int batch,
                             const int* n_ffts, int n_res, float eps, bool target_ready,
                             double* loss_voice_out, float* grad_x, void* ws, unsigned int* err,
                             cudaStream_t st);

// Slaney mel filterbank [n_mels][ld] (unit-area triangles over 0 .. sr/2)
// and its n_mels + 2 band edges in Hz.
std::vector<float> mel_filterbank_host(int n_fft, int n_mels, double sr, int ld);
std::vector<double> mel_edges_host(int n_mels, double sr);

// Log-mel features [batch][frames][128] (bf16, flattened per voice) through a
// shared-memory FFT (logmel_fft.cu): tables (logmel_fft_table_bytes, filled
// once by logmel_fft_init) and one kernel.
size_t logmel_fft_table_bytes();
cudaError_t logmel_fft_init(double sample_rate, void* tables, cudaStream_t st);
cudaError_t logmel_features_fft(const float* audio, int64_t N, int batch, const void* tables,
                                __nv_bfloat16* features, cudaStream_t st);

}  // namespace synth
