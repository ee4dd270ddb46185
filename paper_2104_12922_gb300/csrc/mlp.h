// mlp.h -- the proposal MLP (mlp.cu): byte offsets of every tensor inside one
// device allocation, and the forward / training-step launchers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace synth {

struct MlpLayout {
  int dims[5];      // in, hidden, hidden, hidden, out
  int out_pad;      // out rounded up to a multiple of 8
  int max_batch;
  size_t w[4], b[4], mw[4], vw[4], mb[4], vb[4], gw[4], gb[4], wb[4], wt[4];
  size_t h0t, h[4], ht[4], y, dz, dzt, dzf, dh, loss;
  size_t loss_part, loss_counter;  // per-block loss partials, last-block counter
  size_t splitk, splitk_bytes;     // split-K partial products of the small GEMMs
  size_t total;
};

MlpLayout mlp_layout(int in_dim, int hidden, int out_dim, int max_batch, size_t splitk_bytes);
cudaError_t mlp_init(const MlpLayout& L, char* base, uint64_t seed, cudaStream_t st);
// y_out [batch][out] (FP32 sigmoid outputs), or the model's own buffer if NULL.
cudaError_t mlp_forward(const MlpLayout& L, char* base, const __nv_bfloat16* x, int batch,
                        bool keep_transposes, float* y_out, unsigned int* err, cudaStream_t st);
// Forward, MSE against target [batch][out], backward, one Adam step (step >= 1).
cudaError_t mlp_train_step(const MlpLayout& L, char* base, const __nv_bfloat16* x,
                           const float* target, int batch, float lr, int step, float* loss_out,
                           unsigned int* err, cudaStream_t st);
// Hidden activations H_layer (layer 1..3, bf16, of the last forward or
// training step) as FP32 [batch][hidden].
cudaError_t mlp_hidden_f32(const MlpLayout& L, const char* base, int layer, int batch, float* dst,
                           cudaStream_t st);
cudaError_t param_adam(float* u, const float* g, float* m, float* v, int n, int step, float lr,
                       cudaStream_t st);

}  // namespace synth
