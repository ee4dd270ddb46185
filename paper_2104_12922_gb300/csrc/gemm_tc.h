// gemm_tc.h -- host interface of the tcgen05 BF16 GEMM (gemm_tc.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace synth {

enum GemmEpiKind : int {
  kEpiStoreF32 = 0,     // out_f32[row][col] = alpha * acc
  kEpiBiasActBF16 = 1,  // z = act(acc + bias[col]) -> out_bf16 / out_bf16_t (transposed) / out_f32
};
enum GemmAct : int { kActNone = 0, kActRelu = 1, kActSigmoid = 2 };

struct GemmEpilogue {
  int kind = kEpiStoreF32;
  int act = kActNone;
  float* out_f32 = nullptr;
  __nv_bfloat16* out_bf16 = nullptr;
  __nv_bfloat16* out_bf16_t = nullptr;
  const float* bias = nullptr;
  int ldc = 0;      // row stride (elements) of out_f32 / out_bf16
  int ldc_t = 0;    // row stride of the transposed copy
  float alpha = 1.f;
};

// C = A[M][K] * B[N][K]^T on the tensor cores; A, B bf16 with row strides lda,
// ldb (elements, multiples of 8), K a multiple of 8, 16-byte aligned bases.
// err: device word, bit 0 set if a bounded wait gave up.
// splitk_ws (splitk_bytes, device, 16-byte aligned) or NULL: when the output
// has fewer 128 x BN tiles than the GPU has SMs, K is split into slices whose
// FP32 partial products go there and a second kernel adds them in slice
// order (deterministic) before the epilogue. NULL: no split.
cudaError_t gemm_bf16(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M,
                      int N, int K, const GemmEpilogue& epi, unsigned int* err, cudaStream_t st,
                      float* splitk_ws = nullptr, size_t splitk_bytes = 0);

// Workspace that lets gemm_bf16 split every product of at most max_m x max_n
// outputs as far as it would (0 if the device cannot be queried).
size_t gemm_splitk_workspace_bytes(int max_m, int max_n);

}  // namespace synth
