// sfu_probe.cu -- throughput probe of the special-function unit (MUFU), for
// the denominator of the render's transcendental roofline.
//
// The fused render spends its transcendentals on MUFU instructions: sine
// (sin.approx) for both VCOs, cosine for the square-saw, and ex2.approx plus
// rcp.approx for its tanh. Their per-SM rate on this GPU is measured rather
// than assumed: every thread of a full grid runs kChains independent chains
// x <- op(x), so the unit, not the latency of one chain, sets the pace.
// Host code times one launch with CUDA events; ops per clock per SM follow
// from the sampled SM clock.
//
// The paper has no counterpart (it reports no roofline).

#include <cstdint>

#include "synth.h"

namespace synth {
namespace {

constexpr int kChains = 8;

template <int OP>
__device__ __forceinline__ float mufu(float x) {
  float y;
  if (OP == SYNTH_SFU_SIN) asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  else if (OP == SYNTH_SFU_COS) asm volatile("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  else if (OP == SYNTH_SFU_EX2) asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  else if (OP == SYNTH_SFU_RCP) asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  else if (OP == SYNTH_SFU_LG2) asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  else asm volatile("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int OP>
__global__ void __launch_bounds__(256) sfu_probe_kernel(int iters, float* __restrict__ sink) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 0.001f * (float)(threadIdx.x + c) + 0.5f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      // rcp(rcp(x)) is x: an FP32 add between reciprocals keeps every one
      // of them (the add runs on the FP32 pipe, not the unit under test)
      x[c] = OP == SYNTH_SFU_RCP ? mufu<OP>(x[c]) + 1.0f : mufu<OP>(x[c]);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.678f) sink[threadIdx.x] = s;  // keeps the chains alive
}

}  // namespace
}  // namespace synth

using namespace synth;

extern "C" synth_status synth_sfu_probe(int32_t op, int32_t blocks, int32_t iters, float* sink_dev,
                                        int64_t* ops_out, void* stream) {
  if (op < SYNTH_SFU_SIN || op > SYNTH_SFU_TANH || blocks < 1 || iters < 1 || !sink_dev)
    return SYNTH_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (op) {
    case SYNTH_SFU_SIN: sfu_probe_kernel<SYNTH_SFU_SIN><<<blocks, 256, 0, st>>>(iters, sink_dev); break;
    case SYNTH_SFU_COS: sfu_probe_kernel<SYNTH_SFU_COS><<<blocks, 256, 0, st>>>(iters, sink_dev); break;
    case SYNTH_SFU_EX2: sfu_probe_kernel<SYNTH_SFU_EX2><<<blocks, 256, 0, st>>>(iters, sink_dev); break;
    case SYNTH_SFU_RCP: sfu_probe_kernel<SYNTH_SFU_RCP><<<blocks, 256, 0, st>>>(iters, sink_dev); break;
    case SYNTH_SFU_LG2: sfu_probe_kernel<SYNTH_SFU_LG2><<<blocks, 256, 0, st>>>(iters, sink_dev); break;
    default: sfu_probe_kernel<SYNTH_SFU_TANH><<<blocks, 256, 0, st>>>(iters, sink_dev); break;
  }
  if (ops_out) *ops_out = (int64_t)blocks * 256 * kChains * (int64_t)iters;
  return cudaGetLastError() == cudaSuccess ? SYNTH_OK : SYNTH_ERR_CUDA;
}
