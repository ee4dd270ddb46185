// control_pipeline.cuh -- the control-rate part of the Voice as separate
// module kernels over device buffers (used by the plain render and by the
// adjoint's forward recomputation).
#pragma once

#include "control_ff.cuh"
#include "internal.h"
#include "render_common.cuh"

namespace synth {

struct ControlBuffers {
  double* y;          // [B][78] human-range parameters (FP64)
  VoiceFF* vff;       // [B] per-voice constants
  ff* env;            // [B][6][P] ADSRs at the control points
  double* lfo_inc;    // [B][2][P] LFO phase increment per control interval
  double* lfo_phase;  // [B][2][P] LFO phase (cycles, wrapped)
  ff* dest;           // [B][5][P] modulation mixer outputs
  SegVco* seg;        // [B][2][K] VCO interval descriptions
  double* seg_sum;    // [B][2][K] phase advanced over each interval
  double* seg_start;  // [B][2][K] phase at each interval start (wrapped)
  float* kappa;       // [B][2][K] square-saw drive and 1/tanh(drive)
  float* mixc;        // [B][5] mixer gains (3), square-saw shape, 1 / (1 + shape)
};

// Bytes of the control buffers for `batch` voices (256-byte aligned sections).
size_t control_bytes(const VoiceConst& vc, int batch);
ControlBuffers control_carve(const VoiceConst& vc, int batch, void* ws);
// params -> ... -> interval start phases (10 kernels on `st`).
void launch_control_pipeline(const VoiceConst& vc, uint64_t seed, uint64_t batch_index, int batch,
                             const float* params_in, float* params_out, const ControlBuffers& cb,
                             cudaStream_t st);
// The same buffers, bit for bit, from one kernel (one CTA per voice, the
// steps separated by barriers); hdr takes the bounds-checked build's errors.
void launch_control_fused(const VoiceConst& vc, uint64_t seed, uint64_t batch_index, int batch,
                          const float* params_in, float* params_out, const ControlBuffers& cb,
                          ScratchHeader* hdr, cudaStream_t st);

}  // namespace synth
