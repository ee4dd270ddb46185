// internal.h -- host-side declarations shared by the library's .cu files.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "synth.h"
#include "voice_device.cuh"

namespace synth {

// Device scratch header for the persistent kernels: a work counter, a
// completion counter, a launch epoch that tags look-back flags (so flags of
// an earlier launch are never mistaken for this one's), and an error word.
struct ScratchHeader {
  unsigned int work;
  unsigned int done;
  unsigned int epoch;
  unsigned int error;   // kErr* bits: a bounded wait gave up, an index left its range
  unsigned int pad[60];
};
static_assert(sizeof(ScratchHeader) == 256, "header is one 256-byte block");

// Look-back state of one tile (voice, window) for the two scan chains
// (0: LFO phases, 1: VCO phases), two components each. An aggregate is a
// 64-bit fixed-point phase, or the bits of a float in the FP32-carry mode.
struct TileState {
  unsigned int flag[2];  // (epoch << 2) | 1 once agg[chain] of this launch is published
  unsigned int done;      // (epoch << 2) | 3 once the tile's audio is written (peak variant)
  unsigned int peak;      // the bits of the tile's largest |sample| (peak variant)
  unsigned long long agg[2][2];
};
static_assert(sizeof(TileState) == 48, "tile state layout");

constexpr unsigned int kErrLookbackTimeout = 1u;
constexpr unsigned int kErrTileWaitTimeout = 2u;
constexpr unsigned int kErrBounds = 4u;  // bounds-checked build: an index left its range

// The bounds-checked build (compiled with -DSYNTH_CHECKS into
// libsynth_checked.so; the stand-in for a memory checker, which this
// library's GPUs do not offer): the fused render tests each index it derives
// against the extent of the range it addresses, global (audio, parameters,
// set-up and tile records) or shared (the tile's interval arrays). An index
// outside [0, n) records kErrBounds in the launch's error word and the
// access is skipped, so a wrong index shows up as SYNTH_ERR_BOUNDS from
// synth_sync instead of a fault. In the release build in_bounds is the
// constant true and the checks compile to nothing.
// The status a launch's error word reports: an index out of its range
// first, then a bounded wait that gave up.
inline synth_status status_of_error_word(unsigned int err) {
  if (err & kErrBounds) return SYNTH_ERR_BOUNDS;
  return err ? SYNTH_ERR_TIMEOUT : SYNTH_OK;
}

#if defined(SYNTH_CHECKS)
constexpr bool kBoundsChecks = true;
#else
constexpr bool kBoundsChecks = false;
#endif
__device__ __forceinline__ bool in_bounds(ScratchHeader* hdr, long long i, long long n) {
  if constexpr (!kBoundsChecks) {
    return true;
  } else {
    if (i >= 0 && i < n) return true;
    atomicOr(&hdr->error, kErrBounds);
    return false;
  }
}

constexpr int kFusedThreads = 256;     // one thread per control point of a tile
constexpr int kFusedTilePoints = 256;  // control points per tile of the fused kernel
constexpr int kFusedTileSeg = kFusedTilePoints - 1;  // control intervals per tile

inline int windows_per_voice(int K) { return (K + kFusedTileSeg - 1) / kFusedTileSeg; }

// Sec. 2.2 train/test split of the synth1B1 voice indices: blocks of 1024
// consecutive voices, nine train blocks then one test block, repeating.
// split_voice(split, i) is the global index g of the i-th voice of a split
// (0: every voice, g = i; 1: train; 2: test).
constexpr uint64_t kSplitBlock = 1024;
constexpr uint64_t kSplitPeriod = 10 * kSplitBlock;
constexpr uint64_t kSplitTrain = 9 * kSplitBlock;
__host__ __device__ inline uint64_t split_voice(int split, uint64_t i) {
  if (split == 1) return (i / kSplitTrain) * kSplitPeriod + i % kSplitTrain;
  if (split == 2) return (i / kSplitBlock) * kSplitPeriod + kSplitTrain + i % kSplitBlock;
  return i;
}

// Per-voice peak normalisation inside the fused render: after its last
// render tile the kernel claims normalisation chunks from the same work
// counter, so the scaling pass overlaps the tail of the render.
struct PeakNormArgs {
  float threshold;     // voices with peak >= threshold (and > 0) are scaled to peak 1
  float* peak_out;     // [batch] peak |sample| of each voice as rendered, nullable
  int32_t* silent_out; // [batch] 1 where the voice was left as rendered, nullable
};
constexpr int kNormChunkSamples = 8192;  // samples per normalisation work item

// Launches the fused persistent render of voices g = split_voice(split,
// first + v), v < batch (with `norm`, also the peak normalisation); voice v
// draws with seed + (v / sub_batch) seed_step (sub_batch 0: the whole batch
// one seed). With overlap_previous, the launch may start while the previous
// kernel on the stream finishes (programmatic dependent launch). A fused
// render releases its dependents before it completes, so the request is
// granted only when the previous fused launch on the stream used other
// scratch (hdr) and none of the two launches writes a buffer the other reads
// or writes (params_in, audio, params_out, peak, silent); otherwise the
// launch waits for the previous kernel as usual. Every launch is recorded for
// that check. voice_setups: NULL, or room for `batch` records of
// fused_voice_setup_bytes() each (16-byte aligned) in the same scratch as
// hdr, zeroed before its first use: a voice's first window publishes its
// parameter set-up there and its later windows copy it (epoch-tagged, so
// the records need no clearing between launches). Returns the CUDA error of
// the launch.
cudaError_t launch_render_fused(const VoiceConst& vc, uint64_t seed, uint64_t first, int split,
                                int batch, const float* params_in, float* audio,
                                float* params_out, ScratchHeader* hdr, TileState* tiles,
                                int grid, cudaStream_t stream,
                                const PeakNormArgs* norm = nullptr, uint64_t seed_step = 0,
                                int sub_batch = 0, bool overlap_previous = false,
                                void* voice_setups = nullptr);
size_t fused_voice_setup_bytes();
int fused_max_active_blocks_per_sm();

// The 4-operator FM voice (fm_voice.cu): voices g = batch_index * batch + v.
cudaError_t launch_fm_render(const VoiceConst& vc, uint64_t seed, uint64_t batch_index, int batch,
                             const float* params_in, float* audio, float* params_out,
                             cudaStream_t stream);

// Plain (unfused) form.
size_t plain_workspace_bytes(const VoiceConst& vc, int batch);
cudaError_t launch_render_plain(const VoiceConst& vc, uint64_t seed, uint64_t batch_index,
                                int batch, const float* params_in, float* audio,
                                float* params_out, void* workspace, ScratchHeader* hdr,
                                TileState* tiles, cudaStream_t stream);

// Corpus similarity (mmd.cu): pooled pairwise l1 distances of bf16
// embeddings [m][ld], and the MMD statistic of labelled trials over them.
cudaError_t launch_l1_distances(const __nv_bfloat16* emb, int64_t ld, int m, int dim, float* dist,
                                cudaStream_t st);
cudaError_t launch_mmd_trials(const float* dist, int m, const int8_t* labels, int trials,
                              double* mmd, cudaStream_t st);

// Adjoint.
size_t backward_workspace_bytes(const VoiceConst& vc, int batch);
// hdr: the handle's scratch header, whose error word the bounds-checked
// build's checks write.
cudaError_t launch_render_backward(const VoiceConst& vc, uint64_t seed, uint64_t batch_index,
                                   int batch, const float* params, const float* grad_audio,
                                   float* grad_params, void* workspace, ScratchHeader* hdr,
                                   cudaStream_t stream);

}  // namespace synth
