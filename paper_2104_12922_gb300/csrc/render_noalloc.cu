// render_noalloc.cu -- the fused render for callers that cannot allocate
// device memory.
//
// synth_create allocates the handle's scratch with cudaMalloc. Some callers
// cannot do that: code that runs while another framework owns every device
// allocation (a plugin inside a host application with its own memory pool,
// or a process that reserved the whole GPU up front), or code on a path
// where an allocation would synchronize the device. synth_render_noalloc
// gives them the same fused render with no handle: its scratch (the work
// counters and the look-back records of the tiles) lives in the fixed
// file-scope device array below, which every GPU that loads the library
// holds until the process exits. The caller still owns the inputs and
// outputs.
//
// The paper has no counterpart to this entry point.

#include <cmath>
#include <cstddef>
#include <mutex>

#include "internal.h"
#include "synth.h"

namespace synth {
namespace {

// Fixed scratch: one ScratchHeader followed by TileState records.
constexpr size_t kNoAllocScratchBytes = 256 * 1024;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};
int g_grid[kMaxDevices] = {};

// Set-up on the current device: the device address of the scratch array
// (host code cannot use the symbol itself) and the persistent grid, looked up
// on the first call. Later calls outside stream capture look the address up
// again and keep the new one if it moved: after cudaDeviceReset the runtime
// loads the module afresh and the array may sit elsewhere. Under capture the
// cached address is used (a lookup could load the module there).
synth_status setup_current_device(cudaStream_t st, int* device_out, void** addr_out,
                                  int* grid_out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SYNTH_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return SYNTH_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_addr[dev]) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusActive;
    if (cudaStreamIsCapturing(st, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusNone) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr)
        return SYNTH_ERR_CUDA;
      g_scratch_addr[dev] = ptr;
    } else {
      cudaGetLastError();  // a failed capture query leaves no sticky error
    }
  } else {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return SYNTH_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return SYNTH_ERR_CUDA;
    const int per_sm = fused_max_active_blocks_per_sm();
    g_grid[dev] = sms * (per_sm > 0 ? per_sm : 1);
    g_scratch_addr[dev] = ptr;
  }
  *device_out = dev;
  *addr_out = g_scratch_addr[dev];
  *grid_out = g_grid[dev];
  return SYNTH_OK;
}

// synth_config -> kernel constants (the same checks synth_create makes).
synth_status voice_const_from_config(const synth_config* cfg, VoiceConst* vc) {
  const double sr = cfg->sample_rate, cr = cfg->control_rate;
  if (!(sr > 0.0) || !(cr > 0.0) || !(cfg->seconds > 0.0)) return SYNTH_ERR_ARG;
  if (cfg->carry != SYNTH_CARRY_FIXED64 && cfg->carry != SYNTH_CARRY_FP32) return SYNTH_ERR_ARG;
  if (!voice_geometry(*vc, sr, cr, cfg->seconds)) return SYNTH_ERR_UNSUPPORTED;
  if (vc->general_r && cfg->carry == SYNTH_CARRY_FP32) return SYNTH_ERR_UNSUPPORTED;
  synth_nebula nb;
  if (cfg->nebula) nb = *cfg->nebula;
  else synth_default_nebula(&nb);
  for (int p = 0; p < kNumParams; ++p) {
    if (!(nb.curve[p] > 0.0)) return SYNTH_ERR_ARG;
    vc->lo[p] = nb.lo[p];
    vc->hi[p] = nb.hi[p];
    vc->curve[p] = nb.curve[p];
    vc->sym[p] = nb.symmetric[p] ? 1 : 0;
  }
  vc->sample_rate = sr;
  vc->control_rate = cr;
  vc->m_nyq = 69.0 + 12.0 * std::log2(0.5 * sr / 440.0);
  vc->carry_fp32 = cfg->carry == SYNTH_CARRY_FP32 ? 1 : 0;
  voice_const_derive(*vc);
  return SYNTH_OK;
}

}  // namespace
}  // namespace synth

using namespace synth;

extern "C" synth_status synth_render_noalloc(const synth_config* cfg, uint64_t seed,
                                             uint64_t batch_index, int32_t batch,
                                             const float* params_in_dev, float* audio_dev,
                                             float* params_out_dev, void* stream) {
  if (!cfg || batch < 0) return SYNTH_ERR_ARG;
  VoiceConst vc;
  synth_status s = voice_const_from_config(cfg, &vc);
  if (s != SYNTH_OK) return s;
  if (batch == 0) return SYNTH_OK;
  if (!audio_dev) return SYNTH_ERR_ARG;
  const size_t tiles = (size_t)batch * (size_t)windows_per_voice(vc.K);
  const size_t need = sizeof(ScratchHeader) + tiles * sizeof(TileState);
  if (need > kNoAllocScratchBytes) return SYNTH_ERR_ARG;  // beyond the fixed scratch
  int dev = 0, grid = 0;
  void* scratch = nullptr;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((s = setup_current_device(st, &dev, &scratch, &grid)) != SYNTH_OK) return s;
  // The scratch keeps the previous call's contents: clear the part this call
  // uses (counters, launch epoch, error word and look-back flags start at 0).
  if (cudaMemsetAsync(scratch, 0, need, st) != cudaSuccess) return SYNTH_ERR_CUDA;
  ScratchHeader* hdr = static_cast<ScratchHeader*>(scratch);
  TileState* ts = reinterpret_cast<TileState*>(hdr + 1);
  return launch_render_fused(vc, seed, batch_index * (uint64_t)batch, 0, batch, params_in_dev, audio_dev,
                             params_out_dev, hdr, ts, grid, st) == cudaSuccess
             ? SYNTH_OK
             : SYNTH_ERR_CUDA;
}

// Waits for `stream`, then reads and clears the error word the last
// synth_render_noalloc call left in the fixed scratch array (through the
// symbol: no address, no allocation). Each call clears that word when it
// starts, so this reports only the most recent call and must come before the
// next one.
extern "C" synth_status synth_noalloc_status(void* stream) {
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return SYNTH_ERR_CUDA;
  unsigned int err = 0;
  const size_t at = offsetof(ScratchHeader, error);
  if (cudaMemcpyFromSymbol(&err, g_noalloc_scratch, sizeof(err), at) != cudaSuccess)
    return SYNTH_ERR_CUDA;
  if (err == 0) return SYNTH_OK;
  const unsigned int zero = 0;
  if (cudaMemcpyToSymbol(g_noalloc_scratch, &zero, sizeof(zero), at) != cudaSuccess)
    return SYNTH_ERR_CUDA;
  return status_of_error_word(err);
}
