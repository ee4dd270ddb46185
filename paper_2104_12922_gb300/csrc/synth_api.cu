// synth_api.cu -- the C ABI of libsynth.so (declared in include/synth.h):
// handle lifetime, argument checks, launches, lazy device-error reporting.

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "gemm_tc.h"
#include "internal.h"
#include "mlp.h"
#include "render_common.cuh"
#include "spectral.h"
#include "synth.h"

using namespace synth;

struct synth_handle_s {
  synth_config cfg;
  synth_nebula nebula;
  VoiceConst vc;
  int device = 0;
  int num_sms = 0;
  int fused_grid = 0;
  int n_windows = 0;
  void* scratch = nullptr;  // two slots of ScratchHeader + TileState[max_batch * n_windows]
                            // + the voices' set-up records [max_batch]
  size_t scratch_bytes = 0;  // per slot (256-byte multiple)
  size_t setup_offset = 0;   // of the set-up records within a slot (16-byte multiple)
  int next_slot = 0;         // slot of the next overlappable fused launch
  bool plain_ready = false;
};

namespace {

const double kPi = 3.14159265358979323846;

// The library's default nebula n0 (Sec. 3.3 ranges, curves, symmetric flags).
void fill_default_nebula(synth_nebula* nb) {
  auto set = [&](int i, double lo, double hi, double c, int sym) {
    nb->lo[i] = lo; nb->hi[i] = hi; nb->curve[i] = c; nb->symmetric[i] = sym;
  };
  set(kMidi, 0.0, 127.0, 1.0, 0);
  set(kDuration, 0.0, 4.0, 1.0, 0);
  for (int a = 0; a < 6; ++a) {
    const int b = kAdsr + 5 * a;
    set(b + 0, 0.0, 2.0, 2.0, 0);   // attack s
    set(b + 1, 0.0, 2.0, 2.0, 0);   // decay s
    set(b + 2, 0.0, 1.0, 1.0, 0);   // sustain
    set(b + 3, 0.0, 5.0, 2.0, 0);   // release s
    set(b + 4, 0.1, 6.0, 2.0, 0);   // alpha
  }
  for (int l = 0; l < 2; ++l) {
    const int b = kLfo + 8 * l;
    set(b + 0, 0.0, kLfoMaxHz, 2.0, 0);
    set(b + 1, -20.0, 20.0, 3.0, 1);
    set(b + 2, -kPi, kPi, 1.0, 1);
    for (int s = 0; s < 5; ++s) set(b + 3 + s, 0.0, 1.0, 1.0, 0);
  }
  for (int i = 0; i < 20; ++i) set(kMod + i, 0.0, 1.0, 2.0, 0);
  set(kSine + 0, -24.0, 24.0, 1.0, 1);
  set(kSine + 1, -96.0, 96.0, 3.0, 1);
  set(kSine + 2, -kPi, kPi, 1.0, 1);
  set(kSqr + 0, -24.0, 24.0, 1.0, 1);
  set(kSqr + 1, -96.0, 96.0, 3.0, 1);
  set(kSqr + 2, -kPi, kPi, 1.0, 1);
  set(kSqr + 3, 0.0, 1.0, 1.0, 0);
  for (int i = 0; i < 3; ++i) set(kMix + i, 0.0, 1.0, 1.0, 0);
}

// Host copy of the Sec. 3.3 map (for synth_params_to_human).
double host_range_map(double u, double lo, double hi, double c, int sym) {
  auto cp = [&](double x) {
    if (c == 1.0) return x;
    if (c == 2.0) return x * x;
    if (c == 3.0) return x * x * x;
    return x <= 0.0 ? 0.0 : std::pow(x, c);
  };
  if (!sym) return lo + (hi - lo) * cp(u);
  const double s = 2.0 * u - 1.0;
  const double a = cp(std::fabs(s));
  return lo + (hi - lo) * (1.0 + (s < 0.0 ? -a : a)) * 0.5;
}

synth_status check_cuda(cudaError_t e) { return e == cudaSuccess ? SYNTH_OK : SYNTH_ERR_CUDA; }

bool valid_handle(synth_handle h) { return h != nullptr && h->scratch != nullptr; }

// Scratch slot s (0 or 1): its header and tile states. Slot 0 also carries
// the error word of every other kernel that reports one.
ScratchHeader* slot_header(synth_handle h, int s) {
  return reinterpret_cast<ScratchHeader*>(static_cast<char*>(h->scratch) + (size_t)s * h->scratch_bytes);
}

// The slot for the next fused launch that may overlap the previous one on
// the stream: consecutive such launches alternate slots, so two that overlap
// never share scratch.
ScratchHeader* take_overlap_slot(synth_handle h) {
  ScratchHeader* hdr = slot_header(h, h->next_slot);
  h->next_slot ^= 1;
  return hdr;
}

// The voice set-up records of the slot whose header is hdr.
void* slot_voice_setups(synth_handle h, ScratchHeader* hdr) {
  return reinterpret_cast<char*>(hdr) + h->setup_offset;
}

}  // namespace

extern "C" {

void synth_default_nebula(synth_nebula* out) {
  if (out) fill_default_nebula(out);
}

void synth_default_config(synth_config* out) {
  if (!out) return;
  out->sample_rate = 44100.0;
  out->control_rate = 441.0;
  out->seconds = 4.0;
  out->max_batch = 128;
  out->carry = SYNTH_CARRY_FIXED64;
  out->nebula = nullptr;
}

synth_status synth_create(const synth_config* cfg, synth_handle* out) {
  if (!cfg || !out) return SYNTH_ERR_ARG;
  *out = nullptr;
  const double sr = cfg->sample_rate, cr = cfg->control_rate;
  if (!(sr > 0.0) || !(cr > 0.0) || !(cfg->seconds > 0.0) || cfg->max_batch < 1)
    return SYNTH_ERR_ARG;
  if (cfg->carry != SYNTH_CARRY_FIXED64 && cfg->carry != SYNTH_CARRY_FP32) return SYNTH_ERR_ARG;
  VoiceConst geo{};
  if (!voice_geometry(geo, sr, cr, cfg->seconds)) return SYNTH_ERR_UNSUPPORTED;
  if (geo.general_r && cfg->carry == SYNTH_CARRY_FP32) return SYNTH_ERR_UNSUPPORTED;
  synth_handle h = new (std::nothrow) synth_handle_s();
  if (!h) return SYNTH_ERR_OOM;
  h->cfg = *cfg;
  if (cfg->nebula) h->nebula = *cfg->nebula;
  else fill_default_nebula(&h->nebula);
  h->cfg.nebula = &h->nebula;
  for (int p = 0; p < kNumParams; ++p) {
    if (!(h->nebula.curve[p] > 0.0)) { delete h; return SYNTH_ERR_ARG; }
    h->vc.lo[p] = h->nebula.lo[p];
    h->vc.hi[p] = h->nebula.hi[p];
    h->vc.curve[p] = h->nebula.curve[p];
    h->vc.sym[p] = h->nebula.symmetric[p] ? 1 : 0;
  }
  h->vc.sample_rate = sr;
  h->vc.control_rate = cr;
  h->vc.m_nyq = 69.0 + 12.0 * std::log2(0.5 * sr / 440.0);
  h->vc.n_samples = geo.n_samples;
  h->vc.rate_a = geo.rate_a;
  h->vc.rate_b = geo.rate_b;
  h->vc.general_r = geo.general_r;
  h->vc.R = geo.R;
  h->vc.K = geo.K;
  h->vc.carry_fp32 = cfg->carry == SYNTH_CARRY_FP32 ? 1 : 0;
  voice_const_derive(h->vc);
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
    delete h;
    return SYNTH_ERR_CUDA;
  }
  h->n_windows = windows_per_voice(h->vc.K);
  const int per_sm = fused_max_active_blocks_per_sm();
  h->fused_grid = h->num_sms * (per_sm > 0 ? per_sm : 1);
  h->setup_offset = (sizeof(ScratchHeader) + sizeof(TileState) * (size_t)cfg->max_batch * h->n_windows +
                     15) & ~size_t(15);
  h->scratch_bytes = (h->setup_offset + fused_voice_setup_bytes() * (size_t)cfg->max_batch + 255) &
                     ~size_t(255);
  if (cudaMalloc(&h->scratch, 2 * h->scratch_bytes) != cudaSuccess) {
    h->scratch = nullptr;
    delete h;
    return SYNTH_ERR_OOM;
  }
  if (cudaMemset(h->scratch, 0, 2 * h->scratch_bytes) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    cudaFree(h->scratch);
    delete h;
    return SYNTH_ERR_CUDA;
  }
  *out = h;
  return SYNTH_OK;
}

synth_status synth_destroy(synth_handle h) {
  if (!h) return SYNTH_ERR_ARG;
  if (h->scratch) cudaFree(h->scratch);
  h->scratch = nullptr;
  delete h;
  return SYNTH_OK;
}

int32_t synth_num_params(synth_handle h) { return h ? kNumParams : -1; }
int64_t synth_num_samples(synth_handle h) { return h ? h->vc.n_samples : -1; }

synth_status synth_render(synth_handle h, uint64_t seed, uint64_t batch_index, int32_t batch,
                          const float* params_in_dev, float* audio_dev, float* params_out_dev,
                          void* stream) {
  if (!valid_handle(h)) return SYNTH_ERR_STATE;
  if (batch < 0 || batch > h->cfg.max_batch) return SYNTH_ERR_ARG;
  if (batch == 0) return SYNTH_OK;
  if (!audio_dev) return SYNTH_ERR_ARG;
  ScratchHeader* hdr = take_overlap_slot(h);
  TileState* tiles = reinterpret_cast<TileState*>(hdr + 1);
  return check_cuda(launch_render_fused(h->vc, seed, batch_index * (uint64_t)batch, 0, batch,
                                        params_in_dev, audio_dev, params_out_dev, hdr, tiles,
                                        h->fused_grid, static_cast<cudaStream_t>(stream), nullptr,
                                        0, 0, true, slot_voice_setups(h, hdr)));
}

synth_status synth_render_batches(synth_handle h, uint64_t seed, uint64_t seed_step,
                                  uint64_t batch_index, int32_t batch, int32_t count,
                                  const float* params_in_dev, float* audio_dev,
                                  float* params_out_dev, void* stream) {
  if (!valid_handle(h)) return SYNTH_ERR_STATE;
  if (batch < 0 || count < 0 || (int64_t)batch * count > h->cfg.max_batch) return SYNTH_ERR_ARG;
  if (batch == 0 || count == 0) return SYNTH_OK;
  if (!audio_dev) return SYNTH_ERR_ARG;
  ScratchHeader* hdr = take_overlap_slot(h);
  TileState* tiles = reinterpret_cast<TileState*>(hdr + 1);
  return check_cuda(launch_render_fused(h->vc, seed, batch_index * (uint64_t)batch, 0,
                                        batch * count, params_in_dev, audio_dev, params_out_dev,
                                        hdr, tiles, h->fused_grid,
                                        static_cast<cudaStream_t>(stream), nullptr, seed_step,
                                        batch, true, slot_voice_setups(h, hdr)));
}

synth_status synth_render_normalized(synth_handle h, uint64_t seed, uint64_t batch_index,
                                    int32_t batch, const float* params_in_dev, float* audio_dev,
                                    float* params_out_dev, float threshold, float* peak_out_dev,
                                    int32_t* silent_out_dev, void* stream) {
  if (!valid_handle(h)) return SYNTH_ERR_STATE;
  if (batch < 0 || batch > h->cfg.max_batch) return SYNTH_ERR_ARG;
  if (!(threshold >= 0.f)) return SYNTH_ERR_ARG;
  if (batch == 0) return SYNTH_OK;
  if (!audio_dev) return SYNTH_ERR_ARG;
  ScratchHeader* hdr = take_overlap_slot(h);
  TileState* tiles = reinterpret_cast<TileState*>(hdr + 1);
  const PeakNormArgs norm{threshold, peak_out_dev, silent_out_dev};
  return check_cuda(launch_render_fused(h->vc, seed, batch_index * (uint64_t)batch, 0, batch,
                                        params_in_dev, audio_dev, params_out_dev, hdr, tiles,
                                        h->fused_grid, static_cast<cudaStream_t>(stream), &norm,
                                        0, 0, true, slot_voice_setups(h, hdr)));
}

synth_status synth_fm_render(synth_handle h, uint64_t seed, uint64_t batch_index, int32_t batch,
                             const float* params_in_dev, float* audio_dev, float* params_out_dev,
                             void* stream) {
  if (!valid_handle(h)) return SYNTH_ERR_STATE;
  if (batch < 0 || batch > h->cfg.max_batch || batch > 65535) return SYNTH_ERR_ARG;
  if (batch == 0) return SYNTH_OK;
  if (!audio_dev) return SYNTH_ERR_ARG;
  return check_cuda(launch_fm_render(h->vc, seed, batch_index, batch, params_in_dev, audio_dev,
                                     params_out_dev, static_cast<cudaStream_t>(stream)));
}

synth_status synth_render_plain_workspace_size(synth_handle h, int32_t batch, size_t* bytes) {
  if (!valid_handle(h)) return SYNTH_ERR_STATE;
  if (!bytes || batch < 0 || batch > h->cfg.max_batch) return SYNTH_ERR_ARG;
  if (h->vc.general_r) return SYNTH_ERR_UNSUPPORTED;
  *bytes = plain_workspace_bytes(h->vc, batch);
  return SYNTH_OK;
}

synth_status synth_render_plain(synth_handle h, uint64_t seed, uint64_t batch_index, int32_t batch,
                                const float* params_in_dev, float* audio_dev, float* params_out_dev,
                                void* workspace_dev, size_t workspace_bytes, void* stream) {
  if (!valid_handle(h)) return SYNTH_ERR_STATE;
  if (batch < 0 || batch > h->cfg.max_batch) return SYNTH_ERR_ARG;
  if (h->vc.general_r) return SYNTH_ERR_UNSUPPORTED;
  if (batch == 0) return SYNTH_OK;
  if (!audio_dev || !workspace_dev) return SYNTH_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(workspace_dev) % 256 != 0) return SYNTH_ERR_ARG;
  if (workspace_bytes < plain_workspace_bytes(h->vc, batch)) return SYNTH_ERR_ARG;
  ScratchHeader* hdr = static_cast<ScratchHeader*>(h->scratch);
  TileState* tiles = reinterpret_cast<TileState*>(hdr + 1);
  return check_cuda(launch_render_plain(h->vc, seed, batch_index, batch, params_in_dev, audio_dev,
                                        params_out_dev, workspace_dev, hdr, tiles,
                                        static_cast<cudaStream_t>(stream)));
}

synth_status synth_render_backward_workspace_size(synth_handle h, int32_t batch, size_t* bytes) {
  if (!valid_handle(h)) return SYNTH_ERR_STATE;
  if (!bytes || batch < 0 || batch > h->cfg.max_batch) return SYNTH_ERR_ARG;
  if (h->vc.general_r) return SYNTH_ERR_UNSUPPORTED;
  *bytes = backward_workspace_bytes(h->vc, batch);
  return SYNTH_OK;
}

synth_status synth_render_backward(synth_handle h, uint64_t seed, uint64_t batch_index,
                                   int32_t batch, const float* params_dev,
                                   const float* grad_audio_dev, float* grad_params_dev,
                                   void* workspace_dev, size_t workspace_bytes, void* stream) {
  if (!valid_handle(h)) return SYNTH_ERR_STATE;
  if (batch < 0 || batch > h->cfg.max_batch) return SYNTH_ERR_ARG;
  if (h->vc.general_r) return SYNTH_ERR_UNSUPPORTED;
  if (batch == 0) return SYNTH_OK;
  if (!params_dev || !grad_audio_dev || !grad_params_dev || !workspace_dev) return SYNTH_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(workspace_dev) % 256 != 0) return SYNTH_ERR_ARG;
  if (workspace_bytes < backward_workspace_bytes(h->vc, batch)) return SYNTH_ERR_ARG;
  if (h->vc.R > 128) return SYNTH_ERR_UNSUPPORTED;
  return check_cuda(launch_render_backward(h->vc, seed, batch_index, batch, params_dev,
                                           grad_audio_dev, grad_params_dev, workspace_dev,
                                           static_cast<ScratchHeader*>(h->scratch),
                                           static_cast<cudaStream_t>(stream)));
}

synth_status synth_gemm_bf16_workspace_size(synth_handle h, int32_t m, int32_t n, size_t* bytes) {
  if (!valid_handle(h)) return SYNTH_ERR_STATE;
  if (!bytes || m < 1 || n < 1) return SYNTH_ERR_ARG;
  *bytes = gemm_splitk_workspace_bytes(m, n);
  return *bytes ? SYNTH_OK : SYNTH_ERR_CUDA;
}

synth_status synth_gemm_bf16_splitk(synth_handle h, const void* a_dev, int32_t lda,
                                    const void* b_dev, int32_t ldb, float* c_dev, int32_t ldc,
                                    int32_t m, int32_t n, int32_t k, float alpha,
                                    void* workspace_dev, size_t workspace_bytes, void* stream) {
  if (!valid_handle(h)) return SYNTH_ERR_STATE;
  if (!a_dev || !b_dev || !c_dev || m < 1 || n < 1 || k < 8 || (k % 8) != 0 || lda < k ||
      ldb < k || ldc < n || (lda % 8) != 0 || (ldb % 8) != 0)
    return SYNTH_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(a_dev) & 15) || (reinterpret_cast<uintptr_t>(b_dev) & 15) ||
      (reinterpret_cast<uintptr_t>(workspace_dev) & 15))
    return SYNTH_ERR_ARG;
  GemmEpilogue epi;
  epi.kind = kEpiStoreF32;
  epi.out_f32 = c_dev;
  epi.ldc = ldc;
  epi.alpha = alpha;
  ScratchHeader* hdr = static_cast<ScratchHeader*>(h->scratch);
  return check_cuda(gemm_bf16(static_cast<const __nv_bfloat16*>(a_dev), lda,
                              static_cast<const __nv_bfloat16*>(b_dev), ldb, m, n, k, epi,
                              &hdr->error, static_cast<cudaStream_t>(stream),
                              static_cast<float*>(workspace_dev),
                              workspace_dev ? workspace_bytes : 0));
}

synth_status synth_gemm_bf16(synth_handle h, const void* a_dev, int32_t lda, const void* b_dev,
                             int32_t ldb, float* c_dev, int32_t ldc, int32_t m, int32_t n,
                             int32_t k, float alpha, void* stream) {
  if (!valid_handle(h)) return SYNTH_ERR_STATE;
  if (!a_dev || !b_dev || !c_dev || m < 1 || n < 1 || k < 8 || (k % 8) != 0 || lda < k ||
      ldb < k || ldc < n || (lda % 8) != 0 || (ldb % 8) != 0)
    return SYNTH_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(a_dev) & 15) || (reinterpret_cast<uintptr_t>(b_dev) & 15))
    return SYNTH_ERR_ARG;
  GemmEpilogue epi;
  epi.kind = kEpiStoreF32;
  epi.out_f32 = c_dev;
  epi.ldc = ldc;
  epi.alpha = alpha;
  ScratchHeader* hdr = static_cast<ScratchHeader*>(h->scratch);
  return check_cuda(gemm_bf16(static_cast<const __nv_bfloat16*>(a_dev), lda,
                              static_cast<const __nv_bfloat16*>(b_dev), ldb, m, n, k, epi,
                              &hdr->error, static_cast<cudaStream_t>(stream)));
}

// ---------------------------------------------------------------- MMD
synth_status synth_l1_distances(synth_handle h, const void* emb_dev, int64_t ld, int32_t m,
                                int32_t dim, float* dist_dev, void* stream) {
  if (!valid_handle(h)) return SYNTH_ERR_STATE;
  if (m < 0 || dim < 1 || ld < dim || (ld % 8) != 0 || (m > 0 && (!emb_dev || !dist_dev)) ||
      (reinterpret_cast<uintptr_t>(emb_dev) & 15) || (int64_t)m * ld >= ((int64_t)1 << 40))
    return SYNTH_ERR_ARG;
  return check_cuda(launch_l1_distances(static_cast<const __nv_bfloat16*>(emb_dev), ld, m, dim,
                                        dist_dev, static_cast<cudaStream_t>(stream)));
}

synth_status synth_mmd_trials(synth_handle h, const float* dist_dev, int32_t m,
                              const int8_t* labels_dev, int32_t trials, double* mmd_dev,
                              void* stream) {
  if (!valid_handle(h)) return SYNTH_ERR_STATE;
  if (m < 1 || m > 48 * 1024 || trials < 0 ||
      (trials > 0 && (!dist_dev || !labels_dev || !mmd_dev)))
    return SYNTH_ERR_ARG;
  return check_cuda(launch_mmd_trials(dist_dev, m, labels_dev, trials, mmd_dev,
                                      static_cast<cudaStream_t>(stream)));
}

// ---------------------------------------------------------------- MR-STFT
static const int kMrFFT[3] = {512, 1024, 2048};

synth_status synth_mrstft_workspace_size(synth_handle h, int32_t batch, size_t* bytes) {
  if (!valid_handle(h)) return SYNTH_ERR_STATE;
  if (!bytes || batch < 1) return SYNTH_ERR_ARG;
  if (h->vc.n_samples < 2048) return SYNTH_ERR_UNSUPPORTED;
  *bytes = mrstft_workspace_bytes(h->vc.n_samples, batch, kMrFFT, 3);
  return SYNTH_OK;
}

synth_status synth_mrstft(synth_handle h, const float* x_dev, const float* y_dev, int32_t batch,
                          int32_t target_ready, double* loss_voice_dev, float* grad_x_dev,
                          void* workspace_dev, size_t workspace_bytes, void* stream) {
  if (!valid_handle(h)) return SYNTH_ERR_STATE;
  if (batch < 1 || !x_dev || !y_dev || !workspace_dev) return SYNTH_ERR_ARG;
  if (h->vc.n_samples < 2048) return SYNTH_ERR_UNSUPPORTED;
  if (reinterpret_cast<uintptr_t>(workspace_dev) % 256 != 0) return SYNTH_ERR_ARG;
  if (workspace_bytes < mrstft_workspace_bytes(h->vc.n_samples, batch, kMrFFT, 3))
    return SYNTH_ERR_ARG;
  ScratchHeader* hdr = static_cast<ScratchHeader*>(h->scratch);
  return check_cuda(mrstft_loss_grad(x_dev, y_dev, h->vc.n_samples, batch, kMrFFT, 3, 1e-7f,
                                     target_ready != 0, loss_voice_dev, grad_x_dev, workspace_dev,
                                     &hdr->error, static_cast<cudaStream_t>(stream)));
}

synth_status synth_param_adam(synth_handle h, float* u_dev, const float* grad_dev, float* m_dev,
                              float* v_dev, int32_t count, int32_t step, float lr, void* stream) {
  if (!valid_handle(h)) return SYNTH_ERR_STATE;
  if (!u_dev || !grad_dev || !m_dev || !v_dev || count < 1 || step < 1 || !(lr > 0.f))
    return SYNTH_ERR_ARG;
  return check_cuda(param_adam(u_dev, grad_dev, m_dev, v_dev, count, step, lr,
                               static_cast<cudaStream_t>(stream)));
}

// ------------------------------------------------------------ proposal model
struct synth_model_s {
  synth_handle synth = nullptr;
  MlpLayout L;
  char* mem = nullptr;        // MlpLayout tensors
  void* work = nullptr;       // audio, params, features, log-mel workspace
  float* audio = nullptr;     // [max_batch][N]
  float* params = nullptr;    // [max_batch][78]
  __nv_bfloat16* feats = nullptr;  // [max_batch][frames * 128]
  void* mel_ws = nullptr;
  int max_batch = 0;
  int frames = 0;
  int step = 0;
  int last_batch = 0;  // batch of the last forward or training step
};

static const int kHidden = 1024;

synth_status synth_model_create(synth_handle h, int32_t max_batch, uint64_t seed, synth_model* out) {
  if (!valid_handle(h)) return SYNTH_ERR_STATE;
  if (!out || max_batch < 8 || max_batch % 8 != 0 || max_batch > h->cfg.max_batch) return SYNTH_ERR_ARG;
  if (h->vc.n_samples < kMelFFT) return SYNTH_ERR_UNSUPPORTED;
  *out = nullptr;
  synth_model m = new (std::nothrow) synth_model_s();
  if (!m) return SYNTH_ERR_OOM;
  m->synth = h;
  m->max_batch = max_batch;
  m->frames = stft_frames(h->vc.n_samples, kMelFFT);
  m->L = mlp_layout(m->frames * kMelBands, kHidden, kNumParams, max_batch,
                    gemm_splitk_workspace_bytes(max_batch, kHidden));
  const size_t N = (size_t)h->vc.n_samples;
  const size_t a_bytes = (sizeof(float) * max_batch * N + 255) & ~size_t(255);
  const size_t p_bytes = (sizeof(float) * max_batch * kNumParams + 255) & ~size_t(255);
  const size_t f_bytes = (sizeof(__nv_bfloat16) * max_batch * m->frames * kMelBands + 255) & ~size_t(255);
  const size_t mel_bytes = logmel_fft_table_bytes();
  if (cudaMalloc(reinterpret_cast<void**>(&m->mem), m->L.total) != cudaSuccess) {
    delete m;
    return SYNTH_ERR_OOM;
  }
  if (cudaMalloc(&m->work, a_bytes + p_bytes + f_bytes + mel_bytes) != cudaSuccess) {
    cudaFree(m->mem);
    delete m;
    return SYNTH_ERR_OOM;
  }
  char* w = static_cast<char*>(m->work);
  m->audio = reinterpret_cast<float*>(w);
  m->params = reinterpret_cast<float*>(w + a_bytes);
  m->feats = reinterpret_cast<__nv_bfloat16*>(w + a_bytes + p_bytes);
  m->mel_ws = w + a_bytes + p_bytes + f_bytes;
  if (mlp_init(m->L, m->mem, seed, 0) != cudaSuccess ||
      logmel_fft_init(h->vc.sample_rate, m->mel_ws, 0) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    cudaFree(m->mem);
    cudaFree(m->work);
    delete m;
    return SYNTH_ERR_CUDA;
  }
  *out = m;
  return SYNTH_OK;
}

synth_status synth_model_destroy(synth_model m) {
  if (!m) return SYNTH_ERR_ARG;
  cudaFree(m->mem);
  cudaFree(m->work);
  delete m;
  return SYNTH_OK;
}

int64_t synth_model_feature_dim(synth_model m) {
  return m ? (int64_t)m->frames * kMelBands : -1;
}

synth_status synth_model_features(synth_model m, const float* audio_dev, int32_t batch,
                                  void* features_dev, void* stream) {
  if (!m) return SYNTH_ERR_STATE;
  if (!audio_dev || !features_dev || batch < 1 || batch > m->max_batch) return SYNTH_ERR_ARG;
  return check_cuda(logmel_features_fft(audio_dev, m->synth->vc.n_samples, batch, m->mel_ws,
                                        static_cast<__nv_bfloat16*>(features_dev),
                                        static_cast<cudaStream_t>(stream)));
}

synth_status synth_stream_features(synth_model m, uint64_t seed, int32_t split, uint64_t first,
                                   int64_t count, int32_t chunk, void* features_dev,
                                   float* params_dev, void* stream) {
  if (!m) return SYNTH_ERR_STATE;
  if (split < 0 || split > 2 || count < 0 || chunk < 0 || chunk > m->max_batch) return SYNTH_ERR_ARG;
  if (count == 0) return SYNTH_OK;
  if (!features_dev) return SYNTH_ERR_ARG;
  synth_handle h = m->synth;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  ScratchHeader* hdr = static_cast<ScratchHeader*>(h->scratch);
  TileState* tiles = reinterpret_cast<TileState*>(hdr + 1);
  const int64_t fdim = (int64_t)m->frames * kMelBands;
  const int c_max = chunk > 0 ? chunk : m->max_batch;
  __nv_bfloat16* feats = static_cast<__nv_bfloat16*>(features_dev);
  for (int64_t off = 0; off < count; off += c_max) {
    const int c = (int)std::min<int64_t>(c_max, count - off);
    cudaError_t e = launch_render_fused(h->vc, seed, first + (uint64_t)off, split, c, nullptr,
                                        m->audio, params_dev ? params_dev + off * kNumParams : nullptr,
                                        hdr, tiles, h->fused_grid, st, nullptr, 0, 0, false,
                                        slot_voice_setups(h, hdr));
    if (e != cudaSuccess) return SYNTH_ERR_CUDA;
    e = logmel_features_fft(m->audio, h->vc.n_samples, c, m->mel_ws, feats + off * fdim, st);
    if (e != cudaSuccess) return SYNTH_ERR_CUDA;
  }
  return SYNTH_OK;
}

synth_status synth_model_forward(synth_model m, const void* features_dev, int32_t batch,
                                 float* params_out_dev, void* stream) {
  if (!m) return SYNTH_ERR_STATE;
  if (!features_dev || !params_out_dev || batch < 1 || batch > m->max_batch) return SYNTH_ERR_ARG;
  ScratchHeader* hdr = static_cast<ScratchHeader*>(m->synth->scratch);
  m->last_batch = batch;
  return check_cuda(mlp_forward(m->L, m->mem, static_cast<const __nv_bfloat16*>(features_dev), batch,
                                false, params_out_dev, &hdr->error,
                                static_cast<cudaStream_t>(stream)));
}

synth_status synth_model_train_features(synth_model m, const void* features_dev,
                                        const float* target_dev, int32_t batch, float lr,
                                        float* loss_dev, void* stream) {
  if (!m) return SYNTH_ERR_STATE;
  if (!features_dev || !target_dev || batch < 8 || batch % 8 != 0 || batch > m->max_batch ||
      !(lr > 0.f))
    return SYNTH_ERR_ARG;
  ScratchHeader* hdr = static_cast<ScratchHeader*>(m->synth->scratch);
  m->step += 1;
  m->last_batch = batch;
  return check_cuda(mlp_train_step(m->L, m->mem, static_cast<const __nv_bfloat16*>(features_dev),
                                   target_dev, batch, lr, m->step, loss_dev, &hdr->error,
                                   static_cast<cudaStream_t>(stream)));
}

synth_status synth_model_train_step(synth_model m, uint64_t seed, uint64_t batch_index,
                                    int32_t batch, float lr, float* loss_dev, void* stream) {
  if (!m) return SYNTH_ERR_STATE;
  if (batch < 8 || batch % 8 != 0 || batch > m->max_batch || !(lr > 0.f)) return SYNTH_ERR_ARG;
  synth_status s = synth_render(m->synth, seed, batch_index, batch, nullptr, m->audio, m->params,
                                stream);
  if (s != SYNTH_OK) return s;
  s = synth_model_features(m, m->audio, batch, m->feats, stream);
  if (s != SYNTH_OK) return s;
  return synth_model_train_features(m, m->feats, m->params, batch, lr, loss_dev, stream);
}

synth_status synth_propose(synth_handle h, synth_model m, const float* audio_dev, int32_t batch,
                           float* params_out_dev, void* stream) {
  if (!valid_handle(h) || !m || m->synth != h) return SYNTH_ERR_STATE;
  if (!audio_dev || !params_out_dev || batch < 1 || batch > m->max_batch) return SYNTH_ERR_ARG;
  synth_status s = synth_model_features(m, audio_dev, batch, m->feats, stream);
  if (s != SYNTH_OK) return s;
  return synth_model_forward(m, m->feats, batch, params_out_dev, stream);
}

// which: 0 weights [out][in], 1 biases [out], 2 weight gradients, 3 bias
// gradients (FP32); layer 0..3.
static float* model_tensor(synth_model m, int32_t which, int32_t layer, size_t* count) {
  if (!m || layer < 0 || layer > 3 || which < 0 || which > 3) return nullptr;
  const size_t in = m->L.dims[layer], out = m->L.dims[layer + 1];
  const size_t off[4] = {m->L.w[layer], m->L.b[layer], m->L.gw[layer], m->L.gb[layer]};
  *count = (which == 0 || which == 2) ? in * out : out;
  return reinterpret_cast<float*>(m->mem + off[which]);
}

synth_status synth_model_get_tensor(synth_model m, int32_t which, int32_t layer, float* dst_dev,
                                    size_t count, void* stream) {
  if (m && which == 4) {
    // hidden activations of the last forward / training step, bf16 -> FP32
    if (layer < 1 || layer > 3 || !dst_dev || m->last_batch < 1 ||
        count != (size_t)m->last_batch * kHidden)
      return SYNTH_ERR_ARG;
    return check_cuda(mlp_hidden_f32(m->L, m->mem, layer, m->last_batch, dst_dev,
                                     static_cast<cudaStream_t>(stream)));
  }
  size_t n = 0;
  float* src = model_tensor(m, which, layer, &n);
  if (!src || !dst_dev || count != n) return SYNTH_ERR_ARG;
  return check_cuda(cudaMemcpyAsync(dst_dev, src, n * sizeof(float), cudaMemcpyDeviceToDevice,
                                    static_cast<cudaStream_t>(stream)));
}

synth_status synth_model_save(synth_model m, const char* path) {
  if (!m || !path) return SYNTH_ERR_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return SYNTH_ERR_CUDA;
  FILE* f = std::fopen(path, "wb");
  if (!f) return SYNTH_ERR_ARG;
  std::vector<char> host(m->L.total);
  bool ok = cudaMemcpy(host.data(), m->mem, m->L.total, cudaMemcpyDeviceToHost) == cudaSuccess;
  const uint64_t magic = 0x53594e544d4f444cull, total = m->L.total;
  const int64_t step = m->step;
  ok = ok && std::fwrite(&magic, 8, 1, f) == 1 && std::fwrite(&total, 8, 1, f) == 1 &&
       std::fwrite(&step, 8, 1, f) == 1 && std::fwrite(host.data(), 1, host.size(), f) == host.size();
  std::fclose(f);
  return ok ? SYNTH_OK : SYNTH_ERR_CUDA;
}

synth_status synth_model_load(synth_model m, const char* path) {
  if (!m || !path) return SYNTH_ERR_ARG;
  FILE* f = std::fopen(path, "rb");
  if (!f) return SYNTH_ERR_ARG;
  uint64_t magic = 0, total = 0;
  int64_t step = 0;
  bool ok = std::fread(&magic, 8, 1, f) == 1 && std::fread(&total, 8, 1, f) == 1 &&
            std::fread(&step, 8, 1, f) == 1 && magic == 0x53594e544d4f444cull &&
            total == m->L.total;
  std::vector<char> host(ok ? total : 0);
  ok = ok && std::fread(host.data(), 1, host.size(), f) == host.size();
  std::fclose(f);
  if (!ok) return SYNTH_ERR_ARG;
  if (cudaMemcpy(m->mem, host.data(), total, cudaMemcpyHostToDevice) != cudaSuccess)
    return SYNTH_ERR_CUDA;
  m->step = (int)step;
  return SYNTH_OK;
}

synth_status synth_sync(synth_handle h, void* stream) {
  if (!valid_handle(h)) return SYNTH_ERR_STATE;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return SYNTH_ERR_CUDA;
  unsigned int all = 0;
  for (int slot = 0; slot < 2; ++slot) {
    ScratchHeader* hdr = slot_header(h, slot);
    unsigned int err = 0;
    if (cudaMemcpy(&err, &hdr->error, sizeof(err), cudaMemcpyDeviceToHost) != cudaSuccess)
      return SYNTH_ERR_CUDA;
    if (err != 0) {
      const unsigned int zero = 0;
      if (cudaMemcpy(&hdr->error, &zero, sizeof(zero), cudaMemcpyHostToDevice) != cudaSuccess)
        return SYNTH_ERR_CUDA;
      all |= err;
    }
  }
  return status_of_error_word(all);
}

namespace {
// One warp runs the fused render's look-back wait against a window record
// whose flag is never set (probe[0], zeroed by the caller): the bounded wait
// gives up and records kErrLookbackTimeout in the header, as a render whose
// earlier window never published would. Lane 0 alone touches probe[0]
// (window 0 of 1); probe[1] takes the (unused) result.
__global__ void wait_probe_kernel(TileState* probe, ScratchHeader* hdr) {
  unsigned long long e0, e1;
  lookback_consume<unsigned long long>(probe, 1, 0, 1u, e0, e1, hdr);
  if (threadIdx.x == 0) {
    probe[1].agg[0][0] = e0;
    probe[1].agg[0][1] = e1;
  }
}
}  // namespace

namespace {
// The bounds-checked build's self-test: each of 32 threads derives an index
// one range past a 4-element shared array; in_bounds records kErrBounds and
// the store is skipped. The release build has no such kernel body.
__global__ void bounds_probe_kernel(ScratchHeader* hdr, float* sink) {
  if constexpr (kBoundsChecks) {
    __shared__ float a[4];
    if (threadIdx.x < 4) a[threadIdx.x] = 0.f;
    __syncthreads();
    const int i = 4 + (int)threadIdx.x;
    if (in_bounds(hdr, i, 4)) a[i] = 1.f;
    __syncthreads();
    if (threadIdx.x == 0 && sink) *sink = a[0];
  }
}
}  // namespace

int32_t synth_checked_build(void) { return kBoundsChecks ? 1 : 0; }

synth_status synth_selftest_bounds(synth_handle h, void* stream) {
  if (!valid_handle(h)) return SYNTH_ERR_STATE;
  if (!kBoundsChecks) return SYNTH_ERR_UNSUPPORTED;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  bounds_probe_kernel<<<1, 32, 0, st>>>(static_cast<ScratchHeader*>(h->scratch), nullptr);
  if (cudaGetLastError() != cudaSuccess) return SYNTH_ERR_CUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? SYNTH_OK : SYNTH_ERR_CUDA;
}

synth_status synth_selftest_wait_timeout(synth_handle h, void* stream) {
  if (!valid_handle(h)) return SYNTH_ERR_STATE;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  ScratchHeader* hdr = static_cast<ScratchHeader*>(h->scratch);
  TileState* probe = nullptr;
  if (cudaMalloc(&probe, 2 * sizeof(TileState)) != cudaSuccess) return SYNTH_ERR_CUDA;
  cudaError_t e = cudaMemsetAsync(probe, 0, 2 * sizeof(TileState), st);
  if (e == cudaSuccess) {
    wait_probe_kernel<<<1, 32, 0, st>>>(probe, hdr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  const cudaError_t f = cudaFree(probe);
  return (e == cudaSuccess && f == cudaSuccess) ? SYNTH_OK : SYNTH_ERR_CUDA;
}

synth_status synth_params_to_human(synth_handle h, const float* u_host, double* y_host,
                                   int32_t count) {
  if (!h) return SYNTH_ERR_STATE;
  if (count < 0 || (count > 0 && (!u_host || !y_host))) return SYNTH_ERR_ARG;
  for (int32_t i = 0; i < count; ++i)
    for (int p = 0; p < kNumParams; ++p) {
      double u = (double)u_host[(size_t)i * kNumParams + p];
      u = u < 0.0 ? 0.0 : (u > 1.0 ? 1.0 : u);
      y_host[(size_t)i * kNumParams + p] =
          host_range_map(u, h->vc.lo[p], h->vc.hi[p], h->vc.curve[p], h->vc.sym[p]);
    }
  return SYNTH_OK;
}

int32_t synth_is_test(uint64_t g) { return (g % kSplitPeriod) >= kSplitTrain ? 1 : 0; }

uint64_t synth_split_voice(int32_t split, uint64_t i) { return split_voice(split, i); }

const char* synth_status_string(synth_status s) {
  switch (s) {
    case SYNTH_OK: return "ok";
    case SYNTH_ERR_ARG: return "invalid argument";
    case SYNTH_ERR_CUDA: return "CUDA error";
    case SYNTH_ERR_OOM: return "out of memory";
    case SYNTH_ERR_TIMEOUT: return "device-side wait timed out";
    case SYNTH_ERR_STATE: return "invalid handle state";
    case SYNTH_ERR_UNSUPPORTED: return "unsupported configuration";
    case SYNTH_ERR_BOUNDS: return "an index left its range (bounds-checked build)";
  }
  return "unknown status";
}

}  // extern "C"
