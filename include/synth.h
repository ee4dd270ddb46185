/*
 * synth.h -- C ABI of libsynth.so, the GB300 (sm_103a) batched Voice renderer.
 *
 * Paper: Turian et al., "One Billion Audio Sounds from GPU-enabled Modular
 * Synthesis" (DAFx 2021). The problem statement the calls follow (Sec. 2.1,
 * 2.2): a batch index and a seed in; a replicable batch of 4 s, 44.1 kHz
 * voices paired with their parameter vectors out; batch 128 by default.
 *
 * Conventions for every call below:
 *  - Pointers named *_dev are CUDA device pointers owned by the caller; the
 *    library never frees them and never allocates inside a render call
 *    (scratch lives in the handle and is sized by synth_config.max_batch).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Calls are stream-ordered and asynchronous unless stated.
 *  - Layouts are row-major and contiguous: audio[batch][N] float32 with
 *    N = round(seconds * sample_rate); params[batch][78] float32 holding the
 *    normalized parameters u in [0,1].
 *  - Global voice index: voice v of a call has g = batch_index * batch + v,
 *    and a voice depends only on (seed, g) -- the same g renders the same
 *    sound in any batch size (Sec. 2.2 replicability).
 *  - Every call returns a synth_status and never aborts. Argument errors are
 *    caught before any launch. A device-side error (a bounded wait that gave
 *    up) is recorded in the handle and returned by synth_sync.
 *  - One handle renders one batch at a time: calls on one handle must be
 *    ordered on one stream (they share the handle's scratch).
 *  - Consecutive fused renders on a stream (synth_render,
 *    synth_render_batches, synth_render_normalized) may run partly at the
 *    same time: the next launch's CTAs start while the previous one's last
 *    wave finishes (programmatic dependent launch; the handle alternates two
 *    scratch slots). This is done only when neither launch writes a buffer
 *    the other reads or writes; otherwise, and between a render and any
 *    other kernel, copy or event, stream order holds as usual.
 */
#ifndef SYNTH_H
#define SYNTH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SYNTH_NUM_PARAMS 78

typedef enum {
  SYNTH_OK = 0,
  SYNTH_ERR_ARG = 1,         /* invalid argument; nothing was launched */
  SYNTH_ERR_CUDA = 2,        /* a CUDA runtime call failed */
  SYNTH_ERR_OOM = 3,         /* device or pinned allocation failed (create only) */
  SYNTH_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up (output invalid) */
  SYNTH_ERR_STATE = 5,       /* handle not usable (destroyed / earlier failure) */
  SYNTH_ERR_UNSUPPORTED = 6, /* configuration the kernels do not implement */
  SYNTH_ERR_BOUNDS = 7       /* bounds-checked build only: a kernel index left its
                                range; the access was skipped (output invalid) */
} synth_status;

typedef struct synth_handle_s* synth_handle;

/* Sec. 3.3 range-map hyper-parameters ("nebula"): for each of the 78
 * parameters the human range [lo, hi], a curve exponent c > 0 and a symmetric
 * flag. Non-symmetric: y = lo + (hi - lo) u^c. Symmetric: s = 2u - 1,
 * y = lo + (hi - lo) (1 + sgn(s)|s|^c) / 2. */
typedef struct {
  double lo[SYNTH_NUM_PARAMS];
  double hi[SYNTH_NUM_PARAMS];
  double curve[SYNTH_NUM_PARAMS];
  int32_t symmetric[SYNTH_NUM_PARAMS];
} synth_nebula;

/* Precision of the VCO phase running sums (precision study). */
#define SYNTH_CARRY_FIXED64 0 /* default: 64-bit fixed-point phases (2^-64 cycle
                                 resolution, exact sums mod 1, finer than FP64) */
#define SYNTH_CARRY_FP32 1    /* study only: interval phases summed and carried
                                 in FP32 */

typedef struct {
  double sample_rate;   /* Hz; Sec. 3.1 default 44100 */
  double control_rate;  /* Hz; Sec. 3.1 default 441. R = sample_rate/control_rate
                           in [4, 65532]: an integer, or a fraction of two
                           integer rates (e.g. 16000 / 441). Sample n then lies
                           in control interval k = floor(n CR / SR), at the
                           fraction n CR / SR - k between points k and k + 1.
                           The plain and adjoint renders and FP32 carries need
                           R an integer multiple of 4. */
  double seconds;       /* voice length; Abstract: 4 s */
  int32_t max_batch;    /* largest batch any call on this handle will use */
  int32_t carry;        /* SYNTH_CARRY_FIXED64 (default) or SYNTH_CARRY_FP32 */
  const synth_nebula* nebula; /* NULL = the library's default nebula n0;
                                 otherwise copied at create */
} synth_config;

/* Defaults: 44100 Hz, 441 Hz, 4 s, max_batch 128, fixed-point carry, nebula n0. */
void synth_default_config(synth_config* out);

/* The library's default nebula n0 (its own choice of ranges and curves; the
 * authors' nebula values are not given in the paper). */
void synth_default_nebula(synth_nebula* out);

/* Allocates the handle and its device scratch on the current CUDA device.
 * Errors: SYNTH_ERR_ARG (NULL pointers, rates or seconds <= 0, max_batch < 1,
 * an unknown carry), SYNTH_ERR_UNSUPPORTED (R outside [4, 65532], a
 * fractional R from rates that are not integers in Hz, seconds * sample_rate
 * not an integer or >= 2^31, FP32 carries with R not an integer multiple of
 * 4), SYNTH_ERR_OOM, SYNTH_ERR_CUDA. */
synth_status synth_create(const synth_config* cfg, synth_handle* out);
synth_status synth_destroy(synth_handle h);

int32_t synth_num_params(synth_handle h);   /* 78 (Sec. 1.1.3) */
int64_t synth_num_samples(synth_handle h);  /* N per voice */

/* Batched Voice render, fused form: one persistent kernel launch.
 * Sec. 3.1-3.3: per voice, parameters are drawn (Philox4x32-10, key = seed,
 * counter = (g, block, stream 0)) or taken from params_in_dev, mapped to
 * their ranges; 6 ADSRs, 2 LFOs and the modulation mixer run at the control
 * rate; control signals are linearly upsampled; a prefix scan over the
 * instantaneous frequency gives each VCO's phase; sine, square-saw and noise
 * (Philox, stream 1) pass through VCAs and the mixer.
 *  params_in_dev  [batch][78] float or NULL (NULL = draw from seed). Values
 *                 are clamped to [0,1].
 *  audio_dev      [batch][N] float, required.
 *  params_out_dev [batch][78] float or NULL: the normalized parameters used.
 * Errors: SYNTH_ERR_ARG (batch < 0 or > max_batch, NULL audio_dev),
 * SYNTH_ERR_CUDA. batch == 0 is a no-op. */
synth_status synth_render(synth_handle h, uint64_t seed, uint64_t batch_index, int32_t batch,
                          const float* params_in_dev, float* audio_dev, float* params_out_dev,
                          void* stream);

/* `count` consecutive batches in one persistent launch: batch k (k < count)
 * is synth_render(seed + k * seed_step, batch_index + k, batch) (its voices
 * g = (batch_index + k) * batch + v, the same voices and results), written
 * to audio_dev + k * batch * N and params_out_dev + k * batch * 78.
 * seed_step = 1 with seed = batch_index gives each batch the seed equal to
 * its index. One launch spreads the tiles of all batches over the GPU, so
 * the tail of one batch's tiles overlaps the next batch's.
 * Errors: as synth_render, with batch * count <= max_batch. */
synth_status synth_render_batches(synth_handle h, uint64_t seed, uint64_t seed_step,
                                  uint64_t batch_index, int32_t batch, int32_t count,
                                  const float* params_in_dev, float* audio_dev,
                                  float* params_out_dev, void* stream);

/* Render with per-voice peak normalisation and silence rejection. Sec. 2
 * names nearly silent renders among the undesirable products of sampling
 * parameters uniformly; this is the library's reading of a remedy, not a
 * step the paper specifies. The voices are rendered as by synth_render (same
 * seed, batch_index, params_in and params_out semantics) while the kernel
 * records each voice's peak p = max_n |x[n]|; then a voice with p >= threshold
 * and p > 0 is scaled by 1/p (its peak becomes 1; the factor is the correctly
 * rounded float reciprocal) and any other voice is left as rendered and
 * flagged silent. One kernel launch: the scaling runs as extra work items of
 * the render, so it overlaps the render's tail.
 *  threshold      float >= 0, in full-scale units (e.g. 1e-3 for -60 dBFS).
 *  peak_out_dev   [batch] float or NULL: p before scaling.
 *  silent_out_dev [batch] int32 or NULL: 1 if the voice was left as rendered.
 * Errors: as synth_render, plus SYNTH_ERR_ARG for a negative or NaN threshold.
 * A wait between work items that exceeds its spin limit leaves the affected
 * voices unscaled and flagged silent and makes the next synth_sync return
 * SYNTH_ERR_TIMEOUT. */
synth_status synth_render_normalized(synth_handle h, uint64_t seed, uint64_t batch_index,
                                    int32_t batch, const float* params_in_dev, float* audio_dev,
                                    float* params_out_dev, float threshold, float* peak_out_dev,
                                    int32_t* silent_out_dev, void* stream);

/* 4-operator FM voice. Sec. 3.2 names a 4-operator frequency-modulation
 * architecture as in development and specifies no more; this is the
 * library's own: four sine operators in a serial phase-modulation stack
 * op3 -> op2 -> op1 -> op0, out(n) = y_0(n), y_4 = 0,
 * y_i(n) = level_i E_i(n) sin(2 pi frac(n f0 ratio_i / SR) + y_(i+1)(n)),
 * E_i the Voice's ADSR at the control points, linearly upsampled.
 * SYNTH_FM_NUM_PARAMS normalized parameters per voice, u in [0, 1] mapped by
 * y = lo + (hi - lo) u^c: [0] midi f0 [0, 127]; [1] note-on duration [0, 4] s;
 * then for operator i (0 = carrier) at 2 + 7 i: ratio [0.5, 8] (c = 2), level
 * (carrier: amplitude [0, 1]; modulators: index [0, 8] rad, c = 2), attack
 * [0, 2] s (c = 2), decay [0, 2] s (c = 2), sustain [0, 1], release [0, 5] s
 * (c = 2), alpha [0.1, 6] (c = 2). Drawn parameters come from Philox4x32-10
 * stream 2 (counter (g lo, g hi, block, 2), key = seed).
 *  params_in_dev  [batch][30] float or NULL (NULL = draw); clamped to [0, 1].
 *  audio_dev      [batch][N] float, required; params_out_dev [batch][30] or NULL.
 * Any rates the handle accepts. Errors: SYNTH_ERR_ARG (batch < 0, > max_batch
 * or > 65535, NULL audio_dev), SYNTH_ERR_CUDA. */
#define SYNTH_FM_NUM_PARAMS 30
synth_status synth_fm_render(synth_handle h, uint64_t seed, uint64_t batch_index, int32_t batch,
                             const float* params_in_dev, float* audio_dev, float* params_out_dev,
                             void* stream);

/* The same render as a plain, unfused sequence of module kernels (one per
 * module, every control-rate and audio-rate intermediate in a caller-owned
 * workspace in device memory), the torchsynth-style design of Sec. 3.1.
 * Same results as synth_render to within floating-point reordering.
 * SYNTH_ERR_UNSUPPORTED unless R is an integer multiple of 4.
 * workspace_dev must hold synth_render_plain_workspace_size(h, batch) bytes
 * (256-byte aligned). Errors as synth_render, plus SYNTH_ERR_ARG when the
 * workspace is NULL or too small. */
synth_status synth_render_plain_workspace_size(synth_handle h, int32_t batch, size_t* bytes);
synth_status synth_render_plain(synth_handle h, uint64_t seed, uint64_t batch_index, int32_t batch,
                                const float* params_in_dev, float* audio_dev, float* params_out_dev,
                                void* workspace_dev, size_t workspace_bytes, void* stream);

/* Adjoint of synth_render (reverse mode): for every voice,
 * grad_params[v][p] = sum_n grad_audio[v][n] * d audio[v][n] / d u[v][p],
 * the derivative with respect to the normalized parameters u. The paper
 * lists differentiable modules as future work (Sec. 7); where the render
 * branches (envelope section, clamp, Nyquist cap, square LFO) this is the
 * derivative of the branch taken, and it is 0 at u = 0 for curve exponents
 * whose derivative is unbounded there.
 *  params_dev      [batch][78] float: the normalized parameters the forward
 *                  used (e.g. its params_out), required.
 *  seed, batch_index: as in the forward (they key the noise).
 *  grad_audio_dev  [batch][N] float; grad_params_dev [batch][78] float out.
 *  workspace_dev   synth_render_backward_workspace_size(h, batch) bytes,
 *                  256-byte aligned, caller-owned.
 * The forward control rate is recomputed from the parameters; its
 * per-interval phase descriptions are the checkpoints from which every
 * audio sample is rebuilt. Errors as synth_render_plain (R an integer
 * multiple of 4); SYNTH_ERR_UNSUPPORTED
 * when sample_rate/control_rate > 128. */
synth_status synth_render_backward_workspace_size(synth_handle h, int32_t batch, size_t* bytes);
synth_status synth_render_backward(synth_handle h, uint64_t seed, uint64_t batch_index,
                                   int32_t batch, const float* params_dev,
                                   const float* grad_audio_dev, float* grad_params_dev,
                                   void* workspace_dev, size_t workspace_bytes, void* stream);

/* The dense contraction under the STFT-as-GEMM and the proposal MLP, exposed
 * on its own: C[m][n] = alpha * sum_k A[m][k] B[n][k] with A, B bfloat16
 * (row-major, K contiguous, row strides lda, ldb in elements: multiples of 8,
 * >= k; 16-byte aligned bases), FP32 accumulation on the tcgen05 tensor
 * cores, C float32 row-major with row stride ldc >= n. k must be a multiple
 * of 8; m, n any positive size. Device pointers, caller-owned.
 * Errors: SYNTH_ERR_ARG, SYNTH_ERR_CUDA; a bounded wait that gave up is
 * reported by synth_sync as SYNTH_ERR_TIMEOUT. */
synth_status synth_gemm_bf16(synth_handle h, const void* a_dev, int32_t lda, const void* b_dev,
                             int32_t ldb, float* c_dev, int32_t ldc, int32_t m, int32_t n,
                             int32_t k, float alpha, void* stream);
/* The same product split along K when it has fewer 128-row output tiles than
 * the GPU has SMs (e.g. the proposal network's first layer, 128 x 1024 x
 * 44160): each SM takes a (tile, K-slice) pair and stores its FP32 partial
 * product in workspace_dev; a second kernel adds the slices in slice order
 * (deterministic) into C. workspace_dev: caller-owned device memory of at
 * least synth_gemm_bf16_workspace_size(h, m, n) bytes for the full split
 * (less splits less; NULL or 0 bytes: no split), 16-byte aligned.
 * Errors as synth_gemm_bf16. */
synth_status synth_gemm_bf16_workspace_size(synth_handle h, int32_t m, int32_t n, size_t* bytes);
synth_status synth_gemm_bf16_splitk(synth_handle h, const void* a_dev, int32_t lda,
                                    const void* b_dev, int32_t ldb, float* c_dev, int32_t ldc,
                                    int32_t m, int32_t n, int32_t k, float alpha,
                                    void* workspace_dev, size_t workspace_bytes, void* stream);

/* Multi-resolution log-magnitude STFT distance (the paper's multi-scale
 * spectrogram distance, Sec. 4, Table 2) between x and y, both [batch][N] float
 * device arrays of the handle's voice length (N >= 2048):
 *   L_v = sum over n_fft in {512, 1024, 2048} of the mean over (bins, frames)
 *         of |log(|X| + 1e-7) - log(|Y| + 1e-7)|,
 * periodic Hann window, hop n_fft/4, centred frames with reflect padding,
 * FP32 FFTs; the gradient through the inverse transforms and an overlap-add.
 *  loss_voice_dev [batch] double (device) or NULL: L_v per voice.
 *  grad_x_dev     [batch][N] float or NULL: d(sum_v L_v)/dx.
 *  target_ready   nonzero to reuse the target spectra an earlier call with the
 *                 same y and workspace left there.
 *  workspace      synth_mrstft_workspace_size(h, batch) bytes, 256-byte aligned.
 * Errors: SYNTH_ERR_ARG, SYNTH_ERR_UNSUPPORTED (N < 2048), SYNTH_ERR_CUDA. */
synth_status synth_mrstft_workspace_size(synth_handle h, int32_t batch, size_t* bytes);
synth_status synth_mrstft(synth_handle h, const float* x_dev, const float* y_dev, int32_t batch,
                          int32_t target_ready, double* loss_voice_dev, float* grad_x_dev,
                          void* workspace_dev, size_t workspace_bytes, void* stream);

/* Corpus similarity by maximum mean discrepancy (Sec. 5, the MMD equation):
 * MMD(X, Y) = 1/(n n) sum over i, j < n of [2 d(x_i, y_j) - d(x_i, x_j)
 * - d(y_i, y_j)], d an l1 distance between embeddings of the sounds (the
 * library's embedding: the network input features of synth_model_features,
 * 44160 bf16 values for a 4 s voice).
 *
 * synth_l1_distances: the pooled distance matrix dist_dev [m][m] FP32,
 * dist[i][j] = sum_k |e_i[k] - e_j[k]| over the rows of emb_dev [m][ld]
 * (bf16, row stride ld elements: a multiple of 8 and >= dim; 16-byte
 * aligned base), FP32 sums on the CUDA cores; symmetric, zero diagonal.
 * Errors: SYNTH_ERR_ARG (bad sizes or pointers), SYNTH_ERR_CUDA. */
synth_status synth_l1_distances(synth_handle h, const void* emb_dev, int64_t ld, int32_t m,
                                int32_t dim, float* dist_dev, void* stream);
/* synth_mmd_trials: one MMD per trial over a pooled distance matrix
 * dist_dev [m][m]. labels_dev [trials][m] int8: 0 puts sound j in X, 1 in Y,
 * any other value leaves it out. mmd_dev [trials] FP64 receives
 * 2 S_xy / (n_x n_y) - S_xx / n_x^2 - S_yy / n_y^2 (S_ab the sum of d over
 * ordered pairs, diagonal included; the paper's statistic when n_x = n_y),
 * or 0 when X or Y is empty. Sums in a fixed order: repeatable bit for bit.
 * Diversity within a corpus: X, Y a random 50/50 partition of it; between
 * corpora: n sounds drawn from each. m <= 49152.
 * Errors: SYNTH_ERR_ARG, SYNTH_ERR_CUDA. */
synth_status synth_mmd_trials(synth_handle h, const float* dist_dev, int32_t m,
                              const int8_t* labels_dev, int32_t trials, double* mmd_dev,
                              void* stream);

/* One Adam step (Kingma & Ba; beta 0.9 / 0.999, eps 1e-8, step >= 1) on
 * normalized parameters u[count] with gradient grad[count] and moments m, v
 * (device, caller-owned, zero before step 1); u is kept inside [0, 1]. Used
 * for adjoint refinement in parameter space. */
synth_status synth_param_adam(synth_handle h, float* u_dev, const float* grad_dev, float* m_dev,
                              float* v_dev, int32_t count, int32_t step, float lr, void* stream);

/* ---- learned parameter proposal (inverse synthesis, Sec. 2) ----------------
 * A network maps 128-band log-mel features (|STFT|^2, n_fft 2048, hop 512,
 * Slaney mel, log(x + 1e-6); frames = 1 + N/512) through a 4-layer MLP
 * (1024-1024-1024 ReLU, 78 sigmoid outputs) to normalized Voice parameters.
 * bf16 tensor-core GEMMs with FP32 accumulation; FP32 master weights, Adam.
 * The model owns its device memory (allocated at create) and is tied to the
 * handle it was created with (voice length, renderer for training). */
typedef struct synth_model_s* synth_model;

/* max_batch: a multiple of 8 and <= the handle's max_batch. Weights are drawn
 * from Philox(seed) uniform in +-1/sqrt(fan_in), biases 0. Synchronous.
 * Errors: SYNTH_ERR_ARG, SYNTH_ERR_UNSUPPORTED (voice shorter than 2048
 * samples), SYNTH_ERR_OOM, SYNTH_ERR_CUDA. */
synth_status synth_model_create(synth_handle h, int32_t max_batch, uint64_t seed, synth_model* out);
synth_status synth_model_destroy(synth_model m);
/* Feature length per voice: frames * 128. */
int64_t synth_model_feature_dim(synth_model m);
/* Network input features of audio [batch][N] -> features_dev
 * [batch][feature_dim] bf16: (log(mel + 1e-6) + 2.5) / 6 per band and frame
 * (frames major, bands minor); the fixed affine map keeps the inputs in about
 * [-2, 2]. */
synth_status synth_model_features(synth_model m, const float* audio_dev, int32_t batch,
                                  void* features_dev, void* stream);
/* Network forward on features -> params_out [batch][78] float in (0, 1). */
synth_status synth_model_forward(synth_model m, const void* features_dev, int32_t batch,
                                 float* params_out_dev, void* stream);
/* One training step on given features and target parameters [batch][78]:
 * forward, MSE (mean over batch x 78), backward, Adam(lr). batch: a multiple
 * of 8. loss_dev (device float) receives the loss before the update, or NULL. */
synth_status synth_model_train_features(synth_model m, const void* features_dev,
                                        const float* target_dev, int32_t batch, float lr,
                                        float* loss_dev, void* stream);
/* One training step on voices rendered on the fly: synth_render(seed,
 * batch_index, batch) into the model's buffers, features, train step. */
synth_status synth_model_train_step(synth_model m, uint64_t seed, uint64_t batch_index,
                                    int32_t batch, float lr, float* loss_dev, void* stream);
/* Streaming synth1B1 generator (Sec. 2.2): network input features and
 * normalized parameters of the voices g = synth_split_voice(split, first + i),
 * i < count, rendered (parameters drawn from seed) and transformed chunk by
 * chunk; a chunk's audio lives only in the model's own buffer, so no audio
 * of the range is materialised.
 *  split        0: every voice (g = first + i); 1: the train set; 2: the test set.
 *  chunk        voices per render + features step, 1..model max_batch;
 *               0 = the model's max_batch.
 *  features_dev [count][feature_dim] bf16, as synth_model_features.
 *  params_dev   [count][78] float or NULL.
 * Stream-ordered; the model's audio buffer is reused by every chunk, so calls
 * on one model must not overlap. Errors: SYNTH_ERR_ARG (split outside 0..2,
 * count < 0, chunk outside 0..max_batch, NULL features_dev with count > 0),
 * SYNTH_ERR_CUDA. count == 0 is a no-op. */
synth_status synth_stream_features(synth_model m, uint64_t seed, int32_t split, uint64_t first,
                                   int64_t count, int32_t chunk, void* features_dev,
                                   float* params_dev, void* stream);
/* Proposal: parameters_out [batch][78] for audio [batch][N] (features + forward). */
synth_status synth_propose(synth_handle h, synth_model m, const float* audio_dev, int32_t batch,
                           float* params_out_dev, void* stream);
/* Copies an FP32 tensor out of the model: which = 0 weights [out][in],
 * 1 biases [out], 2 last weight gradients, 3 last bias gradients (layer
 * 0..3); 4 the hidden activations H_layer (layer 1..3, the output of layer
 * layer - 1 after the ReLU, as the GEMMs read them: bf16 values widened to
 * FP32) of the last forward or training step, [batch][1024] for that call's
 * batch. count must equal the tensor's size. */
synth_status synth_model_get_tensor(synth_model m, int32_t which, int32_t layer, float* dst_dev,
                                    size_t count, void* stream);
/* Checkpoint: every model tensor (weights, Adam moments) and the step count
 * to / from a host file. Synchronous. */
synth_status synth_model_save(synth_model m, const char* path);
synth_status synth_model_load(synth_model m, const char* path);

/* The fused render without a handle and without any device allocation, for
 * callers that cannot call cudaMalloc (a plugin whose host application owns
 * all device memory, a process that reserved the whole GPU up front, or a
 * path where an allocation would synchronize the device). The paper has no
 * counterpart to this entry point.
 *  cfg: as for synth_create (max_batch is ignored); seed, batch_index,
 *  params_in_dev, audio_dev, params_out_dev, stream: as for synth_render,
 *  with the same results.
 * Scratch: a fixed 256 KiB device array inside the library, which every GPU
 * that loads the library holds until the process exits. It needs
 * 256 + 48 * batch * ceil(K / 255) bytes, K = floor((N - 1) / R) + 1 control
 * intervals (N = seconds * sample_rate, R = sample_rate / control_rate); for
 * 4 s at 44.1 kHz that allows batch
 * <= 779. Larger requests return SYNTH_ERR_ARG before any launch.
 * The first call on a device (with that device current) looks up the
 * array's device address; make that first call before any stream capture.
 * Calls outside capture look it up again (after cudaDeviceReset the array
 * may have moved); a call captured after a device reset, with no call in
 * between, would use the stale address. All calls share the one array and
 * each clears the part it uses: calls whose kernels overlap on the GPU
 * (other streams, other threads) race and must be serialized by the caller.
 * A device-side wait that gives up sets an error word in the array, which
 * synth_noalloc_status reads (the next call clears it).
 * Errors: SYNTH_ERR_ARG, SYNTH_ERR_UNSUPPORTED, SYNTH_ERR_CUDA. */
synth_status synth_render_noalloc(const synth_config* cfg, uint64_t seed, uint64_t batch_index,
                                  int32_t batch, const float* params_in_dev, float* audio_dev,
                                  float* params_out_dev, void* stream);
/* Status of the last synth_render_noalloc call on the current device: waits
 * for `stream`, then returns SYNTH_ERR_TIMEOUT (and clears the record) if a
 * bounded device-side wait of that render gave up (its audio is invalid),
 * SYNTH_ERR_BOUNDS (bounds-checked build) if an index left its range,
 * SYNTH_ERR_CUDA on a CUDA error, else SYNTH_OK. Allocates nothing; call it
 * after the render and before the next synth_render_noalloc. The paper has
 * no counterpart to this call either. */
synth_status synth_noalloc_status(void* stream);

/* Waits for the stream, then reports (and clears) a device-side error
 * recorded by any earlier call on this handle: SYNTH_ERR_BOUNDS if, in the
 * bounds-checked build, a kernel index left its range; else
 * SYNTH_ERR_TIMEOUT if a bounded wait gave up; SYNTH_ERR_CUDA on a CUDA
 * error; else SYNTH_OK. */
synth_status synth_sync(synth_handle h, void* stream);

/* Special-function-unit (MUFU) throughput probe, for the render's
 * transcendental roofline (the paper reports no roofline; this is the
 * library's own measurement aid). Launches `blocks` CTAs of 256 threads on
 * `stream`; every thread runs 8 independent chains of `iters` applications
 * of one approximate special function (sin, cos, ex2, rcp, lg2 or tanh, the
 * .approx PTX forms the render uses), so the unit's rate, not one chain's
 * latency, bounds the time. *ops_out (host, nullable) receives the number of
 * operations issued. sink_dev: a device buffer of at least 256 floats (only
 * written when a result could otherwise be optimised away). Time the call
 * with CUDA events; ops / time / SMs / SM clock = operations per clock per SM.
 * Errors: SYNTH_ERR_ARG, SYNTH_ERR_CUDA. */
#define SYNTH_SFU_SIN 0
#define SYNTH_SFU_COS 1
#define SYNTH_SFU_EX2 2
#define SYNTH_SFU_RCP 3
#define SYNTH_SFU_LG2 4
#define SYNTH_SFU_TANH 5
synth_status synth_sfu_probe(int32_t op, int32_t blocks, int32_t iters, float* sink_dev,
                             int64_t* ops_out, void* stream);

/* Failure-detection self-test (the library's own; the paper has no device
 * waits). Runs, on `stream`, one look-back wait of the fused render against
 * a window record that nothing ever publishes: the wait gives up after its
 * bounded spin (well under a second) and records a timeout in the handle,
 * exactly as a render whose earlier window never published would. Returns
 * after the stream is idle; the next synth_sync(h, stream) then returns
 * SYNTH_ERR_TIMEOUT and clears the record, and the handle stays usable.
 * Allocates and frees a 2-record device buffer. Errors: SYNTH_ERR_STATE
 * (invalid handle), SYNTH_ERR_CUDA. */
synth_status synth_selftest_wait_timeout(synth_handle h, void* stream);

/* The bounds-checked build (the library's own debugging aid; the paper has
 * none): the same sources compiled with -DSYNTH_CHECKS into
 * libsynth_checked.so, with the same calls and results. Its fused render
 * tests every index it derives -- audio and parameter offsets, the voice's
 * set-up and tile records, the tile's interval arrays in shared memory --
 * against the range it addresses, as do the adjoint's kernels; an index outside it is not used, and the
 * next synth_sync (synth_noalloc_status) returns SYNTH_ERR_BOUNDS. It takes
 * the place of a memory checker where none can run.
 * synth_checked_build: 1 in that library, 0 in the release build.
 * synth_selftest_bounds: runs, on `stream`, a kernel whose 32 threads each
 * derive an index past a 4-element array; the check refuses them, and the
 * next synth_sync(h, stream) returns SYNTH_ERR_BOUNDS and clears the record.
 * Returns after the stream is idle. Errors: SYNTH_ERR_STATE (invalid
 * handle), SYNTH_ERR_UNSUPPORTED (the release build, which launches
 * nothing), SYNTH_ERR_CUDA. */
int32_t synth_checked_build(void);
synth_status synth_selftest_bounds(synth_handle h, void* stream);

/* Host-side range map of normalized parameters (Sec. 3.3): y[count][78]
 * from u[count][78] under the handle's nebula. Host pointers. */
synth_status synth_params_to_human(synth_handle h, const float* u_host, double* y_host,
                                   int32_t count);

/* Sec. 2.2 train/test split: 1 if global voice g is in the test set
 * (blocks of 1024 voices, every tenth block), else 0. */
int32_t synth_is_test(uint64_t global_voice_index);
/* The global voice index g of the i-th voice of a split (0: every voice,
 * g = i; 1: train; 2: test): blocks of 1024 voices, nine train blocks then
 * one test block, repeating. */
uint64_t synth_split_voice(int32_t split, uint64_t i);

const char* synth_status_string(synth_status s);

#ifdef __cplusplus
}
#endif

#endif
