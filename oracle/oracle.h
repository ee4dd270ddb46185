/*
 * oracle.h -- C declarations of the FP64 CPU oracle for the batched Voice render.
 *
 * TEST INFRASTRUCTURE. This is the slow, plain reference the CUDA library is
 * checked against. Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg may load it. It shares no code, header, table
 * or constant with the CUDA library (paper_2104_12922_gb300/csrc), and the
 * CUDA library never includes or links it.
 *
 * Paper: Turian et al., "One Billion Audio Sounds from GPU-enabled Modular
 * Synthesis" (DAFx 2021). The paper names the Voice's modules (Sec. 3.1,
 * 3.2) and the parameter mapping (Sec. 3.3) but prints no DSP formula; each
 * formula here is a reading of those sections, stated next to its code in
 * voice.cpp.
 */
#ifndef SYNTH_ORACLE_H
#define SYNTH_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORACLE_NUM_PARAMS 78
#define ORACLE_FM_NUM_PARAMS 30

/* Range-map hyper-parameters of one nebula (Sec. 3.3): per parameter the
 * human range [lo, hi], the curve exponent and the symmetric flag. */
typedef struct {
  double lo[ORACLE_NUM_PARAMS];
  double hi[ORACLE_NUM_PARAMS];
  double curve[ORACLE_NUM_PARAMS];
  int32_t symmetric[ORACLE_NUM_PARAMS];
} oracle_nebula;

typedef struct {
  double sample_rate;   /* audio rate, Hz (Sec. 3.1 default 44100) */
  double control_rate;  /* control rate, Hz (Sec. 3.1 default 441) */
  double seconds;       /* voice length (Abstract: 4 s) */
  oracle_nebula nebula; /* range map used for every parameter */
} oracle_config;

/* Flags for oracle_render_voice_ex. */
#define ORACLE_ROUND_PITCH_CHAIN_F32 1 /* study only: round control-rate pitch chain to FP32 */

/* Philox4x32-10 (Salmon et al., SC'11): one block of 4 words. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* The default nebula n0 of this project (the authors' own values are not in
 * the paper). */
void oracle_default_nebula(oracle_nebula* out);
void oracle_default_config(oracle_config* out);

/* Normalized parameter draw for global voice index g (Sec. 2.1: deterministic
 * RNG; Sec. 3.3: uniform in [0,1)). u[78] receives exact multiples of 2^-24. */
void oracle_draw_params(uint64_t seed, uint64_t g, double u[ORACLE_NUM_PARAMS]);

/* Sec. 3.3 range map of one normalized value. */
double oracle_range_map(double u, double lo, double hi, double curve, int32_t symmetric);

/* Sec. 3.1 ADSR envelope value at time t (seconds) for note-on duration d. */
double oracle_adsr(double t, double attack, double decay, double sustain,
                   double release, double alpha, double d);

/* LFO shape value (0 sin, 1 tri, 2 saw, 3 rsaw, 4 sqr) at phase p in [0,1). */
double oracle_lfo_shape(int32_t shape, double p);

/* midi -> Hz (equal temperament, A4 = midi 69 = 440 Hz). */
double oracle_midi_to_hz(double m);

/* Control-rate signals of one voice, K+1 points each (k = 0..K, t_k = k/CR):
 * env[6][K+1], lfo[2][K+1], dest[5][K+1]. Any pointer may be NULL. */
int32_t oracle_control(const oracle_config* cfg, const double u[ORACLE_NUM_PARAMS],
                       double* env, double* lfo, double* dest);

/* LFO phases (cycles in [0,1)) at the control points: theta[2][K+1]. */
int32_t oracle_lfo_phase(const oracle_config* cfg, const double u[ORACLE_NUM_PARAMS],
                         double* theta);

/* One voice, FP64 throughout: out[N] with N = seconds * sample_rate.
 * u are normalized parameters (clamped to [0,1]); seed and g key the noise.
 * Returns 0, or -1 when the configuration is not representable. */
int32_t oracle_render_voice(const oracle_config* cfg, const double u[ORACLE_NUM_PARAMS],
                            uint64_t seed, uint64_t g, double* out);
int32_t oracle_render_voice_ex(const oracle_config* cfg, const double u[ORACLE_NUM_PARAMS],
                               uint64_t seed, uint64_t g, double* out, int32_t flags);

/* Per-voice sine-VCO phase (cycles, wrapped to [0,1)) of the same render, for
 * phase-drift reports. phase[N]. vco = 0 sine, 1 square-saw. */
int32_t oracle_vco_phase(const oracle_config* cfg, const double u[ORACLE_NUM_PARAMS],
                         int32_t vco, double* phase);

/* Batch render: voice v of the batch has global index g = batch_index*batch + v.
 * If u_in is NULL the parameters are drawn with oracle_draw_params; otherwise
 * u_in[batch][78] is used. audio[batch][N] (float, rounded from FP64),
 * params_out[batch][78] may be NULL. threads <= 0 uses all hardware threads.
 * voices[] (length n_voices) optionally restricts the work to a subset of
 * voice slots; pass NULL / 0 for all. */
int32_t oracle_render_batch(const oracle_config* cfg, uint64_t seed, uint64_t batch_index,
                            int32_t batch, const double* u_in, float* audio, float* params_out,
                            int32_t threads, const int32_t* voices, int32_t n_voices);

/* Jacobian-vector product by forward-mode dual numbers: grad[78] =
 * sum_n w[n] * d out[n] / d u[p] for one voice (one dual pass per parameter).
 * Where the render has a branch, the derivative of the branch taken. */
int32_t oracle_render_vjp(const oracle_config* cfg, const double u[ORACLE_NUM_PARAMS],
                          uint64_t seed, uint64_t g, const double* w, double grad[ORACLE_NUM_PARAMS],
                          int32_t threads);

int32_t oracle_hardware_threads(void);

/* 4-operator FM voice (the library's reading of the FM architecture that
 * Sec. 3.2 names as in development; the formulas are in voice.cpp):
 * 30 normalized parameters, drawn from Philox stream 2; serial phase
 * modulation op3 -> op2 -> op1 -> op0, each operator a sine at f0 x ratio
 * with its own ADSR. cfg: rates and length (its nebula is not used). */
void oracle_fm_draw_params(uint64_t seed, uint64_t g, double u[ORACLE_FM_NUM_PARAMS]);
int32_t oracle_fm_render_voice(const oracle_config* cfg, const double u[ORACLE_FM_NUM_PARAMS],
                               double* out);
int32_t oracle_fm_render_batch(const oracle_config* cfg, uint64_t seed, uint64_t batch_index,
                               int32_t batch, const double* u_in, float* audio, float* params_out,
                               int32_t threads);

#ifdef __cplusplus
}
#endif

#endif
