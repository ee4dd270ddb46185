// voice.cpp -- FP64 CPU oracle for the batched Voice render.
//
// TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
// cpu_baseline / reference leg may load this code. It is written for reading,
// not speed: per voice it walks every control point and every audio sample in
// order, in FP64, exactly as the definitions below state them. It shares no
// code with the CUDA library.
//
// Paper: Turian et al., "One Billion Audio Sounds from GPU-enabled Modular
// Synthesis", DAFx 2021.
//  * Sec. 3.1: audio modules at 44.1 kHz, control modules (ADSR, LFO) at
//    441 Hz, parameter modules (the monophonic keyboard: midi f0, duration).
//  * Sec. 3.2: the Voice = keyboard, 2 LFOs, 6 ADSRs (each LFO owns one ADSR
//    for its rate and one for its amplitude), sine VCO, square-saw VCO, noise,
//    VCAs, modulation mixer, audio mixer; control signals are upsampled to
//    audio rate before the audio modules. 78 parameters (Sec. 1.1.3).
//  * Sec. 3.3: parameters live in [0,1] and are mapped to [min,max] by a
//    curve and a symmetric flag; synth1B1 draws them uniformly (Sec. 2.1 adds
//    deterministic RNG, "even of noise oscillators").
// The paper prints no DSP formula. Every formula below is this project's
// reading of the module names above; each is stated in a comment at its code.
//
// Parity pins for these functions live in tests/test_oracle_*.py.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

#include "oracle.h"

namespace {

constexpr int NP = ORACLE_NUM_PARAMS;

// ---------------------------------------------------------------------------
// Dual numbers for the forward-mode derivative (value, one tangent).
// ---------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double x) : v(x), d(0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
inline Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
inline Dual operator-(Dual a) { return {-a.v, -a.d}; }
inline Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
inline Dual operator/(Dual a, Dual b) {
  return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)};
}
inline bool operator<(Dual a, Dual b) { return a.v < b.v; }
inline bool operator>(Dual a, Dual b) { return a.v > b.v; }
inline bool operator<=(Dual a, Dual b) { return a.v <= b.v; }
inline bool operator>=(Dual a, Dual b) { return a.v >= b.v; }

inline double val(double x) { return x; }
inline double val(Dual x) { return x.v; }

inline double t_sin(double x) { return std::sin(x); }
inline Dual t_sin(Dual x) { return {std::sin(x.v), std::cos(x.v) * x.d}; }
inline double t_cos(double x) { return std::cos(x); }
inline Dual t_cos(Dual x) { return {std::cos(x.v), -std::sin(x.v) * x.d}; }
inline double t_tanh(double x) { return std::tanh(x); }
inline Dual t_tanh(Dual x) {
  double t = std::tanh(x.v);
  return {t, (1.0 - t * t) * x.d};
}
inline double t_exp2(double x) { return std::exp2(x); }
inline Dual t_exp2(Dual x) {
  double e = std::exp2(x.v);
  return {e, e * std::log(2.0) * x.d};
}
inline double t_abs(double x) { return std::fabs(x); }
inline Dual t_abs(Dual x) { return x.v < 0 ? -x : x; }
// frac(x) = x - floor(x); the integer part carries no derivative.
inline double t_frac(double x) { return x - std::floor(x); }
inline Dual t_frac(Dual x) { return {x.v - std::floor(x.v), x.d}; }
// x^a for x >= 0. At x == 0 the value is 0 and the derivative is taken as 0.
inline double t_pow(double x, double a) { return x <= 0.0 ? 0.0 : std::pow(x, a); }
inline Dual t_pow(Dual x, Dual a) {
  if (x.v <= 0.0) return Dual(0.0);
  double p = std::pow(x.v, a.v);
  return {p, a.v * std::pow(x.v, a.v - 1.0) * x.d + p * std::log(x.v) * a.d};
}
template <class T> inline T t_min(T a, T b) { return b < a ? b : a; }
template <class T> inline T t_max(T a, T b) { return a < b ? b : a; }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11). Round: two 32x32->64 products of counter words 0 and 2
// with the multipliers, outputs permuted and xor-ed with the other counter
// words and the key; the key is bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

void philox(const uint32_t in[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = in[0], c1 = in[1], c2 = in[2], c3 = in[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t prod0 = (uint64_t)kPhiloxM0 * (uint64_t)c0;
    uint64_t prod1 = (uint64_t)kPhiloxM1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Random streams: counter word 3 separates parameter draws from noise.
constexpr uint32_t kStreamParam = 0;
constexpr uint32_t kStreamNoise = 1;

// A 32-bit draw -> uniform in [0,1): the top 24 bits times 2^-24 (exact).
inline double u01(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

// ---------------------------------------------------------------------------
// Parameter layout of the Voice (Sec. 3.2 module list; 78 params, Sec. 1.1.3).
// ---------------------------------------------------------------------------
enum : int {
  kMidi = 0, kDuration = 1,
  kAdsr = 2,   // 6 ADSRs x {attack, decay, sustain, release, alpha}
  kLfo = 32,   // 2 LFOs x {freq, rate_depth, phase0, w_sin, w_tri, w_saw, w_rsaw, w_sqr}
  kMod = 48,   // modulation mixer weight [source i][destination j] at kMod + 5 i + j
  kSine = 68,  // sine VCO {tune, depth, phase0}
  kSqr = 71,   // square-saw VCO {tune, depth, phase0, shape}
  kMix = 75,   // audio mixer levels {sine, square-saw, noise}
};
// ADSR roles: 0, 1 free modulation sources; 2 LFO0 rate, 3 LFO0 amplitude,
// 4 LFO1 rate, 5 LFO1 amplitude (Sec. 3.2: each LFO owns two ADSRs).
// Modulation sources: 0 ADSR0, 1 ADSR1, 2 LFO0, 3 LFO1.
// Destinations: 0 sine pitch, 1 sine amplitude, 2 square-saw pitch,
// 3 square-saw amplitude, 4 noise amplitude.

constexpr double kLfoMaxHz = 20.0;      // LFO rate bound (0..20 Hz)
constexpr double kBrightnessMax = 50.0; // square-saw waveshaper drive bound

void default_nebula(oracle_nebula* nb) {
  const double pi = 3.14159265358979323846;
  auto set = [&](int i, double lo, double hi, double c, int sym) {
    nb->lo[i] = lo; nb->hi[i] = hi; nb->curve[i] = c; nb->symmetric[i] = sym;
  };
  set(kMidi, 0.0, 127.0, 1.0, 0);      // Sec. 3.3 example: 0 <= midi f0 <= 127
  set(kDuration, 0.0, 4.0, 1.0, 0);    // note-on duration within the 4 s voice
  for (int a = 0; a < 6; ++a) {
    int b = kAdsr + 5 * a;
    set(b + 0, 0.0, 2.0, 2.0, 0);      // attack, s
    set(b + 1, 0.0, 2.0, 2.0, 0);      // decay, s
    set(b + 2, 0.0, 1.0, 1.0, 0);      // sustain level
    set(b + 3, 0.0, 5.0, 2.0, 0);      // release, s
    set(b + 4, 0.1, 6.0, 2.0, 0);      // alpha (segment curvature)
  }
  for (int l = 0; l < 2; ++l) {
    int b = kLfo + 8 * l;
    set(b + 0, 0.0, kLfoMaxHz, 2.0, 0);  // frequency, Hz
    set(b + 1, -20.0, 20.0, 3.0, 1);     // rate modulation depth, Hz
    set(b + 2, -pi, pi, 1.0, 1);         // initial phase, rad
    for (int s = 0; s < 5; ++s) set(b + 3 + s, 0.0, 1.0, 1.0, 0);  // shape weights
  }
  for (int i = 0; i < 20; ++i) set(kMod + i, 0.0, 1.0, 2.0, 0);
  set(kSine + 0, -24.0, 24.0, 1.0, 1);  // tune, semitones
  set(kSine + 1, -96.0, 96.0, 3.0, 1);  // pitch modulation depth, semitones
  set(kSine + 2, -pi, pi, 1.0, 1);      // initial phase, rad
  set(kSqr + 0, -24.0, 24.0, 1.0, 1);
  set(kSqr + 1, -96.0, 96.0, 3.0, 1);
  set(kSqr + 2, -pi, pi, 1.0, 1);
  set(kSqr + 3, 0.0, 1.0, 1.0, 0);      // square (0) .. saw-like (1)
  for (int i = 0; i < 3; ++i) set(kMix + i, 0.0, 1.0, 1.0, 0);
}

// Sec. 3.3 range map. Non-symmetric: y = lo + (hi - lo) u^c. Symmetric:
// s = 2u - 1, y = lo + (hi - lo) (1 + sgn(s) |s|^c) / 2, i.e. the curve is
// applied outward from the centre of the range. c = 1 is linear.
template <class T>
T range_map(T u, double lo, double hi, double c, int sym) {
  if (!sym) return T(lo) + T(hi - lo) * t_pow(u, T(c));
  T s = T(2.0) * u - T(1.0);
  T a = t_pow(t_abs(s), T(c));
  T signed_a = (s < T(0.0)) ? -a : a;
  return T(lo) + T(hi - lo) * (T(1.0) + signed_a) * T(0.5);
}

// Sec. 3.1 ADSR. Gate-on shape g(t): attack (t/a)^alpha for t < a; decay
// 1 - (1 - s)((t - a)/dc)^alpha for a <= t < a + dc; sustain s afterwards.
// At note-off d the release starts from L = g(d): L (1 - ((t - d)/r)^alpha)
// while t - d < r, then 0. All comparisons strict, so a zero-length section
// is skipped and the envelope is continuous at every section boundary.
template <class T>
T gate_on(T t, T a, T dc, T s, T alpha) {
  if (t < a) return t_pow(t / a, alpha);
  if (t < a + dc) return T(1.0) - (T(1.0) - s) * t_pow((t - a) / dc, alpha);
  return s;
}
template <class T>
T adsr(T t, T a, T dc, T s, T r, T alpha, T d) {
  if (t < d) return gate_on(t, a, dc, s, alpha);
  T level = gate_on(d, a, dc, s, alpha);
  T tau = t - d;
  if (tau < r) return level * (T(1.0) - t_pow(tau / r, alpha));
  return T(0.0);
}

// LFO shapes at phase p in [0,1): sine sin(2 pi p); triangle 1 - 4|p - 1/2|;
// saw 2p - 1; reverse saw 1 - 2p; square +1 for p < 1/2 else -1.
template <class T>
T lfo_shape(int shape, T p) {
  const double two_pi = 6.28318530717958647692;
  switch (shape) {
    case 0: return t_sin(T(two_pi) * p);
    case 1: return T(1.0) - T(4.0) * t_abs(p - T(0.5));
    case 2: return T(2.0) * p - T(1.0);
    case 3: return T(1.0) - T(2.0) * p;
    default: return (p < T(0.5)) ? T(1.0) : T(-1.0);
  }
}

template <class T>
T midi_to_hz(T m) { return T(440.0) * t_exp2((m - T(69.0)) / T(12.0)); }

// Samples per control interval R = SR / CR = A / B in lowest terms: an
// integer R (B = 1), or, for a fractional R, integer rates in Hz. Control
// point k sits at sample position k A / B; sample n lies in interval
// k = floor(n B / A) at the fraction u = (n B - k A) / A of the way from point
// k to point k + 1 (for an integer R: k = n div R, u = (n mod R) / R).
struct Geometry {
  int64_t N;   // samples per voice, round(seconds * SR)
  int64_t A;   // R = A / B
  int64_t B;
  int64_t K;   // control intervals holding samples, floor((N - 1) B / A) + 1; K + 1 points
};

bool geometry(const oracle_config* cfg, Geometry* g) {
  double sr = cfg->sample_rate, cr = cfg->control_rate;
  if (!(sr > 0) || !(cr > 0) || !(cfg->seconds > 0)) return false;
  double r = sr / cr;
  double n = cfg->seconds * sr;
  g->N = (int64_t)std::llround(n);
  if (std::fabs(n - (double)g->N) > 1e-6 || g->N < 1) return false;
  const int64_t ri = (int64_t)std::llround(r);
  if (ri >= 1 && std::fabs(r - (double)ri) <= 1e-9) {
    g->A = ri;
    g->B = 1;
  } else {
    const int64_t si = (int64_t)std::llround(sr), ci = (int64_t)std::llround(cr);
    if (std::fabs(sr - (double)si) > 1e-9 || std::fabs(cr - (double)ci) > 1e-9) return false;
    int64_t a = si, b = ci;
    while (b != 0) {
      const int64_t t = a % b;
      a = b;
      b = t;
    }
    g->A = si / a;
    g->B = ci / a;
    if (g->A < g->B) return false;  // at least one sample per control interval
  }
  g->K = (g->N - 1) * g->B / g->A + 1;
  return true;
}

// Control-rate signals of one voice (Sec. 3.1: control modules at the control
// rate; Sec. 3.2: each LFO's rate and amplitude ADSRs, modulation mixer).
// Control point k sits at t_k = k / CR, k = 0..K.
//  * env[a][k] = ADSR_a(t_k) with the keyboard's note-on duration d.
//  * LFO l: rate_k = clamp(freq + rate_depth * env[rate ADSR][k], 0, 20 Hz);
//    phase theta_0 = frac(phase0 / 2pi), theta_{k+1} = frac(theta_k + rate_k / CR)
//    (exclusive running sum); mix_k = sum_s w_s shape_s(theta_k) / sum_s w_s
//    (0 when the weights sum to < 1e-12); lfo_k = env[amp ADSR][k] * mix_k.
//  * dest_j[k] = sum_i W[i][j] src_i[k] / max(1, sum_i W[i][j]) with sources
//    (ADSR0, ADSR1, LFO0, LFO1).
template <class T>
struct Control {
  std::vector<T> env[6], lfo[2], dest[5];
};

template <class T>
void control_signals(const oracle_config* cfg, const Geometry& geo, const T* y, Control<T>* c,
                     bool round_f32) {
  const int64_t P = geo.K + 1;
  const double two_pi = 6.28318530717958647692;
  auto rnd = [&](T x) -> T {
    if (!round_f32) return x;
    T r = x;
    r = T((double)(float)val(x));
    return r;
  };
  T d = y[kDuration];
  for (int a = 0; a < 6; ++a) {
    c->env[a].resize(P);
    const T* q = y + kAdsr + 5 * a;
    for (int64_t k = 0; k < P; ++k) {
      T t = T((double)k / cfg->control_rate);
      c->env[a][k] = rnd(adsr(t, q[0], q[1], q[2], q[3], q[4], d));
    }
  }
  for (int l = 0; l < 2; ++l) {
    c->lfo[l].resize(P);
    const T* q = y + kLfo + 8 * l;
    const std::vector<T>& env_rate = c->env[2 + 2 * l];
    const std::vector<T>& env_amp = c->env[3 + 2 * l];
    T wsum = q[3] + q[4] + q[5] + q[6] + q[7];
    T theta = t_frac(q[2] / T(two_pi));
    for (int64_t k = 0; k < P; ++k) {
      T mix = T(0.0);
      if (val(wsum) >= 1e-12) {
        T acc = T(0.0);
        for (int s = 0; s < 5; ++s) acc = acc + q[3 + s] * lfo_shape(s, theta);
        mix = acc / wsum;
      }
      c->lfo[l][k] = rnd(env_amp[k] * mix);
      T rate = q[0] + q[1] * env_rate[k];
      rate = t_min(t_max(rate, T(0.0)), T(kLfoMaxHz));
      theta = t_frac(theta + rate / T(cfg->control_rate));
    }
  }
  for (int j = 0; j < 5; ++j) {
    c->dest[j].resize(P);
    T wsum = T(0.0);
    for (int i = 0; i < 4; ++i) wsum = wsum + y[kMod + 5 * i + j];
    T norm = t_max(T(1.0), wsum);
    for (int64_t k = 0; k < P; ++k) {
      T src[4] = {c->env[0][k], c->env[1][k], c->lfo[0][k], c->lfo[1][k]};
      T acc = T(0.0);
      for (int i = 0; i < 4; ++i) acc = acc + y[kMod + 5 * i + j] * src[i];
      c->dest[j][k] = rnd(acc / norm);
    }
  }
}

template <class T>
void map_params(const oracle_config* cfg, const T* u_in, T* y) {
  for (int p = 0; p < NP; ++p) {
    T u = u_in[p];
    if (u < T(0.0)) u = T(0.0);  // out-of-range inputs are clamped to [0,1]
    if (u > T(1.0)) u = T(1.0);
    y[p] = range_map(u, cfg->nebula.lo[p], cfg->nebula.hi[p], cfg->nebula.curve[p],
                     cfg->nebula.symmetric[p]);
  }
}

// One voice, every audio sample in order (Sec. 3.2 routing):
//  * upsampling: sample n in interval k at fraction u (see Geometry; for an
//    integer R, n = kR + j and u = j/R) takes c_k + u (c_{k+1} - c_k) of each
//    control signal (linear between the control points);
//  * VCO pitch in midi: m(n) = midi_f0 + tune + depth * pitch_dest(n), capped
//    at the Nyquist pitch 69 + 12 log2(SR/2/440); f = 440 * 2^((m - 69)/12);
//  * phase in cycles, exclusive running sum: phi(0) = frac(phase0 / 2pi),
//    phi(n+1) = frac(phi(n) + f(n)/SR);
//  * sine VCO: sin(2 pi phi);
//  * square-saw VCO: theta = 2 pi phi, sq = tanh(kappa sin theta)/tanh(kappa),
//    out = sq (1 + shape cos theta)/(1 + shape); kappa = min(50, 1 + SR/(8 f_k))
//    is held over control interval k, f_k the capped frequency at point k;
//  * noise: Philox4x32-10, key (seed lo, seed hi), counter (g lo, g hi, n/4,
//    1), word n mod 4, v = 2 u01 - 1;
//  * VCAs and mixer: out = (l0 A_sin x_sin + l1 A_sq x_sq + l2 A_noise v)
//    / max(1, l0 + l1 + l2), amplitudes from destinations 1, 3, 4.
template <class T>
int render_voice(const oracle_config* cfg, const T* u_in, uint64_t seed, uint64_t g, T* out,
                 int flags, int phase_vco, double* phase_out) {
  Geometry geo;
  if (!geometry(cfg, &geo)) return -1;
  const bool round_f32 = (flags & ORACLE_ROUND_PITCH_CHAIN_F32) != 0;
  const double two_pi = 6.28318530717958647692;
  const double sr = cfg->sample_rate;
  T y[NP];
  map_params(cfg, u_in, y);
  Control<T> ctl;
  control_signals(cfg, geo, y, &ctl, round_f32);

  const double m_nyq = 69.0 + 12.0 * std::log2(0.5 * sr / 440.0);
  const int64_t P = geo.K + 1;
  // Control-rate pitch (midi) of each VCO at each control point.
  std::vector<T> m_pt[2];
  const int vco_base[2] = {kSine, kSqr};
  const int vco_pitch_dest[2] = {0, 2};
  for (int v = 0; v < 2; ++v) {
    m_pt[v].resize(P);
    for (int64_t k = 0; k < P; ++k) {
      T m = y[kMidi] + y[vco_base[v]] + y[vco_base[v] + 1] * ctl.dest[vco_pitch_dest[v]][k];
      m_pt[v][k] = m;
    }
  }
  T level[3] = {y[kMix], y[kMix + 1], y[kMix + 2]};
  T mix_norm = t_max(T(1.0), level[0] + level[1] + level[2]);
  T shape = y[kSqr + 3];
  T phi[2] = {t_frac(y[kSine + 2] / T(two_pi)), t_frac(y[kSqr + 2] / T(two_pi))};
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t noise_words[4] = {0, 0, 0, 0};

  for (int64_t n = 0; n < geo.N; ++n) {
    const int64_t k = n * geo.B / geo.A;
    const double frac_j = (double)(n * geo.B - k * geo.A) / (double)geo.A;
    auto upsample = [&](const std::vector<T>& c) { return c[k] + T(frac_j) * (c[k + 1] - c[k]); };

    T f[2];
    for (int v = 0; v < 2; ++v) {
      T m = upsample(m_pt[v]);
      if (m > T(m_nyq)) m = T(m_nyq);
      f[v] = midi_to_hz(m);
      if (round_f32) f[v] = T((double)(float)val(f[v]));
    }
    if (phase_out && phase_vco >= 0) phase_out[n] = val(phi[phase_vco]);

    T x_sin = t_sin(T(two_pi) * phi[0]);
    T m_k = m_pt[1][k];
    if (m_k > T(m_nyq)) m_k = T(m_nyq);
    T f_k = midi_to_hz(m_k);
    T kappa = t_min(T(kBrightnessMax), T(1.0) + T(sr / 8.0) / f_k);
    T theta = T(two_pi) * phi[1];
    T sq = t_tanh(kappa * t_sin(theta)) / t_tanh(kappa);
    T x_sq = sq * (T(1.0) + shape * t_cos(theta)) / (T(1.0) + shape);

    if ((n & 3) == 0) {
      const uint32_t ctr[4] = {(uint32_t)g, (uint32_t)(g >> 32), (uint32_t)(n >> 2), kStreamNoise};
      philox(ctr, key, noise_words);
    }
    T x_noise = T(2.0 * u01(noise_words[n & 3]) - 1.0);

    T a_sin = upsample(ctl.dest[1]);
    T a_sq = upsample(ctl.dest[3]);
    T a_noise = upsample(ctl.dest[4]);
    out[n] = (level[0] * a_sin * x_sin + level[1] * a_sq * x_sq + level[2] * a_noise * x_noise) /
             mix_norm;

    for (int v = 0; v < 2; ++v) phi[v] = t_frac(phi[v] + f[v] / T(sr));
  }
  return 0;
}

template <class F>
void parallel_for(int64_t n, int threads, F fn) {
  if (threads <= 0) threads = (int)std::max(1u, std::thread::hardware_concurrency());
  if (threads == 1 || n <= 1) {
    for (int64_t i = 0; i < n; ++i) fn(i);
    return;
  }
  std::atomic<int64_t> next(0);
  std::vector<std::thread> pool;
  int nt = (int)std::min<int64_t>(threads, n);
  for (int t = 0; t < nt; ++t)
    pool.emplace_back([&]() {
      for (;;) {
        int64_t i = next.fetch_add(1);
        if (i >= n) break;
        fn(i);
      }
    });
  for (auto& th : pool) th.join();
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// 4-operator FM voice. Sec. 3.2 names a 4-operator frequency-modulation
// architecture (after Chowning 1973) as in development and gives nothing
// more; everything below is the library's reading:
//  * 30 parameters, normalized u in [0,1] mapped by y = lo + (hi - lo) u^c:
//    midi f0 [0, 127]; note-on duration [0, 4] s; then for operator i = 0..3
//    (0 the carrier) at 2 + 7 i: frequency ratio [0.5, 8] (c = 2); level,
//    the carrier's amplitude [0, 1] or a modulator's index in radians
//    [0, 8] (c = 2); the Voice's ADSR: attack [0, 2] s, decay [0, 2] s
//    (c = 2), sustain [0, 1], release [0, 5] s (c = 2), alpha [0.1, 6]
//    (c = 2), gated by the note-on duration.
//  * drawn from Philox4x32-10 stream 2: counter (g lo, g hi, block, 2), key
//    (seed lo, seed hi), 4 words per block, u = u01(word).
//  * envelopes E_i at the control points t_k = k / CR, upsampled linearly
//    as the Voice's control signals;
//  * operator phase phi_i(n) = frac(n f0 ratio_i / SR) (phase 0 at n = 0,
//    constant pitch);
//  * serial stack op 3 -> op 2 -> op 1 -> op 0 (phase modulation):
//    y_4 = 0, y_i(n) = level_i E_i(n) sin(2 pi phi_i(n) + y_(i+1)(n)),
//    out(n) = y_0(n).
// ---------------------------------------------------------------------------
constexpr int kFmNP = 30;
constexpr uint32_t kStreamFmParam = 2;

struct FmRange {
  double lo, hi, curve;
};

FmRange fm_range(int p) {
  if (p == 0) return {0.0, 127.0, 1.0};
  if (p == 1) return {0.0, 4.0, 1.0};
  const int i = (p - 2) / 7, q = (p - 2) % 7;
  switch (q) {
    case 0: return {0.5, 8.0, 2.0};
    case 1: return i == 0 ? FmRange{0.0, 1.0, 1.0} : FmRange{0.0, 8.0, 2.0};
    case 2: return {0.0, 2.0, 2.0};
    case 3: return {0.0, 2.0, 2.0};
    case 4: return {0.0, 1.0, 1.0};
    case 5: return {0.0, 5.0, 2.0};
    default: return {0.1, 6.0, 2.0};
  }
}

// frac(n x) with the product's rounding error carried (fma), so that the
// phase stays exact to ~1e-16 cycles at any n
double frac_prod(int64_t n, double x) {
  const double nd = (double)n;
  const double p = nd * x;
  const double e = std::fma(nd, x, -p);
  const double f = (p - std::floor(p)) + e;
  return f - std::floor(f);
}

int fm_render_voice(const oracle_config* cfg, const double* u_in, double* out) {
  Geometry geo;
  if (!geometry(cfg, &geo)) return -1;
  const double two_pi = 6.28318530717958647692;
  double y[kFmNP];
  for (int p = 0; p < kFmNP; ++p) {
    double u = u_in[p];
    if (u < 0.0) u = 0.0;
    if (u > 1.0) u = 1.0;
    const FmRange r = fm_range(p);
    y[p] = range_map<double>(u, r.lo, r.hi, r.curve, 0);
  }
  const double f0 = midi_to_hz<double>(y[0]), d = y[1];
  const int64_t P = geo.K + 1;
  std::vector<double> env[4];
  double inc[4], level[4];
  for (int i = 0; i < 4; ++i) {
    const double* o = y + 2 + 7 * i;
    inc[i] = f0 * o[0] / cfg->sample_rate;
    level[i] = o[1];
    env[i].resize(P);
    for (int64_t k = 0; k < P; ++k)
      env[i][k] = adsr<double>((double)k / cfg->control_rate, o[2], o[3], o[4], o[5], o[6], d);
  }
  for (int64_t n = 0; n < geo.N; ++n) {
    const int64_t k = n * geo.B / geo.A;
    const double u = (double)(n * geo.B - k * geo.A) / (double)geo.A;
    double yv = 0.0;
    for (int i = 3; i >= 0; --i) {
      const double e = env[i][k] + u * (env[i][k + 1] - env[i][k]);
      yv = level[i] * e * std::sin(two_pi * frac_prod(n, inc[i]) + yv);
    }
    out[n] = yv;
  }
  return 0;
}

}  // namespace

extern "C" {

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  philox(ctr, key, out);
}

void oracle_default_nebula(oracle_nebula* out) { default_nebula(out); }

void oracle_default_config(oracle_config* out) {
  out->sample_rate = 44100.0;
  out->control_rate = 441.0;
  out->seconds = 4.0;
  default_nebula(&out->nebula);
}

// Parameter p of voice g is word p mod 4 of the Philox block with counter
// (g lo, g hi, p / 4, 0) under key (seed lo, seed hi): 20 blocks, 80 words,
// the first 78 used.
void oracle_draw_params(uint64_t seed, uint64_t g, double u[ORACLE_NUM_PARAMS]) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int b = 0; b < 20; ++b) {
    const uint32_t ctr[4] = {(uint32_t)g, (uint32_t)(g >> 32), (uint32_t)b, kStreamParam};
    uint32_t w[4];
    philox(ctr, key, w);
    for (int l = 0; l < 4; ++l) {
      int p = 4 * b + l;
      if (p < NP) u[p] = u01(w[l]);
    }
  }
}

double oracle_range_map(double u, double lo, double hi, double curve, int32_t symmetric) {
  return range_map<double>(u, lo, hi, curve, symmetric);
}

double oracle_adsr(double t, double attack, double decay, double sustain, double release,
                   double alpha, double d) {
  return adsr<double>(t, attack, decay, sustain, release, alpha, d);
}

double oracle_lfo_shape(int32_t shape, double p) { return lfo_shape<double>(shape, p); }

double oracle_midi_to_hz(double m) { return midi_to_hz<double>(m); }

int32_t oracle_control(const oracle_config* cfg, const double u[ORACLE_NUM_PARAMS], double* env,
                       double* lfo, double* dest) {
  Geometry geo;
  if (!geometry(cfg, &geo)) return -1;
  double y[NP];
  map_params<double>(cfg, u, y);
  Control<double> c;
  control_signals<double>(cfg, geo, y, &c, false);
  const int64_t P = geo.K + 1;
  for (int a = 0; a < 6 && env; ++a) std::memcpy(env + a * P, c.env[a].data(), P * sizeof(double));
  for (int l = 0; l < 2 && lfo; ++l) std::memcpy(lfo + l * P, c.lfo[l].data(), P * sizeof(double));
  for (int j = 0; j < 5 && dest; ++j) std::memcpy(dest + j * P, c.dest[j].data(), P * sizeof(double));
  return 0;
}

// LFO phases theta_k (cycles, wrapped) at the control points, the running sum
// the control signals use: theta[2][K+1].
int32_t oracle_lfo_phase(const oracle_config* cfg, const double u[ORACLE_NUM_PARAMS],
                         double* theta) {
  Geometry geo;
  if (!geometry(cfg, &geo)) return -1;
  double y[NP];
  map_params<double>(cfg, u, y);
  Control<double> c;
  control_signals<double>(cfg, geo, y, &c, false);
  const int64_t P = geo.K + 1;
  const double two_pi = 6.28318530717958647692;
  for (int l = 0; l < 2; ++l) {
    const double* q = y + kLfo + 8 * l;
    double th = t_frac(q[2] / two_pi);
    for (int64_t k = 0; k < P; ++k) {
      theta[l * P + k] = th;
      double rate = q[0] + q[1] * c.env[2 + 2 * l][k];
      rate = t_min(t_max(rate, 0.0), kLfoMaxHz);
      th = t_frac(th + rate / cfg->control_rate);
    }
  }
  return 0;
}

int32_t oracle_render_voice(const oracle_config* cfg, const double u[ORACLE_NUM_PARAMS],
                            uint64_t seed, uint64_t g, double* out) {
  return render_voice<double>(cfg, u, seed, g, out, 0, -1, nullptr);
}

int32_t oracle_render_voice_ex(const oracle_config* cfg, const double u[ORACLE_NUM_PARAMS],
                               uint64_t seed, uint64_t g, double* out, int32_t flags) {
  return render_voice<double>(cfg, u, seed, g, out, flags, -1, nullptr);
}

int32_t oracle_vco_phase(const oracle_config* cfg, const double u[ORACLE_NUM_PARAMS],
                         int32_t vco, double* phase) {
  Geometry geo;
  if (!geometry(cfg, &geo) || vco < 0 || vco > 1) return -1;
  std::vector<double> tmp(geo.N);
  return render_voice<double>(cfg, u, 0, 0, tmp.data(), 0, vco, phase);
}

int32_t oracle_render_batch(const oracle_config* cfg, uint64_t seed, uint64_t batch_index,
                            int32_t batch, const double* u_in, float* audio, float* params_out,
                            int32_t threads, const int32_t* voices, int32_t n_voices) {
  Geometry geo;
  if (!geometry(cfg, &geo) || batch < 0) return -1;
  std::vector<int32_t> slots;
  if (voices && n_voices > 0) {
    slots.assign(voices, voices + n_voices);
  } else {
    for (int32_t v = 0; v < batch; ++v) slots.push_back(v);
  }
  std::atomic<int> failed(0);
  parallel_for((int64_t)slots.size(), threads, [&](int64_t i) {
    const int32_t v = slots[i];
    if (v < 0 || v >= batch) { failed = 1; return; }
    const uint64_t g = batch_index * (uint64_t)batch + (uint64_t)v;
    double u[NP];
    if (u_in) std::memcpy(u, u_in + (int64_t)v * NP, sizeof(u));
    else oracle_draw_params(seed, g, u);
    if (params_out)
      for (int p = 0; p < NP; ++p) params_out[(int64_t)v * NP + p] = (float)u[p];
    std::vector<double> buf(geo.N);
    if (render_voice<double>(cfg, u, seed, g, buf.data(), 0, -1, nullptr) != 0) { failed = 1; return; }
    if (audio) {
      float* dst = audio + (int64_t)v * geo.N;
      for (int64_t n = 0; n < geo.N; ++n) dst[n] = (float)buf[n];
    }
  });
  return failed ? -1 : 0;
}

int32_t oracle_render_vjp(const oracle_config* cfg, const double u[ORACLE_NUM_PARAMS],
                          uint64_t seed, uint64_t g, const double* w, double grad[ORACLE_NUM_PARAMS],
                          int32_t threads) {
  Geometry geo;
  if (!geometry(cfg, &geo)) return -1;
  std::atomic<int> failed(0);
  parallel_for(NP, threads, [&](int64_t p) {
    Dual ud[NP];
    for (int i = 0; i < NP; ++i) ud[i] = Dual(u[i], i == p ? 1.0 : 0.0);
    std::vector<Dual> out(geo.N);
    if (render_voice<Dual>(cfg, ud, seed, g, out.data(), 0, -1, nullptr) != 0) { failed = 1; return; }
    double acc = 0.0;
    for (int64_t n = 0; n < geo.N; ++n) acc += w[n] * out[n].d;
    grad[p] = acc;
  });
  return failed ? -1 : 0;
}

void oracle_fm_draw_params(uint64_t seed, uint64_t g, double u[ORACLE_FM_NUM_PARAMS]) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int b = 0; 4 * b < kFmNP; ++b) {
    const uint32_t ctr[4] = {(uint32_t)g, (uint32_t)(g >> 32), (uint32_t)b, kStreamFmParam};
    uint32_t w[4];
    philox(ctr, key, w);
    for (int l = 0; l < 4; ++l)
      if (4 * b + l < kFmNP) u[4 * b + l] = u01(w[l]);
  }
}

int32_t oracle_fm_render_voice(const oracle_config* cfg, const double u[ORACLE_FM_NUM_PARAMS],
                               double* out) {
  return fm_render_voice(cfg, u, out);
}

int32_t oracle_fm_render_batch(const oracle_config* cfg, uint64_t seed, uint64_t batch_index,
                               int32_t batch, const double* u_in, float* audio, float* params_out,
                               int32_t threads) {
  Geometry geo;
  if (!geometry(cfg, &geo) || batch < 0) return -1;
  std::atomic<int> failed(0);
  parallel_for(batch, threads, [&](int64_t v) {
    const uint64_t g = batch_index * (uint64_t)batch + (uint64_t)v;
    double u[kFmNP];
    if (u_in) std::memcpy(u, u_in + v * kFmNP, sizeof(u));
    else oracle_fm_draw_params(seed, g, u);
    if (params_out)
      for (int p = 0; p < kFmNP; ++p) params_out[v * kFmNP + p] = (float)u[p];
    std::vector<double> buf(geo.N);
    if (fm_render_voice(cfg, u, buf.data()) != 0) { failed = 1; return; }
    if (audio)
      for (int64_t n = 0; n < geo.N; ++n) audio[v * geo.N + n] = (float)buf[n];
  });
  return failed ? -1 : 0;
}

int32_t oracle_hardware_threads(void) {
  return (int32_t)std::max(1u, std::thread::hardware_concurrency());
}

}  // extern "C"
