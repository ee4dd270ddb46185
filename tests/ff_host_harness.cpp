// Host build of the library's float-float header, for accuracy tests on CPU.
// Inputs and outputs are float pairs (hi, lo), so that a test knows the exact
// value each function was given.
#include "ff.cuh"
using namespace synth;
static FFTables g_tab;
static bool g_init = false;
static const FFTables& tab() {
  if (!g_init) {
    ff_tables_fill(g_tab);
    g_init = true;
  }
  return g_tab;
}
static void put(ff r, float* out) {
  out[0] = r.hi;
  out[1] = r.lo;
}
extern "C" {
void h_exp2(float hi, float lo, float* out) { put(ff_exp2({hi, lo}, tab()), out); }
void h_log2(float hi, float lo, float* out) { put(ff_log2({hi, lo}, tab()), out); }
void h_expm1(float hi, float lo, float* out) { put(ff_expm1({hi, lo}, tab()), out); }
void h_pow01(float xh, float xl, float ah, float al, float* out) {
  put(ff_pow01({xh, xl}, {ah, al}, tab()), out);
}
void h_sin2pi(float hi, float lo, float* out) { put(ff_sin2pi({hi, lo}, tab()), out); }
void h_div(float ah, float al, float bh, float bl, float* out) { put(ff_div({ah, al}, {bh, bl}), out); }
void h_rcp(float hi, float lo, float* out) { put(ff_rcp({hi, lo}), out); }
void h_mul(float ah, float al, float bh, float bl, float* out) { put(ff_mul({ah, al}, {bh, bl}), out); }
void h_add(float ah, float al, float bh, float bl, float* out) { put(ff_add({ah, al}, {bh, bl}), out); }
void h_frac(float hi, float lo, float* out) { put(ff_frac({hi, lo}), out); }
unsigned long long h_to_fix64(float hi, float lo) { return ff_to_fix64({hi, lo}); }
void h_fix64_to_ff(unsigned long long u, float* out) { put(fix64_to_ff(u), out); }
}
