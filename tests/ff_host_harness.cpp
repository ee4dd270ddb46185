// Host build of the library's float-float header, for accuracy tests on CPU.
#include "ff.cuh"
using namespace synth;
static FFTables g_tab;
static bool g_init = false;
static void init() {
  if (!g_init) { for (int i = 0; i < 33; ++i) ff_tables_fill_entry(g_tab, i); g_init = true; }
}
static ff mk(double x) { return ff_from_double(x); }
extern "C" {
double h_exp2(double y) { init(); return ff_to_double(ff_exp2(mk(y), g_tab)); }
double h_log2(double x) { init(); return ff_to_double(ff_log2(mk(x), g_tab)); }
double h_pow01(double x, double a) { init(); return ff_to_double(ff_pow01(mk(x), mk(a), g_tab)); }
double h_expm1(double x) { init(); return ff_to_double(ff_expm1(mk(x), g_tab)); }
double h_sin2pi(double p) { init(); return ff_to_double(ff_sin2pi(mk(p), g_tab)); }
double h_div(double a, double b) { return ff_to_double(ff_div(mk(a), mk(b))); }
double h_mul(double a, double b) { return ff_to_double(ff_mul(mk(a), mk(b))); }
double h_add(double a, double b) { return ff_to_double(ff_add(mk(a), mk(b))); }
double h_frac(double a) { return ff_to_double(ff_frac(mk(a))); }
}
