// Host build of the render's split noise generator (philox_noise.cuh), for a
// CPU check that it equals the plain Philox4x32-10 rounds bit for bit.
#include "philox_noise.cuh"
using namespace synth;
extern "C" {
// out[4 * i .. 4 * i + 3] = block q[i] of counter (c0, c1, q[i], c3), key (k0, k1)
void h_philox_noise(uint32_t c0, uint32_t c1, uint32_t c3, uint32_t k0, uint32_t k1,
                    const uint32_t* q, int n, uint32_t* out) {
  const PhiloxNoise p = philox_noise_setup(c0, c1, c3, k0, k1);
  for (int i = 0; i < n; ++i) philox_noise(p, q[i], out + 4 * i);
}
}
