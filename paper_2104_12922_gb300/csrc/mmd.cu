// mmd.cu -- corpus similarity by maximum mean discrepancy (Sec. 5 of the
// paper, the MMD equation): MMD(X, Y) = 1/(n n) sum over i, j of
// [2 d(x_i, y_j) - d(x_i, x_j) - d(y_i, y_j)], with d an l1 distance between
// embeddings of the sounds. The library's embedding is its log-mel feature
// vector (345 frames x 128 bands = 44160 bf16 values for a 4 s voice).
//
// Two kernels:
//  * l1_distance_kernel: the pooled pairwise distance matrix of m embeddings,
//    d[i][j] = sum_k |e_i[k] - e_j[k]| in FP32 on the CUDA cores. It is not a
//    contraction (no products), so there is no tensor-core form: the bound is
//    the FP32 pipe, two instructions (a subtraction and an addition of the
//    absolute value) per element pair. A CTA of 256 threads computes a
//    128 x 128 tile of the upper triangle; embedding chunks of 32 values are
//    staged in shared memory as FP32 (k-major, so each thread reads its 8
//    rows and 8 columns as float4 pairs), and each thread keeps an 8 x 8 block
//    of distances in registers. Off-diagonal tiles also write their mirror
//    image, so the whole matrix is filled.
//  * mmd_trials_kernel: one CTA per trial; a trial labels each pooled sound
//    0 (in X), 1 (in Y) or neither. Each warp walks rows of the distance
//    matrix that belong to X or Y and sums them by the column's label (FP32
//    within a row, FP64 across rows); the block adds its warps' sums in warp
//    order (deterministic) and forms
//    2 S_xy / (n_x n_y) - S_xx / n_x^2 - S_yy / n_y^2.

#include <cuda_bf16.h>

#include <cstdint>

#include "internal.h"

namespace synth {

namespace {

constexpr int kDT = 128;    // distance tile (rows and columns)
constexpr int kDK = 32;     // embedding values per shared-memory chunk
constexpr int kDThreads = 256;

__global__ void __launch_bounds__(kDThreads, 2)
    l1_distance_kernel(const __nv_bfloat16* __restrict__ emb, int64_t ld, int m, int dim,
                       float* __restrict__ dist) {
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bi > bj) return;  // upper triangle of tiles; mirrored below
  __shared__ __align__(16) float As[kDK][kDT];
  __shared__ __align__(16) float Bs[kDK][kDT];
  const int tid = threadIdx.x;
  // this thread's 8 rows are ty*4 + {0..3} and 64 + ty*4 + {0..3} of the tile,
  // its 8 columns likewise from tx: a quarter-warp's float4 reads then cover
  // 32 distinct banks
  const int tx = tid & 15, ty = tid >> 4;
  const int r0 = bi * kDT, c0 = bj * kDT;
  float acc[8][8];
#pragma unroll
  for (int p = 0; p < 8; ++p)
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[p][q] = 0.f;

  for (int k0 = 0; k0 < dim; k0 += kDK) {
    // stage 128 rows x 32 values of each side, 4 values (8 bytes) per load;
    // consecutive threads take consecutive rows, so the transposing stores
    // into shared memory hit 32 distinct banks
    __syncthreads();
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int e = tid + l * kDThreads;  // 0 .. 1023
      const int row = e & (kDT - 1), col = (e >> 7) * 4;
      float va[4] = {0.f, 0.f, 0.f, 0.f}, vb[4] = {0.f, 0.f, 0.f, 0.f};
      const int ra = r0 + row, rb = c0 + row, k = k0 + col;
      if (k + 3 < dim) {
        if (ra < m) {
          const uint2 w = *reinterpret_cast<const uint2*>(emb + ra * ld + k);
          const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&w.x);
          const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&w.y);
          va[0] = __low2float(lo); va[1] = __high2float(lo);
          va[2] = __low2float(hi); va[3] = __high2float(hi);
        }
        if (rb < m) {
          const uint2 w = *reinterpret_cast<const uint2*>(emb + rb * ld + k);
          const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&w.x);
          const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&w.y);
          vb[0] = __low2float(lo); vb[1] = __high2float(lo);
          vb[2] = __low2float(hi); vb[3] = __high2float(hi);
        }
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (k + u < dim) {
            if (ra < m) va[u] = __bfloat162float(emb[ra * ld + k + u]);
            if (rb < m) vb[u] = __bfloat162float(emb[rb * ld + k + u]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        As[col + u][row] = va[u];  // past the end of the rows or of dim: 0 on both sides
        Bs[col + u][row] = vb[u];
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int c = 0; c < kDK; ++c) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[c][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[c][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[c][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[c][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int p = 0; p < 8; ++p)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[p][q] += fabsf(a[p] - b[q]);
    }
  }
  // d[i][j] for this tile's pairs and, off the diagonal, the mirror d[j][i]
  int ri[8], cj[8];
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    ri[p] = r0 + (p < 4 ? ty * 4 + p : 64 + ty * 4 + p - 4);
    cj[p] = c0 + (p < 4 ? tx * 4 + p : 64 + tx * 4 + p - 4);
  }
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    if (ri[p] >= m) continue;
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (cj[q] < m) dist[(int64_t)ri[p] * m + cj[q]] = acc[p][q];
  }
  if (bi == bj) return;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    if (cj[q] >= m) continue;
#pragma unroll
    for (int p = 0; p < 8; ++p)
      if (ri[p] < m) dist[(int64_t)cj[q] * m + ri[p]] = acc[p][q];
  }
}

constexpr int kMThreads = 256;
constexpr int kMWarps = kMThreads / 32;

__global__ void __launch_bounds__(kMThreads)
    mmd_trials_kernel(const float* __restrict__ dist, int m, const int8_t* __restrict__ labels,
                      double* __restrict__ mmd_out) {
  extern __shared__ int8_t lab[];  // this trial's labels, m bytes
  __shared__ double red[kMWarps][4];
  __shared__ int count[2];
  const int t = blockIdx.x;
  const int8_t* lt = labels + (int64_t)t * m;
  if (threadIdx.x < 2) count[threadIdx.x] = 0;
  __syncthreads();
  int nx = 0, ny = 0;
  for (int j = threadIdx.x; j < m; j += kMThreads) {
    const int8_t l = lt[j];
    lab[j] = l;
    nx += l == 0;
    ny += l == 1;
  }
  for (int o = 16; o > 0; o >>= 1) {
    nx += __shfl_xor_sync(0xffffffffu, nx, o);
    ny += __shfl_xor_sync(0xffffffffu, ny, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&count[0], nx);  // integer counts: exact in any order
    atomicAdd(&count[1], ny);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // s[a][b]: sum of d(i, j) over rows i with label a and columns j with label b
  double s[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int i = warp; i < m; i += kMWarps) {
    const int li = lab[i];
    if (li != 0 && li != 1) continue;
    const float* row = dist + (int64_t)i * m;
    float r0 = 0.f, r1 = 0.f;
    for (int j = lane; j < m; j += 32) {
      const int lj = lab[j];
      const float d = row[j];
      r0 += lj == 0 ? d : 0.f;
      r1 += lj == 1 ? d : 0.f;
    }
    for (int o = 16; o > 0; o >>= 1) {
      r0 += __shfl_xor_sync(0xffffffffu, r0, o);
      r1 += __shfl_xor_sync(0xffffffffu, r1, o);
    }
    s[li][0] += (double)r0;
    s[li][1] += (double)r1;
  }
  if (lane == 0) {
    red[warp][0] = s[0][0];
    red[warp][1] = s[0][1];
    red[warp][2] = s[1][0];
    red[warp][3] = s[1][1];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sxx = 0.0, sxy = 0.0, syx = 0.0, syy = 0.0;
    for (int w = 0; w < kMWarps; ++w) {
      sxx += red[w][0];
      sxy += red[w][1];
      syx += red[w][2];
      syy += red[w][3];
    }
    const double fx = (double)count[0], fy = (double)count[1];
    mmd_out[t] = (count[0] > 0 && count[1] > 0)
                     ? (sxy + syx) / (fx * fy) - sxx / (fx * fx) - syy / (fy * fy)
                     : 0.0;
  }
}

}  // namespace

cudaError_t launch_l1_distances(const __nv_bfloat16* emb, int64_t ld, int m, int dim, float* dist,
                                cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  const int nb = (m + kDT - 1) / kDT;
  l1_distance_kernel<<<dim3(nb, nb), kDThreads, 0, st>>>(emb, ld, m, dim, dist);
  return cudaGetLastError();
}

cudaError_t launch_mmd_trials(const float* dist, int m, const int8_t* labels, int trials,
                              double* mmd, cudaStream_t st) {
  if (trials <= 0) return cudaSuccess;
  if ((size_t)m > 48 * 1024) return cudaErrorInvalidValue;
  mmd_trials_kernel<<<trials, kMThreads, (size_t)m, st>>>(dist, m, labels, mmd);
  return cudaGetLastError();
}

}  // namespace synth
