// mlp.cu -- the learned parameter proposal: log-mel features -> 4-layer MLP
// (ReLU hidden layers of width 1024, sigmoid output of the 78 normalized
// parameters), trained with MSE against the parameters the synth drew, on
// voices rendered on the fly (inverse synthesis, Sec. 2 of the paper; the
// paper trains no network itself).
//
// All contractions run on the tcgen05 GEMM (gemm_tc.cu) with bf16 operands
// and FP32 accumulation; master weights, gradients and Adam moments are FP32.
// Every operand the GEMM reads is K-contiguous, so the forward epilogues also
// write the transposed activations the weight gradients need, and the
// optimizer writes a transposed bf16 copy of the hidden weights for the
// input gradients.

#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>

#include "gemm_tc.h"
#include "mlp.h"
#include "pdl.cuh"
#include "voice_device.cuh"

namespace synth {

namespace {

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

int grid_of(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 64 ? b : 152 * 64);
}

// Uniform(-bound, bound) from Philox (key = seed, counter = (i / 4, tensor id, 0, 2)).
__global__ void init_uniform(float* w, int64_t n, float bound, uint64_t seed, uint32_t tensor) {
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint4 r = philox4x32_10(make_uint4((uint32_t)(i >> 2), tensor, 0u, 2u), key);
    const uint32_t words[4] = {r.x, r.y, r.z, r.w};
    w[i] = bound * fmaf(2.f, u01f(words[i & 3]), -1.f);
  }
}

__global__ void to_bf16(const float* __restrict__ w, int rows, int cols, __nv_bfloat16* __restrict__ wb,
                        __nv_bfloat16* __restrict__ wt, int ld_t) {
  const int64_t total = (int64_t)rows * cols;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i / cols), c = (int)(i % cols);
    const __nv_bfloat16 b = __float2bfloat16(w[i]);
    wb[i] = b;
    if (wt) wt[(int64_t)c * ld_t + r] = b;
  }
}

// out[c][r] = in[r][c] (bf16), for the input features of the first layer.
__global__ void transpose_bf16(const __nv_bfloat16* __restrict__ in, int rows, int cols,
                               __nv_bfloat16* __restrict__ out) {
  pdl_wait();     // earlier kernels' writes are visible
  pdl_release();  // the next kernel may be scheduled
  __shared__ __nv_bfloat16 tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int r = r0 + dy, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[dy][threadIdx.x] = in[(int64_t)r * cols + c];
  }
  __syncthreads();
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int c = c0 + dy, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[(int64_t)c * rows + r] = tile[threadIdx.x][dy];
  }
}

// Output layer: MSE against the target (mean over batch x outputs) through
// the sigmoid: dZ = 2 (y - u) / (B P) * y (1 - y); writes dZ and dZ^T (bf16,
// zero-padded to P_pad columns / rows), the FP32 dZ, and the loss. One
// element per thread; each block leaves its partial sum of squares in
// part[block], and the block that finishes last (a counter it resets) adds
// the partials in block order, so the loss does not depend on which block
// came last.
__global__ void __launch_bounds__(256) mse_sigmoid_grad(
    const float* __restrict__ y, const float* __restrict__ target, int batch, int P, int P_pad,
    __nv_bfloat16* __restrict__ dz, __nv_bfloat16* __restrict__ dzt, float* __restrict__ dzf,
    float* __restrict__ part, unsigned int* __restrict__ counter, float* __restrict__ loss) {
  pdl_wait();     // earlier kernels' writes are visible
  pdl_release();  // the next kernel may be scheduled
  __shared__ float red[8];
  __shared__ bool last;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const float scale = 2.f / (float)(batch * P);
  float local = 0.f;
  if (i < batch * P_pad) {
    const int b = i / P_pad, p = i % P_pad;
    float g = 0.f;
    if (p < P) {
      const float yy = y[b * P + p], d = yy - target[b * P + p];
      local = d * d;
      g = scale * d * yy * (1.f - yy);
    }
    dz[i] = __float2bfloat16(g);
    dzt[(int64_t)p * batch + b] = __float2bfloat16(g);
    dzf[i] = g;
  }
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  float t = 0.f;
  for (unsigned int k = 0; k < gridDim.x; ++k) t += reinterpret_cast<volatile float*>(part)[k];
  *counter = 0u;
  if (loss) *loss = t / (float)(batch * P);
}

// Hidden layer: dZ = dH * relu'(Z) with relu'(Z) = (H > 0); writes dZ, dZ^T
// and the FP32 dZ. A block covers 32 batch rows x 32 columns (32 x 8
// threads); the transposed copy goes through shared memory so that its
// stores are coalesced too.
__global__ void __launch_bounds__(256) relu_grad(const float* __restrict__ dh,
                                                 const __nv_bfloat16* __restrict__ h, int batch,
                                                 int width, __nv_bfloat16* __restrict__ dz,
                                                 __nv_bfloat16* __restrict__ dzt,
                                                 float* __restrict__ dzf) {
  pdl_wait();     // earlier kernels' writes are visible
  pdl_release();  // the next kernel may be scheduled
  __shared__ __nv_bfloat16 tile[32][34];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + tx, b0 = blockIdx.y * 32;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int b = b0 + ty + 8 * k;
    __nv_bfloat16 gb = __float2bfloat16(0.f);
    if (b < batch && c < width) {
      const int64_t i = (int64_t)b * width + c;
      const float g = __bfloat162float(h[i]) > 0.f ? dh[i] : 0.f;
      gb = __float2bfloat16(g);
      dz[i] = gb;
      dzf[i] = g;
    }
    tile[ty + 8 * k][tx] = gb;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int cc = blockIdx.x * 32 + ty + 8 * k, b = b0 + tx;
    if (cc < width && b < batch) dzt[(int64_t)cc * batch + b] = tile[tx][ty + 8 * k];
  }
}

// Bias gradient: db[c] = sum_b dZ[b][c] from the FP32 dZ. A block covers 32
// columns with 8 threads per column, each adding every 8th row; the eight
// partial sums are then added in thread order (deterministic).
__global__ void __launch_bounds__(256) bias_grad(const float* __restrict__ dz, int batch, int width,
                                                 int ld, float* __restrict__ db) {
  pdl_wait();     // earlier kernels' writes are visible
  pdl_release();  // the next kernel may be scheduled
  __shared__ float part[8][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + tx;
  float s = 0.f;
  if (c < width)
    for (int b = ty; b < batch; b += 8) s += dz[(int64_t)b * ld + c];
  part[ty][tx] = s;
  __syncthreads();
  if (ty == 0 && c < width) {
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += part[k][tx];
    db[c] = t;
  }
}

// Adam (Kingma & Ba, 2015) on FP32 master values; also refreshes the bf16
// copy the GEMMs read. Vectorised by 4 (n a multiple of 4, 16-byte aligned
// arrays): an HBM-bound stream of 16 bytes read and 14 written per value.
__device__ __forceinline__ float adam_one(float& w, float g, float& m, float& v, float lr,
                                          float b1, float b2, float eps, float c1, float c2) {
  m = b1 * m + (1.f - b1) * g;
  v = b2 * v + (1.f - b2) * g * g;
  w = w - lr * (m / c1) / (sqrtf(v / c2) + eps);
  return w;
}

// A layer's bias vector, updated by the same launch as its weights.
struct BiasAdam {
  float* w;
  const float* g;
  float* m;
  float* v;
  int n;
};

__device__ __forceinline__ void bias_adam_one(const BiasAdam& b, int j, float lr, float b1,
                                              float b2, float eps, float c1, float c2) {
  float wi = b.w[j], mi = b.m[j], vi = b.v[j];
  adam_one(wi, b.g[j], mi, vi, lr, b1, b2, eps, c1, c2);
  b.w[j] = wi;
  b.m[j] = mi;
  b.v[j] = vi;
}

__global__ void adam_update_vec4(float4* __restrict__ w, const float4* __restrict__ g,
                                 float4* __restrict__ m, float4* __restrict__ v, int64_t n4,
                                 float lr, float b1, float b2, float eps, float c1, float c2,
                                 uint2* __restrict__ wb, const BiasAdam bias) {
  pdl_wait();     // earlier kernels' writes are visible
  pdl_release();  // the next kernel may be scheduled
  // indices n4 .. n4 + bias.n - 1 are the bias entries
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4 + bias.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i >= n4) {
      bias_adam_one(bias, (int)(i - n4), lr, b1, b2, eps, c1, c2);
      continue;
    }
    float4 wi = w[i], mi = m[i], vi = v[i];
    const float4 gi = g[i];
    adam_one(wi.x, gi.x, mi.x, vi.x, lr, b1, b2, eps, c1, c2);
    adam_one(wi.y, gi.y, mi.y, vi.y, lr, b1, b2, eps, c1, c2);
    adam_one(wi.z, gi.z, mi.z, vi.z, lr, b1, b2, eps, c1, c2);
    adam_one(wi.w, gi.w, mi.w, vi.w, lr, b1, b2, eps, c1, c2);
    w[i] = wi;
    m[i] = mi;
    v[i] = vi;
    if (wb) {
      __nv_bfloat162 lo = __floats2bfloat162_rn(wi.x, wi.y), hi = __floats2bfloat162_rn(wi.z, wi.w);
      wb[i] = make_uint2(*reinterpret_cast<uint32_t*>(&lo), *reinterpret_cast<uint32_t*>(&hi));
    }
  }
}

// Adam on a weight matrix [rows][cols] that also keeps a transposed bf16 copy
// wt[col][row] (row stride ld_t): a block updates a 32 x 32 tile (32 x 8
// threads) and writes the transposed copy through shared memory, coalesced;
// the blocks of the first tile column also update the bias of their rows.
__global__ void __launch_bounds__(256) adam_update_tiled(
    float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
    float* __restrict__ v, int rows, int cols, float lr, float b1, float b2, float eps, float c1,
    float c2, __nv_bfloat16* __restrict__ wb, __nv_bfloat16* __restrict__ wt, int ld_t,
    const BiasAdam bias) {
  pdl_wait();     // earlier kernels' writes are visible
  pdl_release();  // the next kernel may be scheduled
  __shared__ __nv_bfloat16 tile[32][34];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + tx, r0 = blockIdx.y * 32;
  if (blockIdx.x == 0 && ty == 0 && r0 + tx < bias.n)
    bias_adam_one(bias, r0 + tx, lr, b1, b2, eps, c1, c2);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int r = r0 + ty + 8 * k;
    __nv_bfloat16 b = __float2bfloat16(0.f);
    if (r < rows && c < cols) {
      const int64_t i = (int64_t)r * cols + c;
      float wi = w[i], mi = m[i], vi = v[i];
      adam_one(wi, g[i], mi, vi, lr, b1, b2, eps, c1, c2);
      w[i] = wi;
      m[i] = mi;
      v[i] = vi;
      b = __float2bfloat16(wi);
      wb[i] = b;
    }
    tile[ty + 8 * k][tx] = b;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int cc = blockIdx.x * 32 + ty + 8 * k, r = r0 + tx;
    if (cc < cols && r < rows) wt[(int64_t)cc * ld_t + r] = tile[tx][ty + 8 * k];
  }
}

// Hidden activations (bf16) to FP32, for inspection.
__global__ void bf16_to_f32(const __nv_bfloat16* __restrict__ in, int64_t n, float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __bfloat162float(in[i]);
}

}  // namespace

// ---------------------------------------------------------------- layout
MlpLayout mlp_layout(int in_dim, int hidden, int out_dim, int max_batch, size_t splitk_bytes) {
  MlpLayout L;
  L.dims[0] = in_dim;
  L.dims[1] = L.dims[2] = L.dims[3] = hidden;
  L.dims[4] = out_dim;
  L.out_pad = (out_dim + 7) & ~7;
  L.max_batch = max_batch;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o = al256(o + bytes); return at; };
  for (int l = 0; l < 4; ++l) {
    const size_t in = L.dims[l], out = L.dims[l + 1];
    L.w[l] = take(sizeof(float) * in * out);
    L.b[l] = take(sizeof(float) * out);
    L.mw[l] = take(sizeof(float) * in * out);
    L.vw[l] = take(sizeof(float) * in * out);
    L.mb[l] = take(sizeof(float) * out);
    L.vb[l] = take(sizeof(float) * out);
    L.gw[l] = take(sizeof(float) * in * out);
    L.gb[l] = take(sizeof(float) * out);
    L.wb[l] = take(sizeof(__nv_bfloat16) * in * out);
    // transposed bf16 weights [in][out_pad] for the input gradient (layers 1..3)
    const size_t outp = l == 3 ? (size_t)L.out_pad : out;
    L.wt[l] = l == 0 ? 0 : take(sizeof(__nv_bfloat16) * in * outp);
  }
  const size_t B = max_batch;
  L.h0t = take(sizeof(__nv_bfloat16) * in_dim * B);
  for (int l = 1; l < 4; ++l) {
    L.h[l] = take(sizeof(__nv_bfloat16) * B * hidden);
    L.ht[l] = take(sizeof(__nv_bfloat16) * hidden * B);
  }
  L.y = take(sizeof(float) * B * out_dim);
  L.dz = take(sizeof(__nv_bfloat16) * B * (hidden > L.out_pad ? hidden : L.out_pad));
  L.dzt = take(sizeof(__nv_bfloat16) * B * (hidden > L.out_pad ? hidden : L.out_pad));
  L.dzf = take(sizeof(float) * B * (hidden > L.out_pad ? hidden : L.out_pad));
  L.dh = take(sizeof(float) * B * hidden);
  L.loss = take(sizeof(float) * 4);
  L.loss_part = take(sizeof(float) * (size_t)((max_batch * L.out_pad + 255) / 256));
  L.loss_counter = take(sizeof(unsigned int));
  L.splitk_bytes = splitk_bytes;
  L.splitk = take(splitk_bytes);
  L.total = o;
  return L;
}

cudaError_t mlp_init(const MlpLayout& L, char* base, uint64_t seed, cudaStream_t st) {
  cudaMemsetAsync(base, 0, L.total, st);
  for (int l = 0; l < 4; ++l) {
    const int64_t n = (int64_t)L.dims[l] * L.dims[l + 1];
    const float bound = 1.0f / sqrtf((float)L.dims[l]);
    init_uniform<<<grid_of(n), 256, 0, st>>>(reinterpret_cast<float*>(base + L.w[l]), n, bound,
                                             seed, (uint32_t)l);
    const int outp = l == 3 ? L.out_pad : L.dims[l + 1];
    to_bf16<<<grid_of(n), 256, 0, st>>>(reinterpret_cast<float*>(base + L.w[l]), L.dims[l + 1],
                                        L.dims[l], reinterpret_cast<__nv_bfloat16*>(base + L.wb[l]),
                                        l == 0 ? nullptr
                                               : reinterpret_cast<__nv_bfloat16*>(base + L.wt[l]),
                                        outp);
  }
  return cudaGetLastError();
}

cudaError_t mlp_forward(const MlpLayout& L, char* base, const __nv_bfloat16* x, int batch,
                        bool keep_transposes, float* y_out, unsigned int* err, cudaStream_t st) {
  const __nv_bfloat16* in = x;
  int in_dim = L.dims[0];
  cudaError_t e;
  for (int l = 0; l < 4; ++l) {
    const int out = L.dims[l + 1];
    GemmEpilogue ep;
    ep.kind = kEpiBiasActBF16;
    ep.bias = reinterpret_cast<const float*>(base + L.b[l]);
    if (l < 3) {
      ep.act = kActRelu;
      ep.out_bf16 = reinterpret_cast<__nv_bfloat16*>(base + L.h[l + 1]);
      ep.ldc = out;
      if (keep_transposes) {
        ep.out_bf16_t = reinterpret_cast<__nv_bfloat16*>(base + L.ht[l + 1]);
        ep.ldc_t = batch;
      }
    } else {
      ep.act = kActSigmoid;
      ep.out_f32 = y_out ? y_out : reinterpret_cast<float*>(base + L.y);
      ep.ldc = out;
    }
    e = gemm_bf16(in, in_dim, reinterpret_cast<const __nv_bfloat16*>(base + L.wb[l]), in_dim, batch,
                  out, in_dim, ep, err, st, reinterpret_cast<float*>(base + L.splitk),
                  L.splitk_bytes);
    if (e != cudaSuccess) return e;
    in = reinterpret_cast<const __nv_bfloat16*>(base + L.h[l + 1 < 4 ? l + 1 : 3]);
    in_dim = out;
  }
  return cudaGetLastError();
}

cudaError_t mlp_train_step(const MlpLayout& L, char* base, const __nv_bfloat16* x,
                           const float* target, int batch, float lr, int step, float* loss_out,
                           unsigned int* err, cudaStream_t st) {
  if (batch % 8 != 0 || batch > L.max_batch) return cudaErrorInvalidValue;
  cudaError_t e = mlp_forward(L, base, x, batch, true, nullptr, err, st);
  if (e != cudaSuccess) return e;
  __nv_bfloat16* h0t = reinterpret_cast<__nv_bfloat16*>(base + L.h0t);
  {
    dim3 g((L.dims[0] + 31) / 32, (batch + 31) / 32), b(32, 8);
    if ((e = launch_pdl(transpose_bf16, g, b, 0, st, x, batch, L.dims[0], h0t)) != cudaSuccess)
      return e;
  }
  __nv_bfloat16* dz = reinterpret_cast<__nv_bfloat16*>(base + L.dz);
  __nv_bfloat16* dzt = reinterpret_cast<__nv_bfloat16*>(base + L.dzt);
  float* dh = reinterpret_cast<float*>(base + L.dh);
  float* dzf = reinterpret_cast<float*>(base + L.dzf);
  float* loss = reinterpret_cast<float*>(base + L.loss);
  const int P = L.dims[4], Pp = L.out_pad;
  if ((e = launch_pdl(mse_sigmoid_grad, dim3((batch * Pp + 255) / 256), dim3(256), 0, st,
                      reinterpret_cast<const float*>(base + L.y), target, batch, P, Pp, dz, dzt,
                      dzf, reinterpret_cast<float*>(base + L.loss_part),
                      reinterpret_cast<unsigned int*>(base + L.loss_counter), loss)) != cudaSuccess)
    return e;
  for (int l = 3; l >= 0; --l) {
    const int in = L.dims[l], out = L.dims[l + 1];
    const int ldz = l == 3 ? Pp : out;
    // bias and weight gradients: dW[out][in] = dZ^T[out][B] * H_{l}^T[in][B]^T
    if ((e = launch_pdl(bias_grad, dim3((out + 31) / 32), dim3(256), 0, st, (const float*)dzf,
                        batch, out, ldz, reinterpret_cast<float*>(base + L.gb[l]))) != cudaSuccess)
      return e;
    const __nv_bfloat16* hprev_t =
        l == 0 ? h0t : reinterpret_cast<const __nv_bfloat16*>(base + L.ht[l]);
    GemmEpilogue ew;
    ew.kind = kEpiStoreF32;
    ew.out_f32 = reinterpret_cast<float*>(base + L.gw[l]);
    ew.ldc = in;
    if ((e = gemm_bf16(dzt, batch, hprev_t, batch, out, in, batch, ew, err, st)) != cudaSuccess)
      return e;
    if (l > 0) {
      // dH_{l}[B][in] = dZ[B][ldz] * W^T[in][ldz]^T
      GemmEpilogue eh;
      eh.kind = kEpiStoreF32;
      eh.out_f32 = dh;
      eh.ldc = in;
      if ((e = gemm_bf16(dz, ldz, reinterpret_cast<const __nv_bfloat16*>(base + L.wt[l]), ldz,
                         batch, in, ldz, eh, err, st, reinterpret_cast<float*>(base + L.splitk),
                         L.splitk_bytes)) != cudaSuccess)
        return e;
      if ((e = launch_pdl(relu_grad, dim3((in + 31) / 32, (batch + 31) / 32), dim3(256), 0, st,
                          (const float*)dh, reinterpret_cast<const __nv_bfloat16*>(base + L.h[l]),
                          batch, in, dz, dzt, dzf)) != cudaSuccess)
        return e;
    }
  }
  // Adam: each layer's weights and bias in one launch
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  for (int l = 0; l < 4; ++l) {
    const int in = L.dims[l], out = L.dims[l + 1];
    float* w = reinterpret_cast<float*>(base + L.w[l]);
    const float* g = reinterpret_cast<const float*>(base + L.gw[l]);
    float* mw = reinterpret_cast<float*>(base + L.mw[l]);
    float* vw = reinterpret_cast<float*>(base + L.vw[l]);
    __nv_bfloat16* wb = reinterpret_cast<__nv_bfloat16*>(base + L.wb[l]);
    const BiasAdam bias{reinterpret_cast<float*>(base + L.b[l]),
                        reinterpret_cast<const float*>(base + L.gb[l]),
                        reinterpret_cast<float*>(base + L.mb[l]),
                        reinterpret_cast<float*>(base + L.vb[l]), out};
    if (l == 0) {
      // no transposed copy: a vectorised stream (in * out is a multiple of 4)
      const int64_t n4 = (int64_t)in * out / 4;
      if ((e = launch_pdl(adam_update_vec4, dim3(grid_of(n4 + out)), dim3(256), 0, st,
                          reinterpret_cast<float4*>(w), reinterpret_cast<const float4*>(g),
                          reinterpret_cast<float4*>(mw), reinterpret_cast<float4*>(vw), n4, lr, b1,
                          b2, eps, c1, c2, reinterpret_cast<uint2*>(wb), bias)) != cudaSuccess)
        return e;
    } else {
      const int outp = l == 3 ? Pp : out;
      if ((e = launch_pdl(adam_update_tiled, dim3((in + 31) / 32, (out + 31) / 32), dim3(256), 0,
                          st, w, g, mw, vw, out, in, lr, b1, b2, eps, c1, c2, wb,
                          reinterpret_cast<__nv_bfloat16*>(base + L.wt[l]), outp, bias)) !=
          cudaSuccess)
        return e;
    }
  }
  // the loss last, so that no copy splits the chain of kernels above
  if (loss_out &&
      (e = cudaMemcpyAsync(loss_out, loss, sizeof(float), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
    return e;
  return cudaGetLastError();
}

cudaError_t mlp_hidden_f32(const MlpLayout& L, const char* base, int layer, int batch, float* dst,
                           cudaStream_t st) {
  if (layer < 1 || layer > 3 || batch < 1 || batch > L.max_batch) return cudaErrorInvalidValue;
  const int64_t n = (int64_t)batch * L.dims[layer];
  bf16_to_f32<<<grid_of(n), 256, 0, st>>>(
      reinterpret_cast<const __nv_bfloat16*>(base + L.h[layer]), n, dst);
  return cudaGetLastError();
}

// Adam on normalized Voice parameters (refinement in parameter space), kept
// inside [0, 1].
__global__ void param_adam_kernel(float* u, const float* g, float* m, float* v, int n, float lr,
                                  float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  u[i] = fminf(fmaxf(u[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f), 0.f), 1.f);
}

cudaError_t param_adam(float* u, const float* g, float* m, float* v, int n, int step, float lr,
                       cudaStream_t st) {
  const float c1 = 1.f - powf(0.9f, (float)step), c2 = 1.f - powf(0.999f, (float)step);
  param_adam_kernel<<<(n + 255) / 256, 256, 0, st>>>(u, g, m, v, n, lr, c1, c2);
  return cudaGetLastError();
}

}  // namespace synth
