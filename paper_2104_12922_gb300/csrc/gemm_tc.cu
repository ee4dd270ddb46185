// gemm_tc.cu -- BF16 GEMM on Blackwell's 5th-generation tensor cores.
//
// C[M][N] = A[M][K] * B[N][K]^T, A and B bf16 and K-contiguous, FP32
// accumulation in tensor memory (TMEM), a fused epilogue. Used for the
// proposal MLP (and exposed as synth_gemm_bf16).
//
// Persistent: one CTA per SM walks work items -- 128 x BN output tiles (N
// fastest, so neighbouring CTAs share A rows in L2), or, when the output has
// fewer tiles than the GPU has SMs and a partial-sum workspace is given,
// (tile, K-slice) pairs of a split-K product, K-slice major so that the CTAs
// working on one slice at a time share its A columns in L2. Each split-K item
// stores its raw FP32 partial tile; splitk_reduce then adds the slices in
// slice order (the same sum whichever CTA finished first: deterministic) and
// applies the epilogue. 6 warps per CTA:
//   warp 0      TMA producer: cp.async.bulk.tensor loads of 128x64 A and BNx64 B
//               tiles (128-byte swizzle) into a STAGES-deep shared-memory ring
//               that runs on across tiles;
//   warp 1      allocates two TMEM accumulators of BN columns; one elected
//               lane issues tcgen05.mma (kind::f16, M = 128, N = BN, K = 16
//               per instruction) into the accumulator of the tile's parity;
//               tcgen05.commit frees each stage and hands a finished
//               accumulator to the epilogue;
//   warps 2..5  epilogue: tcgen05.ld of the accumulator rows (warp w owns TMEM
//               lanes 32 (w mod 4) ..), the fused epilogue, global stores, then
//               the accumulator is released -- while the MMAs of the next tile
//               already run in the other one.
// Every mbarrier wait is bounded; on timeout the CTA records an error and
// finishes.

#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "gemm_tc.h"
#include "pdl.cuh"

namespace synth {

namespace {

constexpr int BM = 128;
constexpr int BK = 64;          // one 128-byte swizzle row of bf16
constexpr int kStages = 4;
constexpr int kEpiWarps = 8;       // two per TMEM lane quarter, each half the columns
constexpr int kGemmThreads = 64 + 32 * kEpiWarps;
constexpr long long kWaitLimit = 1ll << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Waits for the phase with the given parity; false if the bounded wait ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long long i = 0; i < kWaitLimit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor for a K-major operand tile stored with the
// 128-byte swizzle (as TMA writes it): start address >> 4 in bits 0-13,
// leading byte offset (unused for this layout) in 16-29, stride byte offset
// 1024 B (8 rows of 128 B) in 32-45, descriptor version 1 in 46-47, swizzle
// mode "128B" (2) in 61-63.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits
// 4-5 = 1), bf16 A and B (bits 7-9, 10-12 = 1), both K-major, N >> 3 in bits
// 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive accumulator columns of this thread's TMEM lane, one wait.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <int BN>
struct __align__(1024) GemmSmem {
  __nv_bfloat16 a[kStages][BM * BK];
  __nv_bfloat16 b[kStages][BN * BK];
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t acc_full[2];   // MMA -> epilogue: accumulator b holds a finished tile
  uint64_t acc_empty[2];  // epilogue -> MMA: accumulator b may be overwritten
  float stage[kEpiWarps][32][33];  // per epilogue warp: a 32 x 32 chunk of its rows, padded
  uint32_t tmem_base;
  int failed;
};

static_assert(sizeof(GemmSmem<256>) + 1024 <= 232448, "GEMM shared memory within the 227 KB per CTA");

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ float sigmoidf(float x) { return 1.f / (1.f + __expf(-x)); }

// Work item -> output tile, K-slice and its k-block range [kb0, kb1).
struct GemmItem {
  int m0, n0, split, kb0, kb1;
};

__device__ __forceinline__ GemmItem gemm_item(int item, int n_tiles, int tiles_n, int bn,
                                              int kb_per, int nk) {
  GemmItem g;
  const int tile = item % n_tiles;
  g.split = item / n_tiles;
  g.m0 = (tile / tiles_n) * BM;
  g.n0 = (tile % tiles_n) * bn;
  g.kb0 = g.split * kb_per;
  g.kb1 = min(nk, g.kb0 + kb_per);
  return g;
}

// part == nullptr: the epilogue `epi` is applied to each finished tile.
// Otherwise (split-K, `splits` slices of kb_per k-blocks each) the raw
// accumulator of slice s goes to part[s][M][N].
template <int BN>
__global__ void __launch_bounds__(kGemmThreads, 1) gemm_bf16_tc(
    const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
    GemmEpilogue epi, int M, int N, int K, int splits, int kb_per, float* part,
    unsigned int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  GemmSmem<BN>& sm = *reinterpret_cast<GemmSmem<BN>*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = (K + BK - 1) / BK;
  const int tiles_n = (N + BN - 1) / BN;
  const int n_tiles = tiles_n * ((M + BM - 1) / BM);
  const int n_items = n_tiles * splits;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sm.acc_full[b], 1);
      mbar_init(&sm.acc_empty[b], kEpiWarps);  // one arrival per epilogue warp
    }
    sm.failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&sm.tmem_base)),
                 "r"((uint32_t)(2 * BN)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sm.tmem_base;
  // the set-up above reads and writes no global memory: only now wait for
  // the kernels ahead, and let the next one be scheduled
  pdl_wait();
  pdl_release();

  if (warp == 0 && lane == 0) {
    // producer: the stage ring runs on across this CTA's tiles
    int it = 0;
    for (int item = blockIdx.x; item < n_items && !sm.failed; item += gridDim.x) {
      const GemmItem g = gemm_item(item, n_tiles, tiles_n, BN, kb_per, nk);
      for (int kb = g.kb0; kb < g.kb1; ++kb, ++it) {
        const int s = it % kStages;
        const uint32_t ph = (uint32_t)(it / kStages) & 1u;
        if (!mbar_wait(&sm.empty[s], ph ^ 1u)) { sm.failed = 1; break; }
        mbar_expect_tx(&sm.full[s], (uint32_t)((BM + BN) * BK * 2));
        tma_load_2d(sm.a[s], &map_a, &sm.full[s], kb * BK, g.m0);
        tma_load_2d(sm.b[s], &map_b, &sm.full[s], kb * BK, g.n0);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: tile t of this CTA accumulates in TMEM buffer t & 1
    constexpr uint32_t idesc = idesc_bf16_f32(BM, BN);
    int it = 0, t = 0;
    for (int item = blockIdx.x; item < n_items && !sm.failed; item += gridDim.x, ++t) {
      const GemmItem g = gemm_item(item, n_tiles, tiles_n, BN, kb_per, nk);
      const int buf = t & 1;
      const uint32_t use = (uint32_t)(t >> 1);
      if (!mbar_wait(&sm.acc_empty[buf], (use & 1u) ^ 1u)) { sm.failed = 1; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t acc = tmem + (uint32_t)(buf * BN);
      for (int kb = g.kb0; kb < g.kb1; ++kb, ++it) {
        const int s = it % kStages;
        const uint32_t ph = (uint32_t)(it / kStages) & 1u;
        if (!mbar_wait(&sm.full[s], ph)) { sm.failed = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = smem_u32(sm.a[s]), b0 = smem_u32(sm.b[s]);
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk)
          umma_bf16(acc, smem_desc_sw128(a0 + kk * 32), smem_desc_sw128(b0 + kk * 32), idesc,
                    (kb != g.kb0 || kk != 0) ? 1u : 0u);
        umma_commit(&sm.empty[s]);
      }
      umma_commit(&sm.acc_full[buf]);
    }
  } else if (warp >= 2) {
    // epilogue: a warp owns 32 rows of the tile (its TMEM lane quarter). Per
    // 32-column chunk it loads the accumulator (lane = row), applies the
    // element-wise epilogue in registers, stages the chunk in shared memory
    // and writes it back row by row (lane = column: 128-byte coalesced
    // stores) and, for a transposed copy, column by column (lane = row)
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int half = (warp - 2) >> 2;  // which half of the tile's columns
    float(*S)[33] = sm.stage[warp - 2];
    int t = 0;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x, ++t) {
      const GemmItem g = gemm_item(item, n_tiles, tiles_n, BN, kb_per, nk);
      const int buf = t & 1;
      const uint32_t use = (uint32_t)(t >> 1);
      const bool ok = mbar_wait(&sm.acc_full[buf], use & 1u);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (!ok) { sm.failed = 1; break; }
      const int row0 = g.m0 + 32 * q;
      const uint32_t acc = tmem + (uint32_t)(buf * BN) + ((uint32_t)(32 * q) << 16);
      const bool act = !part && epi.kind == kEpiBiasActBF16;
#pragma unroll 1
      for (int c = half * (BN / 2); c < (half + 1) * (BN / 2); c += 32) {
        float v[32];
        tmem_ld32(acc + (uint32_t)c, v);
        const int col0 = g.n0 + c;
        if (act) {
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int col = min(col0 + i, N - 1);
            float z = v[i] + (epi.bias ? epi.bias[col] : 0.f);
            if (epi.act == kActRelu) z = fmaxf(z, 0.f);
            else if (epi.act == kActSigmoid) z = sigmoidf(z);
            v[i] = z;
          }
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 32; ++i) S[lane][i] = v[i];
        __syncwarp();
        // FP32 rows: lane = (row within 4, 4-column group); one 16-byte store
        // per lane covers four whole 128-byte row segments per instruction
        float* f32 = part ? part + (size_t)g.split * M * N : epi.out_f32;
        const size_t ld32 = part ? (size_t)N : (size_t)epi.ldc;
        const float mul = part || act ? 1.f : epi.alpha;
        const bool f32_out = part || epi.kind == kEpiStoreF32 || epi.out_f32;
        const int c4 = 4 * (lane & 7), rs = lane >> 3;
        const bool vec4 = col0 + 31 < N && (ld32 & 3) == 0 &&
                          (reinterpret_cast<uintptr_t>(f32) & 15) == 0;
        if (f32_out) {
#pragma unroll 2
          for (int r = 0; r < 32; r += 4) {
            const int row = row0 + r + rs;
            if (row >= M) continue;
            float* o = f32 + (size_t)row * ld32 + col0 + c4;
            const float* sr = S[r + rs] + c4;
            if (vec4) {
              *reinterpret_cast<float4*>(o) =
                  make_float4(sr[0] * mul, sr[1] * mul, sr[2] * mul, sr[3] * mul);
            } else {
#pragma unroll
              for (int i = 0; i < 4; ++i)
                if (col0 + c4 + i < N) o[i] = sr[i] * mul;
            }
          }
        }
        if (act && epi.out_bf16 && col0 + lane < N) {
#pragma unroll 4
          for (int r = 0; r < 32; ++r) {
            const int row = row0 + r;
            if (row >= M) break;
            epi.out_bf16[(size_t)row * epi.ldc + col0 + lane] = __float2bfloat16(S[r][lane]);
          }
        }
        if (act && epi.out_bf16_t && row0 + lane < M) {
          const int row = row0 + lane;
#pragma unroll 4
          for (int cc = 0; cc < 32; ++cc) {
            if (col0 + cc >= N) break;
            epi.out_bf16_t[(size_t)(col0 + cc) * epi.ldc_t + row] = __float2bfloat16(S[lane][cc]);
          }
        }
      }
      // the accumulator's values are all in registers or stored: release it
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.acc_empty[buf]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0 && lane == 0 && sm.failed) atomicOr(err, 1u);
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)(2 * BN)));
  }
}

// Split-K reduction with the fused epilogue: C = sum over slices s = 0, 1, ...
// of part[s] in that order, then the epilogue of `epi`. A block covers a
// 16 x 32 output tile (32 x 8 threads, 2 rows each: 256 blocks for a
// 128 x 1024 output); the transposed bf16 copy goes through shared memory
// so both of its stores are coalesced.
constexpr int kRedRows = 16;
__global__ void __launch_bounds__(256) splitk_reduce(const float* __restrict__ part, int splits,
                                                     int M, int N, GemmEpilogue epi) {
  pdl_wait();     // earlier kernels' writes are visible
  pdl_release();  // the next kernel may be scheduled
  __shared__ float tile[kRedRows][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + tx, r0 = blockIdx.y * kRedRows;
  const size_t slice = (size_t)M * N;
  // the two rows' slices, eight at a time: 16 loads in flight per thread,
  // added in slice order afterwards
  const float* p[2];
  bool ok[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int r = r0 + ty + 8 * i;
    ok[i] = r < M && c < N;
    p[i] = part + (size_t)(ok[i] ? r : 0) * N + (ok[i] ? c : 0);
  }
  float acc[2] = {0.f, 0.f};
  int k = 0;
  for (; k + 8 <= splits; k += 8) {
    float t[2][8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int i = 0; i < 2; ++i) t[i][u] = ok[i] ? p[i][(size_t)(k + u) * slice] : 0.f;
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int i = 0; i < 2; ++i) acc[i] += t[i][u];
  }
  for (; k < splits; ++k)
#pragma unroll
    for (int i = 0; i < 2; ++i) acc[i] += ok[i] ? p[i][(size_t)k * slice] : 0.f;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int r = r0 + ty + 8 * i;
    float z = 0.f;
    if (ok[i]) {
      if (epi.kind == kEpiStoreF32) {
        epi.out_f32[(size_t)r * epi.ldc + c] = acc[i] * epi.alpha;
      } else {
        z = acc[i] + (epi.bias ? epi.bias[c] : 0.f);
        if (epi.act == kActRelu) z = fmaxf(z, 0.f);
        else if (epi.act == kActSigmoid) z = sigmoidf(z);
        const __nv_bfloat16 b = __float2bfloat16(z);
        if (epi.out_bf16) epi.out_bf16[(size_t)r * epi.ldc + c] = b;
        if (epi.out_f32) epi.out_f32[(size_t)r * epi.ldc + c] = z;
        z = __bfloat162float(b);
      }
    }
    tile[ty + 8 * i][tx] = z;
  }
  if (epi.kind != kEpiBiasActBF16 || !epi.out_bf16_t) return;
  __syncthreads();
  // transposed: 16 rows of each of the 32 columns, lanes along the rows
  const int rr = threadIdx.x & 15, cq = threadIdx.x >> 4;  // 16 rows x 16 column pairs
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int cc = blockIdx.x * 32 + 2 * cq + j, r = r0 + rr;
    if (cc < N && r < M)
      epi.out_bf16_t[(size_t)cc * epi.ldc_t + r] = __float2bfloat16(tile[rr][2 * cq + j]);
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  // looked up once (thread-safe initialisation of a function-local static)
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeTiledFn>(p);
    return nullptr;
  }();
  return fn;
}

// 2-D bf16 tensor map: rows x cols (cols contiguous), row stride in elements,
// box 64 columns x box_rows rows, 128-byte swizzle, zero fill out of bounds.
bool make_map(CUtensorMap* map, const void* ptr, int rows, int cols, int ld, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  if ((reinterpret_cast<uintptr_t>(ptr) & 15) != 0 || ((size_t)ld * 2) % 16 != 0) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Per-device launch facts, set up once per device under a lock: the SM count
// and whether each instantiation's dynamic shared-memory limit is raised.
struct GemmDevice {
  int sms = 0;
  bool attr128 = false, attr256 = false;
};
constexpr int kGemmMaxDevices = 64;
std::mutex g_gemm_mutex;
GemmDevice g_gemm_dev[kGemmMaxDevices];

template <int BN>
cudaError_t gemm_device_setup(int* sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kGemmMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_gemm_mutex);
  GemmDevice& d = g_gemm_dev[dev];
  bool& attr = BN == 256 ? d.attr256 : d.attr128;
  if (!attr) {
    e = cudaFuncSetAttribute(gemm_bf16_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(GemmSmem<BN>) + 1024));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (d.sms == 0) {
    e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
  }
  *sms = d.sms;
  return cudaSuccess;
}

// K-slices for a product with `tiles` output tiles and nk k-blocks: enough
// to give every SM an item, at least 4 k-blocks per slice, within the
// workspace. Returns 1 (no split) when the tiles alone fill the GPU.
int choose_splits(int tiles, int nk, int sms, size_t slice_bytes, size_t ws_bytes, int* kb_per) {
  *kb_per = nk;
  if (tiles >= sms || slice_bytes == 0) return 1;
  int s = sms / tiles;
  s = std::min(s, (nk + 3) / 4);
  s = (int)std::min<size_t>((size_t)s, ws_bytes / slice_bytes);
  if (s <= 1) return 1;
  *kb_per = (nk + s - 1) / s;
  return (nk + *kb_per - 1) / *kb_per;
}

template <int BN>
cudaError_t launch_bn(const CUtensorMap& ma, const CUtensorMap& mb, const GemmEpilogue& epi, int M,
                      int N, int K, float* ws, size_t ws_bytes, unsigned int* err,
                      cudaStream_t st) {
  int sms = 0;
  cudaError_t e = gemm_device_setup<BN>(&sms);
  if (e != cudaSuccess) return e;
  const size_t smem = sizeof(GemmSmem<BN>) + 1024;
  const int nk = (K + BK - 1) / BK;
  const long long tiles = (long long)((N + BN - 1) / BN) * ((M + BM - 1) / BM);
  int kb_per = nk;
  const int splits =
      ws ? choose_splits((int)std::min<long long>(tiles, 1 << 30), nk, sms,
                         sizeof(float) * (size_t)M * N, ws_bytes, &kb_per)
         : 1;
  const long long items = tiles * splits;
  const int grid = (int)(items < sms ? items : sms);  // persistent: one CTA per SM
  float* part = splits > 1 ? ws : nullptr;
  e = launch_pdl(gemm_bf16_tc<BN>, dim3((unsigned)grid), dim3(kGemmThreads), smem, st, ma, mb, epi,
                 M, N, K, splits, kb_per, part, err);
  if (e != cudaSuccess || (e = cudaGetLastError()) != cudaSuccess || splits == 1) return e;
  const dim3 rgrid((N + 31) / 32, (M + kRedRows - 1) / kRedRows);
  e = launch_pdl(splitk_reduce, rgrid, dim3(256), 0, st, (const float*)ws, splits, M, N, epi);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace

cudaError_t gemm_bf16(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M,
                      int N, int K, const GemmEpilogue& epi, unsigned int* err, cudaStream_t st,
                      float* splitk_ws, size_t splitk_bytes) {
  if (M <= 0 || N <= 0 || K <= 0 || (K % 8) != 0) return cudaErrorInvalidValue;
  const int bn = N > 128 ? 256 : 128;
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, M, K, lda, BM) || !make_map(&mb, B, N, K, ldb, bn))
    return cudaErrorInvalidValue;
  if (bn == 256) return launch_bn<256>(ma, mb, epi, M, N, K, splitk_ws, splitk_bytes, err, st);
  return launch_bn<128>(ma, mb, epi, M, N, K, splitk_ws, splitk_bytes, err, st);
}

size_t gemm_splitk_workspace_bytes(int max_m, int max_n) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  // splits <= sms / tiles with tiles >= ceil(M / 128) ceil(N / 256): at most
  // sms slices of one 128 x 256 tile's worth of the output each
  const size_t tiles = (size_t)((max_m + BM - 1) / BM) * (size_t)((max_n + 255) / 256);
  const size_t per_slice = sizeof(float) * (size_t)max_m * max_n;
  const size_t slices = tiles >= (size_t)sms ? 1 : (size_t)sms / tiles;
  return slices * per_slice;
}

}  // namespace synth
