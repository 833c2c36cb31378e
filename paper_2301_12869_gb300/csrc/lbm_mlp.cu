// Learned warm start for the liquid-column runs: a 6 -> 128 -> 128 -> 128 -> 1 SiLU
// network that predicts the steady density profile rho(z)/rho_c of a column from
// (T/T_c, log10|g|, gravity form, <rho>/rho_c, z/H, log2 H). It has no counterpart in the paper;
// it only initialises lattice Boltzmann runs (Sec. IV set-up), which decide the result.
//
// Arithmetic: bfloat16 inputs, weights and activations as matrix operands, FP32
// accumulation, FP32 biases, output layer, loss and Adam (FP32 master weights).
//
// Every matrix product runs on the tcgen05 tensor cores through one GEMM kernel,
// C[M x N] = A[M x K] B[N x K]^T with A and B bfloat16, K contiguous:
//  * a CTA (4 warps) owns a 128 x 128 output tile whose FP32 accumulator lives in 128
//    TMEM columns; K is consumed in chunks of 64 through kStages shared-memory stages;
//  * one thread (the producer) fills a stage with two TMA tile copies: a 2-D tensor map
//    over each row-major operand with a 64-element (128 B) x 128-row box and the 128-byte
//    swizzle lands the chunk as 128 rows of 128 B, the 16-byte pieces of row r permuted by
//    r mod 8 - the K-major SWIZZLE_128B layout that the MMA's matrix descriptor names
//    (8-row groups 1024 B apart; the K = 16 steps start 32 B apart); the copies complete
//    on the stage's `full` mbarrier;
//  * a second thread waits for a full stage, issues four 128 x 128 x 16 MMAs on it and
//    commits them to the stage's `empty` mbarrier, which the producer waits for before
//    refilling the stage, and after the last chunk to the `done` mbarrier;
//  * the epilogue reads the accumulator with tcgen05.ld (warp w: rows 32w..32w+31, one row
//    per lane), turns each 32 x 32 piece around in shared memory so that the lanes run
//    along a row of C, and applies a fused operation with coalesced accesses: store,
//    split-K atomic add, bias + SiLU (forward), or the SiLU derivative (backward) with the
//    bias gradient as a column sum; transposed bfloat16 copies go out with the lanes
//    along the rows again.
// Waits are bounded (clock64); a timeout sets the status word and the CTA still waits
// (bounded) for its MMAs and frees its TMEM before returning.
#include "lbm.h"
#include "lbm_internal.h"
#include "lbm_ptx.cuh"

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

namespace {

using bf16 = __nv_bfloat16;
using lbm::kWaitCycles;

constexpr int W = LBM_MLP_WIDTH;      // 128
constexpr int KIN = LBM_MLP_IN_PAD;   // 16: inputs padded to one MMA K step
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + W * KIN;
constexpr int OFF_W2 = OFF_B1 + W;
constexpr int OFF_B2 = OFF_W2 + W * W;
constexpr int OFF_W3 = OFF_B2 + W;
constexpr int OFF_B3 = OFF_W3 + W * W;
constexpr int OFF_W4 = OFF_B3 + W;
constexpr int OFF_B4 = OFF_W4 + W;
constexpr int NPARAM = OFF_B4 + 1;
static_assert(NPARAM == LBM_MLP_NPARAMS, "parameter layout");

// feature normalisation x_norm = (x - c) / s
__constant__ float kCenter[LBM_MLP_INPUTS] = {0.825f, -5.0f, 1.5f, 1.4f, 0.5f, 8.0f};
__constant__ float kScale[LBM_MLP_INPUTS] = {0.125f, 1.0f, 0.5f, 1.1f, 0.5f, 2.0f};

// ------------------------------------------------------------------ GEMM
constexpr int BM = 128, BN = 128, BK = 64, GT = 128;
constexpr int kStages = 3;
constexpr int TILE_BYTES = BM * BK * 2;   // one operand, one stage: 16 KB
constexpr int GEMM_SMEM = 2 * kStages * TILE_BYTES + 1024 + 128;  // stages, alignment, barriers
// instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B bfloat16 (bits 7-9,
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(BN >> 3) << 17) | (uint32_t(BM >> 4) << 24);

enum Epi : int { EPI_STORE = 0, EPI_ATOMIC = 1, EPI_FWD = 2, EPI_BWD = 3 };

struct GemmArgs {
  const bf16* A;
  int lda;
  const bf16* B;
  int ldb;
  int M, N, K, k_split;  // k_split: K range per blockIdx.z (multiple of BK)
  float* C;              // EPI_STORE / EPI_ATOMIC: C[m * ldc + n]
  int ldc;
  const float* bias;     // EPI_FWD: z = acc + bias[n]
  float* Z;              // EPI_FWD: z stored; EPI_BWD: z read (SiLU derivative)
  int ldz;
  bf16* H;               // EPI_FWD: silu(z); EPI_BWD: dz = acc silu'(z)  ([m][n], may be NULL)
  int ldh;
  bf16* HT;              // the same values transposed ([n][m], may be NULL)
  int ldht;
  float* colsum;         // EPI_BWD: colsum[n] += sum over m of dz (may be NULL)
  int* status;
};

// shared-memory matrix descriptor, K-major with the 128-byte swizzle (layout type 2 in bits
// 61-63): SBO = 1024 B between 8-row groups, LBO unused inside one swizzle atom (16 B by
// convention), descriptor version 1 (bits 46-47); p lies in a 1024-byte aligned tile,
// offset by 32 B per K = 16 step
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
  const uint32_t a = lbm::smem_u32(p);
  return uint64_t((a >> 4) & 0x3FFF) | (uint64_t(1) << 16) | (uint64_t(1024 >> 4) << 32) | (uint64_t(1) << 46) |
         (uint64_t(2) << 61);
}

// TMA: one box of a 2-D tensor map (x = element along K, y = row) into shared memory,
// completing on an mbarrier
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          lbm::smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(lbm::smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(lbm::smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float dsilu_f(float z) {
  const float s = 1.0f / (1.0f + expf(-z));
  return s * (1.0f + z * (1.0f - s));
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int EPI>
__global__ void __launch_bounds__(GT, 1)
    gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, const GemmArgs g) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;                          // stage s at sA + s * TILE_BYTES
  uint8_t* sB = smem + kStages * TILE_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + 2 * kStages * TILE_BYTES);
  uint64_t* empty = full + kStages;
  uint64_t* done = empty + kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* err_s = reinterpret_cast<int*>(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kbeg = blockIdx.z * g.k_split;
  const int kend = min(g.K, kbeg + g.k_split);
  const int nchunks = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;
  if (nchunks == 0) return;  // uniform over the CTA, before any allocation

  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      lbm::mbar_init(&full[i], 1);
      lbm::mbar_init(&empty[i], 1);
    }
    lbm::mbar_init(done, 1);
    *err_s = 0;
    lbm::fence_mbar_init();
  }
  if (warp == 0) {
    lbm::tmem_alloc(tmem_slot, BN);
    lbm::tmem_relinquish();
  }
  lbm::tc_fence_before();
  __syncthreads();
  lbm::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // K = 16 steps of chunk c (the last chunk may be short: K is a multiple of 16; the box
  // reads zeros beyond K, and a split boundary is a multiple of BK)
  auto ksteps = [&](int c) { return min(BK, kend - (kbeg + c * BK)) / 16; };

  int c = 0;  // producer: chunks whose copies were issued
  if (tid == 0) {
    // producer: TMA copies of A and B for every chunk, each into a free stage
    for (; c < nchunks; ++c) {
      const int st = c % kStages;
      if (c >= kStages && !lbm::mbar_wait_bounded(&empty[st], uint32_t(((c / kStages) - 1) & 1))) {
        atomicOr(err_s, 1);
        break;
      }
      mbar_expect_tx(&full[st], uint32_t(2 * TILE_BYTES));  // whole boxes, zero fill included
      const int k = kbeg + c * BK;
      tma_load_2d(sA + st * TILE_BYTES, &mapA, k, m0, &full[st]);
      tma_load_2d(sB + st * TILE_BYTES, &mapB, k, n0, &full[st]);
    }
  } else if (tid == 32) {
    // MMA issuer: four K = 16 steps per chunk, the stage freed by the commit
    for (int c = 0; c < nchunks; ++c) {
      const int st = c % kStages;
      if (!lbm::mbar_wait_bounded(&full[st], uint32_t((c / kStages) & 1))) {
        atomicOr(err_s, 1);
        break;
      }
      lbm::tc_fence_after();
      const int steps = ksteps(c);
      for (int j = 0; j < steps; ++j)
        lbm::tc_mma_f16(tmem, smem_desc(sA + st * TILE_BYTES + 32 * j), smem_desc(sB + st * TILE_BYTES + 32 * j),
                        kIdesc, (c > 0 || j > 0) ? 1u : 0u);
      lbm::tc_commit(&empty[st]);
    }
    lbm::tc_commit(done);  // every MMA issued so far, also after an error
  }
  // the accumulator is final once `done` completes
  const bool fin = lbm::mbar_wait_bounded(done, 0u);
  bool ok = __syncthreads_and(fin && *err_s == 0);
  lbm::tc_fence_after();
  if (!ok) {
    if (tid == 0) {
      atomicOr(g.status, lbm::STATUS_TIMEOUT);
      // copies in flight must land before the CTA's shared memory goes away: only the last
      // kStages issued chunks can be outstanding (a stage is refilled after its previous
      // chunk was consumed); bounded waits
      for (int q = max(0, c - kStages); q < c; ++q)
        (void)lbm::mbar_wait_bounded(&full[q % kStages], uint32_t((q / kStages) & 1), kWaitCycles / 8);
    }
  } else {
    // each warp stages its 32 x 32 pieces of the accumulator through a padded shared tile
    // (the drained stage buffers) so that global rows are written by 32 lanes at once:
    // t[r][c] holds row 32 warp + r, column nb + c
    float* t = reinterpret_cast<float*>(smem) + warp * (32 * 33);
    const int mw = m0 + 32 * warp;
    float csum = 0.0f;  // EPI_BWD: this lane's column sum over the warp's rows
#pragma unroll 1
    for (int cc = 0; cc < BN / 32; ++cc) {
      float v[32];
      lbm::tmem_ld32(tmem + (uint32_t(32 * warp) << 16) + uint32_t(32 * cc), v);
      const int nb = n0 + 32 * cc;
      const int n = nb + lane;
#pragma unroll
      for (int i = 0; i < 32; ++i) t[lane * 33 + i] = v[i];
      __syncwarp();
      if constexpr (EPI == EPI_BWD) csum = 0.0f;
#pragma unroll 4
      for (int r = 0; r < 32; ++r) {
        const int m = mw + r;
        const bool in = m < g.M && n < g.N;
        const float x = t[r * 33 + lane];
        if constexpr (EPI == EPI_STORE) {
          if (in) g.C[size_t(m) * g.ldc + n] = x;
        } else if constexpr (EPI == EPI_ATOMIC) {
          if (in) atomicAdd(g.C + size_t(m) * g.ldc + n, x);
        } else if constexpr (EPI == EPI_FWD) {
          if (in) {
            const float z = x + g.bias[n];
            g.Z[size_t(m) * g.ldz + n] = z;
            const bf16 h = __float2bfloat16_rn(silu_f(z));
            if (g.H) g.H[size_t(m) * g.ldh + n] = h;
            t[r * 33 + lane] = __bfloat162float(h);
          }
        } else {  // EPI_BWD
          const float dz = in ? x * dsilu_f(g.Z[size_t(m) * g.ldz + n]) : 0.0f;
          const bf16 d = __float2bfloat16_rn(dz);
          if (in && g.H) g.H[size_t(m) * g.ldh + n] = d;
          t[r * 33 + lane] = __bfloat162float(d);
          csum += dz;
        }
      }
      if constexpr (EPI == EPI_FWD || EPI == EPI_BWD) {
        if (g.colsum && n < g.N) atomicAdd(g.colsum + n, csum);
        // the transposed copy, lanes along rows again: HT[n][m] for consecutive m
        if (g.HT) {
          __syncwarp();
          const int m = mw + lane;
#pragma unroll 4
          for (int i = 0; i < 32; ++i)
            if (m < g.M && nb + i < g.N) g.HT[size_t(nb + i) * g.ldht + m] = __float2bfloat16_rn(t[lane * 33 + i]);
        }
      }
      __syncwarp();
    }
  }
  lbm::tc_fence_before();
  __syncthreads();
  if (warp == 0) lbm::tmem_dealloc(tmem, BN);
}

// ------------------------------------------------------------------ fused forward pass
// The whole network for 128-row tiles in one persistent kernel (inference: lbm_mlp_predict
// and the warm start). The weights stay in shared memory for the CTA's lifetime (TMA, the
// GEMM's 128-byte-swizzled K-major layout), the biases and w4 beside them. The CTA runs
// four independent tile pipelines (groups of 4 warps), each with its own activation
// buffer, TMEM accumulator (128 of the SM's 512 columns), mbarrier and named barrier, so
// the groups' MMAs overlap each other's epilogues. Per tile
// the group's 128 threads (one row each) write their normalised bfloat16 inputs into the
// A-operand buffer, one thread issues the layer's MMAs, and every thread reads its row
// back (tcgen05.ld), adds the bias, applies SiLU and writes the bfloat16 activations
// straight into the same A-operand buffer in the swizzled layout the next layer's
// descriptor names (16-byte piece j of row r at piece position j ^ (r mod 8)). After the
// third layer the output layer is a dot product with w4 in registers. Rounding points as
// in the GEMM path: bfloat16 inputs, weights and H1, H2; FP32 accumulation, biases, H3
// and output.
constexpr int FF_GROUPS = 4;                         // tile pipelines per CTA
constexpr int FF_THREADS = 128 * FF_GROUPS;           // one group = 4 warps = 128 rows
constexpr int FF_BOX = BK * 128 * 2;                 // one 64-element x 128-row swizzled box: 16 KB
constexpr int FF_W1 = 0;                             // W1 (K = 16, zero-filled to the box)
constexpr int FF_W2 = FF_W1 + FF_BOX;                // W2: two K boxes
constexpr int FF_W3 = FF_W2 + 2 * FF_BOX;            // W3: two K boxes
constexpr int FF_H = FF_W3 + 2 * FF_BOX;             // per group: activations / inputs, two K boxes
constexpr int FF_VEC = FF_H + 2 * FF_BOX * FF_GROUPS; // b1, b2, b3, w4 (FP32), b4
constexpr int FF_BAR = FF_VEC + (4 * 128 + 4) * 4;   // mbarriers, TMEM slot
constexpr int FF_SMEM = FF_BAR + 64 + 1024;          // + alignment slack: 211 KB

// 16-byte piece (8 bfloat16 values, k = 8 j .. 8 j + 7) of row r of a K-major operand held in
// 128-byte-swizzled boxes of 64 K values
__device__ __forceinline__ void ff_store8(uint8_t* base, int r, int j, const float (&v)[8]) {
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    w[i] = *reinterpret_cast<const uint32_t*>(&b);
  }
  uint8_t* dst = base + (j >> 3) * FF_BOX + r * 128 + (((j & 7) ^ (r & 7)) << 4);
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(lbm::smem_u32(dst)), "r"(w[0]), "r"(w[1]),
               "r"(w[2]), "r"(w[3])
               : "memory");
}

__device__ __forceinline__ float silu_fast(float z) { return __fdividef(z, 1.0f + __expf(-z)); }

// barrier among the 128 threads of group g (named barrier 1 + g) returning the AND of v
__device__ __forceinline__ bool group_and(bool v, int g) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.b32 p, %1, 0;\n\t"
      "bar.red.and.pred q, %2, 128, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(uint32_t(v)), "r"(1 + g)
      : "memory");
  return r != 0;
}

__global__ void __launch_bounds__(FF_THREADS, 1)
    mlp_forward_kernel(const __grid_constant__ CUtensorMap mapW1, const __grid_constant__ CUtensorMap mapW2,
                       const __grid_constant__ CUtensorMap mapW3, const float* __restrict__ P,
                       const float* __restrict__ feat, long long n, float* __restrict__ y, int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* wbar = reinterpret_cast<uint64_t*>(smem + FF_BAR);
  uint64_t* mbars = wbar + 1;  // one per group
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbars + FF_GROUPS);
  float* vec = reinterpret_cast<float*>(smem + FF_VEC);  // b1 [0, 128), b2, b3, w4, b4 [512]
  const int tid = threadIdx.x, warp = tid >> 5;
  const int g = warp >> 2, r = tid & 127;  // group, and this thread's row within the tile
  const long long ntiles = (n + 127) / 128;

  if (tid == 0) {
    lbm::mbar_init(wbar, 1);
    for (int i = 0; i < FF_GROUPS; ++i) lbm::mbar_init(&mbars[i], 1);
    lbm::fence_mbar_init();
  }
  for (int i = tid; i < 4 * 128 + 1; i += FF_THREADS)
    vec[i] = P[i < 128 ? OFF_B1 + i : (i < 256 ? OFF_B2 + i - 128 : (i < 384 ? OFF_B3 + i - 256 : (i < 512 ? OFF_W4 + i - 384 : OFF_B4)))];
  if (warp == 0) {
    lbm::tmem_alloc(tmem_slot, 128 * FF_GROUPS);
    lbm::tmem_relinquish();
  }
  lbm::tc_fence_before();
  __syncthreads();
  lbm::tc_fence_after();
  const uint32_t tmem = *tmem_slot + uint32_t(128 * g) + (uint32_t(32 * (warp & 3)) << 16);  // group columns, warp lanes
  const uint32_t tmem_acc = *tmem_slot + uint32_t(128 * g);
  uint8_t* sH = smem + FF_H + g * 2 * FF_BOX;
  uint64_t* mbar = &mbars[g];
  if (tid == 0) {  // the three weight matrices, once per CTA
    mbar_expect_tx(wbar, uint32_t(5 * FF_BOX));
    tma_load_2d(smem + FF_W1, &mapW1, 0, 0, wbar);
    tma_load_2d(smem + FF_W2, &mapW2, 0, 0, wbar);
    tma_load_2d(smem + FF_W2 + FF_BOX, &mapW2, BK, 0, wbar);
    tma_load_2d(smem + FF_W3, &mapW3, 0, 0, wbar);
    tma_load_2d(smem + FF_W3 + FF_BOX, &mapW3, BK, 0, wbar);
  }
  bool ok = __syncthreads_and(lbm::mbar_wait_bounded(wbar, 0u));
  uint32_t uses = 0;  // completed phases of this group's mbarrier
  // one layer: the group's A buffer is complete; one thread issues k_steps K = 16 MMAs of
  // A (sH) and B (weights) into the group's accumulator and commits them to its mbarrier
  auto mma_layer = [&](const uint8_t* sB, int k_steps) {
    lbm::fence_proxy_async_smem();  // this group's st.shared of A -> visible to the tensor cores
    lbm::tc_fence_before();
    (void)group_and(true, g);
    lbm::tc_fence_after();
    if (r == 0) {
      for (int j = 0; j < k_steps; ++j) {
        const int off = (j >> 2) * FF_BOX + 32 * (j & 3);
        lbm::tc_mma_f16(tmem_acc, smem_desc(sH + off), smem_desc(sB + off), kIdesc, j > 0 ? 1u : 0u);
      }
      lbm::tc_commit(mbar);
    }
    const bool done = lbm::mbar_wait_bounded(mbar, uses & 1u);
    ++uses;
    lbm::tc_fence_after();
    return group_and(done, g);
  };
  for (long long t = FF_GROUPS * (long long)blockIdx.x + g; ok && t < ntiles; t += FF_GROUPS * (long long)gridDim.x) {
    const long long m = t * 128 + r;  // this thread's row
    {  // normalised inputs, bfloat16, K = 16 (6 used)
      float a[8], b[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) a[j] = b[j] = 0.0f;
      if (m < n) {
#pragma unroll
        for (int j = 0; j < LBM_MLP_INPUTS; ++j) a[j] = (feat[m * LBM_MLP_INPUTS + j] - kCenter[j]) / kScale[j];
      }
      ff_store8(sH, r, 0, a);
      ff_store8(sH, r, 1, b);
    }
    float out = vec[512];
#pragma unroll 1
    for (int layer = 0; layer < 3; ++layer) {
      const uint8_t* sB = smem + (layer == 0 ? FF_W1 : (layer == 1 ? FF_W2 : FF_W3));
      if (!mma_layer(sB, layer == 0 ? 1 : 8)) {
        ok = false;
        break;
      }
      const float* bias = vec + 128 * layer;
#pragma unroll 1
      for (int cc = 0; cc < 4; ++cc) {  // columns 32 cc .. 32 cc + 31 of this row
        float v[32];
        lbm::tmem_ld32(tmem + uint32_t(32 * cc), v);
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = silu_fast(v[i] + bias[32 * cc + i]);
        if (layer < 2) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float piece[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) piece[i] = v[8 * q + i];
            ff_store8(sH, r, 4 * cc + q, piece);
          }
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i) out = fmaf(v[i], vec[384 + 32 * cc + i], out);
        }
      }
      // every read of the accumulator is complete before the group's next MMAs overwrite it
      lbm::tc_fence_before();
    }
    if (ok && m < n) y[m] = out;
  }
  if (!ok && r == 0) {
    atomicOr(status, lbm::STATUS_TIMEOUT);
    // the weight copies and this group's issued MMAs finish before the CTA goes (bounded)
    (void)lbm::mbar_wait_bounded(wbar, 0u, kWaitCycles / 8);
    lbm::tc_commit(mbar);
    (void)lbm::mbar_wait_bounded(mbar, uses & 1u, kWaitCycles / 8);
  }
  lbm::tc_fence_before();
  __syncthreads();
  if (warp == 0) lbm::tmem_dealloc(*tmem_slot, 128 * FF_GROUPS);
}

// ------------------------------------------------------------------ other kernels
__device__ __forceinline__ uint64_t splitmix64(uint64_t counter, uint64_t seed) {
  uint64_t z = seed + (counter + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// network inputs of Bc rows: rows < count take sample first + i (or a SplitMix64 draw when
// random), the rest are zero; X [Bc][16] and XT [16][Bc] bfloat16, targets FP32
__global__ void gather_kernel(const float* __restrict__ feat, const float* __restrict__ tgt, long long n,
                              long long first, int count, int random, unsigned long long seed, long long step,
                              int Bc, bf16* __restrict__ X, bf16* __restrict__ XT, float* __restrict__ tout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Bc) return;
  float x[KIN];
#pragma unroll
  for (int j = 0; j < KIN; ++j) x[j] = 0.0f;
  float t = 0.0f;
  if (i < count) {
    const long long idx =
        random ? (long long)(splitmix64((unsigned long long)step * (unsigned long long)count + i, seed) % (unsigned long long)n)
               : first + i;
#pragma unroll
    for (int j = 0; j < LBM_MLP_INPUTS; ++j) x[j] = (feat[idx * LBM_MLP_INPUTS + j] - kCenter[j]) / kScale[j];
    if (tgt) t = tgt[idx];
  }
#pragma unroll
  for (int j = 0; j < KIN; ++j) {
    const bf16 b = __float2bfloat16_rn(x[j]);
    X[size_t(i) * KIN + j] = b;
    XT[size_t(j) * Bc + i] = b;
  }
  if (tout) tout[i] = t;
}

// output layer y = silu(Z3) . w4 + b4; with train: loss, dy = 2 (y - t)/count, the
// gradients of w4, b4, b3 and dZ3 = dy w4 silu'(Z3) (bfloat16, [Bc][128] and [128][Bc])
__global__ void __launch_bounds__(128) head_kernel(const float* __restrict__ Z3, const float* __restrict__ P,
                                                   const float* __restrict__ tgt, int count, int Bc, int train,
                                                   float* __restrict__ y_out, float* __restrict__ grad,
                                                   double* __restrict__ loss, bf16* __restrict__ dZ,
                                                   bf16* __restrict__ dZT) {
  __shared__ float w4[W];
  for (int j = threadIdx.x; j < W; j += blockDim.x) w4[j] = P[OFF_W4 + j];
  __syncthreads();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;  // Bc is a multiple of 128: every thread has a row
  const int lane = threadIdx.x & 31;
  const float* z = Z3 + size_t(s) * W;
  float y = P[OFF_B4];
  for (int j = 0; j < W; ++j) y += silu_f(z[j]) * w4[j];
  const bool valid = s < count;
  if (!train) {
    if (valid) y_out[s] = y;
    return;
  }
  const float e = valid ? y - tgt[s] : 0.0f;
  const float dy = 2.0f * e / float(count);
  double e2 = double(e) * double(e);
#pragma unroll
  for (int o = 16; o; o >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, o);
  const float sdy = warp_sum_f(dy);
  if (lane == 0) {
    atomicAdd(loss, e2);
    atomicAdd(grad + OFF_B4, sdy);
  }
  for (int j = 0; j < W; ++j) {
    const float zj = z[j];
    const float dz = dy * w4[j] * dsilu_f(zj);
    const bf16 d = __float2bfloat16_rn(dz);
    dZ[size_t(s) * W + j] = d;
    dZT[size_t(j) * Bc + s] = d;
    const float a = warp_sum_f(dz), b = warp_sum_f(silu_f(zj) * dy);
    if (lane == 0) {
      atomicAdd(grad + OFF_B3 + j, a);
      atomicAdd(grad + OFF_W4 + j, b);
    }
  }
}

__global__ void adam_kernel(float* __restrict__ P, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float bc1,
                            float bc2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

// bfloat16 operand copies of the master weights: W1 [128][16], W2, W3 [out][in] and the
// transposes W2t, W3t [in][out]
__global__ void cast_kernel(const float* __restrict__ P, bf16* __restrict__ W1, bf16* __restrict__ W2,
                            bf16* __restrict__ W3, bf16* __restrict__ W2t, bf16* __restrict__ W3t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < W * KIN) W1[i] = __float2bfloat16_rn(P[OFF_W1 + i]);
  if (i < W * W) {
    const int o = i / W, k = i % W;
    const bf16 a = __float2bfloat16_rn(P[OFF_W2 + i]), b = __float2bfloat16_rn(P[OFF_W3 + i]);
    W2[i] = a;
    W3[i] = b;
    W2t[size_t(k) * W + o] = a;
    W3t[size_t(k) * W + o] = b;
  }
}

struct ColFeat {
  int ny;
  long long row_off;   // first row of this column in the concatenated row list
  long long node_off;  // first node of this column in the concatenated [col][y][x] fields
  float t, lg, form, mean;  // T/T_c, log10|g|, form, <rho>/rho_c (NaN: from rho)
  float lh;                 // log2 H
};

// raw features (T/T_c, log10|g|, form, <rho>/rho_c, z/H, log2 H) of every row of every column;
// with rho != NULL also the targets rho(y, x = 0)/rho_c and <rho> from rho itself
__global__ void features_kernel(const ColFeat* __restrict__ cols, int ncols, int nx, const double* __restrict__ rho,
                                double rho_c, float* __restrict__ feat, float* __restrict__ tgt) {
  const int c = blockIdx.x;
  if (c >= ncols) return;
  const ColFeat cf = cols[c];
  __shared__ double part[32];
  float mean = cf.mean;
  if (rho) {  // column mean of rho (every node)
    double s = 0.0;
    for (long long q = threadIdx.x; q < (long long)cf.ny * nx; q += blockDim.x) s += rho[cf.node_off + q];
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    double tot = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) tot += part[w];
    mean = float(tot / (double(cf.ny) * nx) / rho_c);
  }
  for (int y = threadIdx.x; y < cf.ny; y += blockDim.x) {
    float* f = feat + (cf.row_off + y) * LBM_MLP_INPUTS;
    f[0] = cf.t;
    f[1] = cf.lg;
    f[2] = cf.form;
    f[3] = mean;
    f[4] = (float(y) + 0.5f) / float(cf.ny);
    f[5] = cf.lh;
    if (rho && tgt) tgt[cf.row_off + y] = float(rho[cf.node_off + (long long)y * nx] / rho_c);
  }
}

// FP64 sum over the block (every thread gets it); red: 32 doubles of shared memory
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();  // red may still be read from the previous call
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double tot = 0.0;
  for (int w = 0; w < int(blockDim.x >> 5); ++w) tot += red[w];
  return tot;
}

// warm start: rho0 of column c = the predicted profile p(y) (times rho_c, floored at rho_min)
// moved along y by the shift s that gives the column's mass, the same on every x. The moved
// profile at row y is p at y - s, linear between rows and constant beyond the ends, so its
// mass M(s) runs from ny p(ny - 1) (s = -ny: the top value everywhere) to ny p(0) (s = ny);
// s follows by bisection on [-ny, ny] (60 halvings). Matching the mass by moving the
// profile keeps the predicted bulk densities: scaling it instead would change them by the
// relative mass error, a pressure error in the nearly incompressible liquid that excites
// the column's slowest mode. A mass outside that range (no bracket) keeps s = 0. A last
// factor M_target / M(s), within rounding of 1, makes the mass exact.
__global__ void warm_profile_kernel(const ColFeat* __restrict__ cols, int ncols, int nx, const float* __restrict__ yhat,
                                    const double* __restrict__ mean_rho, double rho_c, double rho_min,
                                    double* __restrict__ rho0) {
  const int c = blockIdx.x;
  if (c >= ncols) return;
  const ColFeat cf = cols[c];
  __shared__ double red[32];
  const int ny = cf.ny;
  auto prof = [&](int y) { return fmax(double(yhat[cf.row_off + y]) * rho_c, rho_min); };
  auto moved = [&](int y, double sh) {
    const double z = double(y) - sh;
    if (!(z > 0.0)) return prof(0);
    if (z >= double(ny - 1)) return prof(ny - 1);
    const int k = int(z);
    const double t = z - double(k);
    const double p0 = prof(k);
    return p0 + t * (prof(k + 1) - p0);
  };
  auto mass = [&](double sh) {
    double v = 0.0;
    for (int y = threadIdx.x; y < ny; y += blockDim.x) v += moved(y, sh);
    return block_sum(v, red);
  };
  const double target = mean_rho[c] * double(ny);
  double lo = -double(ny), hi = double(ny), sh = 0.0;
  if (mass(lo) <= target && target <= mass(hi)) {
    for (int it = 0; it < 60; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mass(mid) < target) lo = mid; else hi = mid;
    }
    sh = 0.5 * (lo + hi);
  }
  const double scale = target / mass(sh);
  for (long long q = threadIdx.x; q < (long long)ny * nx; q += blockDim.x) {
    const int y = int(q / nx);
    rho0[cf.node_off + q] = moved(y, sh) * scale;
  }
}

thread_local char g_err[512] = "";
int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  lbm::set_last_error(g_err);
  return code;
}

}  // namespace

// ------------------------------------------------------------------ handle
struct lbm_mlp {
  cudaStream_t stream = nullptr;
  int Bc = 0;  // batch capacity (multiple of 128)
  void* mem = nullptr;
  float *P = nullptr, *G = nullptr, *Mo = nullptr, *Vo = nullptr;
  bf16 *W1 = nullptr, *W2 = nullptr, *W3 = nullptr, *W2t = nullptr, *W3t = nullptr;
  bf16 *X = nullptr, *XT = nullptr, *H1 = nullptr, *H2 = nullptr, *H1T = nullptr, *H2T = nullptr;
  bf16 *dZa = nullptr, *dZb = nullptr, *dZTa = nullptr, *dZTb = nullptr;
  float *Z1 = nullptr, *Z2 = nullptr, *Z3 = nullptr, *tgt = nullptr, *y = nullptr;
  double* loss = nullptr;
  int* status = nullptr;
  long long adam_t = 0;
};

namespace {

#define MLP_CUDA(call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return fail(LBM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

cudaError_t gemm_prepare() {
  cudaError_t e = cudaSuccess;
  for (const void* fn : {(const void*)gemm_kernel<EPI_STORE>, (const void*)gemm_kernel<EPI_ATOMIC>,
                         (const void*)gemm_kernel<EPI_FWD>, (const void*)gemm_kernel<EPI_BWD>})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, FF_SMEM);
  return e;
}

// cuTensorMapEncodeTiled, looked up once through the runtime (no libcuda link)
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encoder() {
  static EncodeTiled fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

// 2-D map of a row-major bfloat16 matrix (rows x cols, ld elements per row) with a
// BK-element x 128-row box written with the 128-byte swizzle; reads outside the matrix
// fill zeros
bool make_map(CUtensorMap* m, const bf16* base, int rows, int cols, int ld) {
  EncodeTiled enc = encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {cuuint64_t(cols), cuuint64_t(rows)};
  const cuuint64_t strides[1] = {cuuint64_t(ld) * 2};
  const cuuint32_t box[2] = {BK, 128};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int EPI>
cudaError_t gemm(const GemmArgs& a, int splits, cudaStream_t s) {
  const dim3 grid((a.M + BM - 1) / BM, (a.N + BN - 1) / BN, splits);
  CUtensorMap mA, mB;
  if (!make_map(&mA, a.A, a.M, a.K, a.lda) || !make_map(&mB, a.B, a.N, a.K, a.ldb)) return cudaErrorInvalidValue;
  gemm_kernel<EPI><<<grid, GT, GEMM_SMEM, s>>>(mA, mB, a);
  return cudaGetLastError();
}

GemmArgs gargs(const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, int* status) {
  GemmArgs a{};
  a.A = A;
  a.lda = lda;
  a.B = B;
  a.ldb = ldb;
  a.M = M;
  a.N = N;
  a.K = K;
  a.k_split = (K + BK - 1) / BK * BK;
  a.status = status;
  return a;
}

int status_of(lbm_mlp* h) {
  int st = 0;
  MLP_CUDA(cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  MLP_CUDA(cudaStreamSynchronize(h->stream));
  if (st & lbm::STATUS_TIMEOUT) return fail(LBM_ETIMEOUT, "a tensor-core wait timed out");
  return LBM_OK;
}

// forward of rows [0, Bc) of X (count valid), then the head (train: loss and all gradients)
int run_pass(lbm_mlp* h, int count, bool train) {
  const int Bc = h->Bc;
  cudaStream_t s = h->stream;
  GemmArgs a = gargs(h->X, KIN, h->W1, KIN, Bc, W, KIN, h->status);
  a.bias = h->P + OFF_B1;
  a.Z = h->Z1;
  a.ldz = W;
  a.H = h->H1;
  a.ldh = W;
  a.HT = train ? h->H1T : nullptr;
  a.ldht = Bc;
  MLP_CUDA(gemm<EPI_FWD>(a, 1, s));
  a = gargs(h->H1, W, h->W2, W, Bc, W, W, h->status);
  a.bias = h->P + OFF_B2;
  a.Z = h->Z2;
  a.ldz = W;
  a.H = h->H2;
  a.ldh = W;
  a.HT = train ? h->H2T : nullptr;
  a.ldht = Bc;
  MLP_CUDA(gemm<EPI_FWD>(a, 1, s));
  a = gargs(h->H2, W, h->W3, W, Bc, W, W, h->status);
  a.bias = h->P + OFF_B3;
  a.Z = h->Z3;
  a.ldz = W;
  MLP_CUDA(gemm<EPI_FWD>(a, 1, s));
  if (train) {
    MLP_CUDA(cudaMemsetAsync(h->G, 0, sizeof(float) * NPARAM, s));
    MLP_CUDA(cudaMemsetAsync(h->loss, 0, sizeof(double), s));
  }
  head_kernel<<<Bc / 128, 128, 0, s>>>(h->Z3, h->P, h->tgt, count, Bc, train ? 1 : 0, h->y, h->G, h->loss, h->dZa,
                                       h->dZTa);
  MLP_CUDA(cudaGetLastError());
  if (!train) return LBM_OK;
  // weight gradients are sums over the batch (K = Bc): split K over CTAs, atomic epilogue
  const int ksplit = 1024, splits = (Bc + ksplit - 1) / ksplit;
  auto wgrad = [&](const bf16* dZT, const bf16* HTm, int N, float* C, int ldc) {
    GemmArgs w = gargs(dZT, Bc, HTm, Bc, W, N, Bc, h->status);
    w.k_split = ksplit;
    w.C = C;
    w.ldc = ldc;
    return gemm<EPI_ATOMIC>(w, splits, s);
  };
  auto dgrad = [&](const bf16* dZ, const bf16* Wt, const float* Z, bf16* dZo, bf16* dZTo, float* colsum) {
    GemmArgs d = gargs(dZ, W, Wt, W, Bc, W, W, h->status);
    d.Z = const_cast<float*>(Z);
    d.ldz = W;
    d.H = dZo;
    d.ldh = W;
    d.HT = dZTo;
    d.ldht = Bc;
    d.colsum = colsum;
    return gemm<EPI_BWD>(d, 1, s);
  };
  MLP_CUDA(wgrad(h->dZTa, h->H2T, W, h->G + OFF_W3, W));                          // dW3
  MLP_CUDA(dgrad(h->dZa, h->W3t, h->Z2, h->dZb, h->dZTb, h->G + OFF_B2));           // dZ2, db2
  MLP_CUDA(wgrad(h->dZTb, h->H1T, W, h->G + OFF_W2, W));                          // dW2
  MLP_CUDA(dgrad(h->dZb, h->W2t, h->Z1, h->dZa, h->dZTa, h->G + OFF_B1));           // dZ1, db1
  MLP_CUDA(wgrad(h->dZTa, h->XT, KIN, h->G + OFF_W1, KIN));                        // dW1
  return LBM_OK;
}

int cast_weights(lbm_mlp* h) {
  cast_kernel<<<(W * W + 255) / 256, 256, 0, h->stream>>>(h->P, h->W1, h->W2, h->W3, h->W2t, h->W3t);
  MLP_CUDA(cudaGetLastError());
  return LBM_OK;
}

int gather(lbm_mlp* h, const float* x, const float* t, long long n, long long first, int count, bool random,
           unsigned long long seed, long long step) {
  gather_kernel<<<h->Bc / 128, 128, 0, h->stream>>>(x, t, n, first, count, random ? 1 : 0, seed, step, h->Bc, h->X,
                                                   h->XT, h->tgt);
  MLP_CUDA(cudaGetLastError());
  return LBM_OK;
}

bool device_pointer(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int column_table(const lbm_column* cols, int ncols, int nx, double a, double b, double R, const double* mean_rho,
                 std::vector<ColFeat>& out, double* rho_c, long long* rows) {
  double rc, Tc, pc;
  if (lbm_critical_point(a, b, R, &rc, &Tc, &pc) != LBM_OK) return fail(LBM_EINVAL, "need a, b, R > 0");
  out.resize(ncols);
  long long r = 0, q = 0;
  for (int c = 0; c < ncols; ++c) {
    const lbm_column& in = cols[c];
    if (in.ny <= 0) return fail(LBM_EINVAL, "column %d has ny <= 0", c);
    const double gmag = std::sqrt(in.gx * in.gx + in.gy * in.gy);
    ColFeat& f = out[c];
    f.ny = in.ny;
    f.row_off = r;
    f.node_off = q;
    f.t = float(in.T / Tc);
    f.lg = float(gmag > 0 ? std::log10(gmag) : -12.0);
    f.form = float(in.gravity_form);
    f.mean = mean_rho ? float(mean_rho[c] / rc) : NAN;
    f.lh = float(std::log2(double(in.ny)));
    r += in.ny;
    q += (long long)in.ny * nx;
  }
  *rho_c = rc;
  *rows = r;
  return LBM_OK;
}

}  // namespace

// ================================================================== public ABI
extern "C" {

int lbm_mlp_create(const float* params, int batch_capacity, void* stream, lbm_mlp** out) {
  if (!params || !out) return fail(LBM_EINVAL, "params and out must not be NULL");
  if (batch_capacity < 128 || batch_capacity % 128 || batch_capacity > (1 << 22))
    return fail(LBM_EINVAL, "batch_capacity must be a multiple of 128 in [128, 4194304]");
  *out = nullptr;
  cudaError_t e = gemm_prepare();
  if (e != cudaSuccess) return fail(LBM_ECUDA, "kernel attributes: %s", cudaGetErrorString(e));
  lbm_mlp* h = new (std::nothrow) lbm_mlp();
  if (!h) return fail(LBM_ENOMEM, "out of host memory");
  h->stream = static_cast<cudaStream_t>(stream);
  h->Bc = batch_capacity;
  const size_t Bc = size_t(batch_capacity);
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t at = off; off = (off + bytes + 255) / 256 * 256; return at; };
  const size_t oP = take(4 * NPARAM), oG = take(4 * NPARAM), oM = take(4 * NPARAM), oV = take(4 * NPARAM);
  const size_t oW1 = take(2 * W * KIN), oW2 = take(2 * W * W), oW3 = take(2 * W * W), oW2t = take(2 * W * W),
               oW3t = take(2 * W * W);
  const size_t oX = take(2 * Bc * KIN), oXT = take(2 * Bc * KIN);
  const size_t oH1 = take(2 * Bc * W), oH2 = take(2 * Bc * W), oH1T = take(2 * Bc * W), oH2T = take(2 * Bc * W);
  const size_t odZa = take(2 * Bc * W), odZb = take(2 * Bc * W), odZTa = take(2 * Bc * W), odZTb = take(2 * Bc * W);
  const size_t oZ1 = take(4 * Bc * W), oZ2 = take(4 * Bc * W), oZ3 = take(4 * Bc * W);
  const size_t oT = take(4 * Bc), oY = take(4 * Bc), oL = take(8), oS = take(4);
  e = cudaMalloc(&h->mem, off);
  if (e != cudaSuccess) {
    delete h;
    return fail(LBM_ENOMEM, "cudaMalloc %zu bytes: %s", off, cudaGetErrorString(e));
  }
  char* base = static_cast<char*>(h->mem);
  h->P = reinterpret_cast<float*>(base + oP);
  h->G = reinterpret_cast<float*>(base + oG);
  h->Mo = reinterpret_cast<float*>(base + oM);
  h->Vo = reinterpret_cast<float*>(base + oV);
  h->W1 = reinterpret_cast<bf16*>(base + oW1);
  h->W2 = reinterpret_cast<bf16*>(base + oW2);
  h->W3 = reinterpret_cast<bf16*>(base + oW3);
  h->W2t = reinterpret_cast<bf16*>(base + oW2t);
  h->W3t = reinterpret_cast<bf16*>(base + oW3t);
  h->X = reinterpret_cast<bf16*>(base + oX);
  h->XT = reinterpret_cast<bf16*>(base + oXT);
  h->H1 = reinterpret_cast<bf16*>(base + oH1);
  h->H2 = reinterpret_cast<bf16*>(base + oH2);
  h->H1T = reinterpret_cast<bf16*>(base + oH1T);
  h->H2T = reinterpret_cast<bf16*>(base + oH2T);
  h->dZa = reinterpret_cast<bf16*>(base + odZa);
  h->dZb = reinterpret_cast<bf16*>(base + odZb);
  h->dZTa = reinterpret_cast<bf16*>(base + odZTa);
  h->dZTb = reinterpret_cast<bf16*>(base + odZTb);
  h->Z1 = reinterpret_cast<float*>(base + oZ1);
  h->Z2 = reinterpret_cast<float*>(base + oZ2);
  h->Z3 = reinterpret_cast<float*>(base + oZ3);
  h->tgt = reinterpret_cast<float*>(base + oT);
  h->y = reinterpret_cast<float*>(base + oY);
  h->loss = reinterpret_cast<double*>(base + oL);
  h->status = reinterpret_cast<int*>(base + oS);
  int rc = lbm_mlp_set_params(h, params);
  if (rc) {
    lbm_mlp_destroy(h);
    return rc;
  }
  *out = h;
  return LBM_OK;
}

int lbm_mlp_set_params(lbm_mlp* h, const float* params) {
  if (!h || !params) return fail(LBM_EINVAL, "handle and params must not be NULL");
  MLP_CUDA(cudaMemcpyAsync(h->P, params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, h->stream));
  MLP_CUDA(cudaMemsetAsync(h->Mo, 0, sizeof(float) * NPARAM, h->stream));
  MLP_CUDA(cudaMemsetAsync(h->Vo, 0, sizeof(float) * NPARAM, h->stream));
  MLP_CUDA(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
  h->adam_t = 0;
  int rc = cast_weights(h);
  if (rc) return rc;
  MLP_CUDA(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

int lbm_mlp_get_params(lbm_mlp* h, float* params) {
  if (!h || !params) return fail(LBM_EINVAL, "handle and params must not be NULL");
  MLP_CUDA(cudaMemcpyAsync(params, h->P, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, h->stream));
  MLP_CUDA(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

int lbm_mlp_gradients(lbm_mlp* h, const float* x, const float* t, int n, float* grads, double* loss) {
  if (!h || !x || !t || !grads) return fail(LBM_EINVAL, "handle, x, t and grads must not be NULL");
  if (n < 1 || n > h->Bc) return fail(LBM_EINVAL, "n must be in [1, batch_capacity]");
  if (!device_pointer(x) || !device_pointer(t)) return fail(LBM_EINVAL, "x and t must be device pointers");
  int rc = gather(h, x, t, n, 0, n, false, 0, 0);
  if (!rc) rc = run_pass(h, n, true);
  if (rc) return rc;
  MLP_CUDA(cudaMemcpyAsync(grads, h->G, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, h->stream));
  double l = 0.0;
  MLP_CUDA(cudaMemcpyAsync(&l, h->loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  rc = status_of(h);
  if (loss) *loss = l / n;
  return rc;
}

int lbm_mlp_train(lbm_mlp* h, const float* x, const float* t, long long n, int batch, int iters, float lr,
                  unsigned long long seed, float* losses) {
  if (!h || !x || !t) return fail(LBM_EINVAL, "handle, x and t must not be NULL");
  if (n < 1 || batch < 1 || batch > h->Bc || iters < 0 || !(lr > 0))
    return fail(LBM_EINVAL, "need n >= 1, 1 <= batch <= batch_capacity, iters >= 0, lr > 0");
  if (!device_pointer(x) || !device_pointer(t)) return fail(LBM_EINVAL, "x and t must be device pointers");
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int it = 0; it < iters; ++it) {
    int rc = gather(h, x, t, n, 0, batch, true, seed, h->adam_t);
    if (!rc) rc = run_pass(h, batch, true);
    if (rc) return rc;
    ++h->adam_t;
    const float bc1 = 1.0f - std::pow(b1, float(h->adam_t)), bc2 = 1.0f - std::pow(b2, float(h->adam_t));
    adam_kernel<<<(NPARAM + 255) / 256, 256, 0, h->stream>>>(h->P, h->G, h->Mo, h->Vo, NPARAM, lr, b1, b2, eps, bc1,
                                                             bc2);
    MLP_CUDA(cudaGetLastError());
    rc = cast_weights(h);
    if (rc) return rc;
    if (losses) {
      double l = 0.0;
      MLP_CUDA(cudaMemcpyAsync(&l, h->loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      MLP_CUDA(cudaStreamSynchronize(h->stream));
      losses[it] = float(l / batch);
    }
  }
  return status_of(h);
}

int lbm_mlp_predict(lbm_mlp* h, const float* x, long long n, float* y) {
  if (!h || !x || !y) return fail(LBM_EINVAL, "handle, x and y must not be NULL");
  if (n < 0) return fail(LBM_EINVAL, "n must be >= 0");
  if (!device_pointer(x) || !device_pointer(y)) return fail(LBM_EINVAL, "x and y must be device pointers");
  if (n == 0) return LBM_OK;
  // the fused forward kernel: one persistent CTA per SM at most, four 128-row tiles in flight each
  CUtensorMap m1, m2, m3;
  if (!make_map(&m1, h->W1, W, KIN, KIN) || !make_map(&m2, h->W2, W, W, W) || !make_map(&m3, h->W3, W, W, W))
    return fail(LBM_ECUDA, "tensor maps of the weights");
  int dev = 0, nsm = 0;
  MLP_CUDA(cudaGetDevice(&dev));
  MLP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const long long ntiles = (n + 127) / 128;
  const int grid = int(std::min<long long>(nsm, (ntiles + FF_GROUPS - 1) / FF_GROUPS));
  mlp_forward_kernel<<<grid, FF_THREADS, FF_SMEM, h->stream>>>(m1, m2, m3, h->P, x, n, y, h->status);
  MLP_CUDA(cudaGetLastError());
  return status_of(h);
}

int lbm_mlp_features(const lbm_column* cols, int ncols, int nx, double a, double b, double R, const double* rho,
                     const double* mean_rho, float* x, float* t, void* stream) {
  if (!cols || ncols < 1 || nx < 1 || !x) return fail(LBM_EINVAL, "cols, ncols >= 1, nx >= 1 and x are required");
  if (!rho && !mean_rho) return fail(LBM_EINVAL, "one of rho (device) and mean_rho (host) is required");
  if (!device_pointer(x) || (t && !device_pointer(t)) || (rho && !device_pointer(rho)))
    return fail(LBM_EINVAL, "x, t and rho must be device pointers");
  std::vector<ColFeat> tab;
  double rho_c;
  long long rows;
  int rc = column_table(cols, ncols, nx, a, b, R, rho ? nullptr : mean_rho, tab, &rho_c, &rows);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ColFeat* dtab = nullptr;
  MLP_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&dtab), sizeof(ColFeat) * ncols, s));
  cudaError_t e = cudaMemcpyAsync(dtab, tab.data(), sizeof(ColFeat) * ncols, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    features_kernel<<<ncols, 256, 0, s>>>(dtab, ncols, nx, rho, rho_c, x, t);
    e = cudaGetLastError();
  }
  cudaFreeAsync(dtab, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(LBM_ECUDA, "features: %s", cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_mlp_warm_start(lbm_mlp* h, const lbm_column* cols, int ncols, int nx, double a, double b, double R,
                       const double* mean_rho, double* rho0) {
  if (!h || !cols || ncols < 1 || nx < 1 || !mean_rho || !rho0)
    return fail(LBM_EINVAL, "handle, cols, ncols >= 1, nx >= 1, mean_rho and rho0 are required");
  if (!device_pointer(rho0)) return fail(LBM_EINVAL, "rho0 must be a device pointer");
  std::vector<ColFeat> tab;
  double rho_c;
  long long rows;
  int rc = column_table(cols, ncols, nx, a, b, R, mean_rho, tab, &rho_c, &rows);
  if (rc) return rc;
  cudaStream_t s = h->stream;
  char* mem = nullptr;
  const size_t b_tab = (sizeof(ColFeat) * ncols + 255) / 256 * 256, b_mean = (8 * size_t(ncols) + 255) / 256 * 256;
  const size_t b_feat = (4 * LBM_MLP_INPUTS * size_t(rows) + 255) / 256 * 256;
  MLP_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&mem), b_tab + b_mean + b_feat + 4 * size_t(rows), s));
  ColFeat* dtab = reinterpret_cast<ColFeat*>(mem);
  double* dmean = reinterpret_cast<double*>(mem + b_tab);
  float* feat = reinterpret_cast<float*>(mem + b_tab + b_mean);
  float* yhat = reinterpret_cast<float*>(mem + b_tab + b_mean + b_feat);
  cudaError_t e = cudaMemcpyAsync(dtab, tab.data(), sizeof(ColFeat) * ncols, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dmean, mean_rho, 8 * size_t(ncols), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    features_kernel<<<ncols, 256, 0, s>>>(dtab, ncols, nx, nullptr, rho_c, feat, nullptr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) rc = lbm_mlp_predict(h, feat, rows, yhat);
  if (e == cudaSuccess && rc == LBM_OK) {
    // floor: a tenth of the smallest coexistence vapour density the inputs cover
    warm_profile_kernel<<<ncols, 256, 0, s>>>(dtab, ncols, nx, yhat, dmean, rho_c, 1e-3, rho0);
    e = cudaGetLastError();
  }
  cudaFreeAsync(mem, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(LBM_ECUDA, "warm start: %s", cudaGetErrorString(e));
  return rc;
}

namespace {
// checks of lbm_mlp_gemm / lbm_mlp_gemm_enqueue, then the launch on stream s
int gemm_launch(const uint16_t* A, int lda, const uint16_t* B, int ldb, float* C, int ldc, int M, int N, int K,
                int k_split, int accumulate, int* status, cudaStream_t s) {
  if (!A || !B || !C || M < 1 || N < 1 || K < 16 || K % 16) return fail(LBM_EINVAL, "need M, N >= 1 and K a multiple of 16");
  if (lda % 8 || ldb % 8 || lda < K || ldb < K || ldc < N) return fail(LBM_EINVAL, "lda, ldb multiples of 8 and >= K; ldc >= N");
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15) return fail(LBM_EINVAL, "A and B 16-byte aligned");
  if (k_split <= 0) k_split = K;
  if (k_split % BK && k_split < K) return fail(LBM_EINVAL, "k_split must be a multiple of 64");
  if (!accumulate && k_split < K) return fail(LBM_EINVAL, "split K needs accumulate");
  cudaError_t e = gemm_prepare();
  if (e != cudaSuccess) return fail(LBM_ECUDA, "kernel attributes: %s", cudaGetErrorString(e));
  GemmArgs a = gargs(reinterpret_cast<const bf16*>(A), lda, reinterpret_cast<const bf16*>(B), ldb, M, N, K, status);
  a.k_split = std::min(K, (k_split + BK - 1) / BK * BK);
  a.C = C;
  a.ldc = ldc;
  const int splits = (K + a.k_split - 1) / a.k_split;
  e = accumulate ? gemm<EPI_ATOMIC>(a, splits, s) : gemm<EPI_STORE>(a, 1, s);
  if (e != cudaSuccess) return fail(LBM_ECUDA, "gemm: %s", cudaGetErrorString(e));
  return LBM_OK;
}
}  // namespace

int lbm_mlp_gemm(const uint16_t* A, int lda, const uint16_t* B, int ldb, float* C, int ldc, int M, int N, int K,
                 int k_split, int accumulate, void* stream) {
  int* status = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  MLP_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&status), sizeof(int), s));
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);
  int rc = e == cudaSuccess ? gemm_launch(A, lda, B, ldb, C, ldc, M, N, K, k_split, accumulate, status, s)
                            : fail(LBM_ECUDA, "gemm: %s", cudaGetErrorString(e));
  int st = 0;
  if (rc == LBM_OK) e = cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(status, s);
  const cudaError_t es = cudaStreamSynchronize(s);
  if (rc != LBM_OK) return rc;
  if (e == cudaSuccess) e = es;
  if (e != cudaSuccess) return fail(LBM_ECUDA, "gemm: %s", cudaGetErrorString(e));
  if (st & lbm::STATUS_TIMEOUT) return fail(LBM_ETIMEOUT, "a tensor-core wait timed out");
  return LBM_OK;
}

int lbm_mlp_gemm_enqueue(const uint16_t* A, int lda, const uint16_t* B, int ldb, float* C, int ldc, int M, int N,
                         int K, int k_split, int accumulate, int* status, void* stream) {
  if (!status || reinterpret_cast<uintptr_t>(status) % alignof(int)) return fail(LBM_EINVAL, "status: an aligned device int");
  return gemm_launch(A, lda, B, ldb, C, ldc, M, N, K, k_split, accumulate, status, static_cast<cudaStream_t>(stream));
}

int lbm_mlp_destroy(lbm_mlp* h) {
  if (!h) return LBM_OK;
  int rc = LBM_OK;
  if (h->mem) {
    cudaStreamSynchronize(h->stream);
    if (cudaFree(h->mem) != cudaSuccess) rc = LBM_ECUDA;
  }
  delete h;
  return rc;
}

}  // extern "C"
