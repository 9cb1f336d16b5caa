#pragma once
// Surrogate forward pass on the 5th-generation tensor cores (tcgen05 + TMEM):
// logits of the MLP 9 -> 256 -> 256 -> 256 -> 1 (SiLU) with BF16 operands and
// FP32 accumulation, rounded at the same points as the training forward pass
// (standardised input, every SiLU output and the weight copies in bf16;
// biases FP32), for the learned reachability gate of Sec. IV-E. The SiLU uses
// the SFU's tanh (see silu_f).
//
// One persistent CTA of 8 warps per SM works through tiles of 128 rows:
//   layer 1  A = features [128 x 16],  B = W1 [256 x 16]   -> TMEM D [128 x 256] f32
//   layer 2  A = h1 [128 x 256],       B = W2 [256 x 256]  -> TMEM D
//   layer 3  A = h2,                   B = W3              -> TMEM D
// D row i lives in TMEM lane i. Warp w reads lanes 32 (w % 4) .. + 31 and
// columns 128 (w / 4) .. + 127 (tcgen05.ld), adds the bias, applies SiLU,
// rounds to bf16 and writes the next layer's A operand; after layer 3 it
// forms its half of W4 . h3 and the two halves are summed through shared
// memory. Operands sit in shared memory in the canonical no-swizzle K-major
// layout of core matrices (8 rows x 16 bytes): core matrices adjacent in K are
// 128 bytes apart (leading byte offset), 8-row groups K / 8 * 128 bytes apart
// (stride byte offset). W2 and W3 arrive by 1-D bulk copies (cp.async.bulk)
// from weight copies kept in that layout, the copy of the next weights
// overlapping the current epilogue. One thread issues the MMAs and commits
// them to an mbarrier. Every wait is bounded: on timeout the CTA latches
// kDevTimeout, waits (bounded) for its own copies and MMAs still in flight,
// frees TMEM and returns.
//
// Core of the tensor-core surrogate forward pass (tcgen05 + TMEM), templated
// on where its rows come from and where their logits go; included by the
// plain inference (mlp_tc.cu) and by the generation loop's fused gate.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace sc {

namespace {

constexpr int H = 256;
constexpr int TILE = 128;
constexpr int THREADS = 256;  // the training kernels' CTA; the forward pass takes 128 x IO::kColGroups
// Shared memory of the inference kernel (two tiles in flight):
constexpr int PP_KS = 64;                             // inputs per streamed weight slice
constexpr int PP_SLICE = H * PP_KS * 2;               // 32 KB: PP_KS inputs of all 256 outputs
constexpr int PP_RING = 2;                            // weight slices in flight
constexpr int SM_A = 0;                               // [2 slots][128][256] bf16 canonical operands
constexpr int SM_WR = SM_A + 2 * TILE * H * 2;        // the weight slice ring
constexpr int SM_W1 = SM_WR + PP_RING * PP_SLICE;     // [256][16] bf16 canonical, 8 KB
constexpr int SM_BIAS = SM_W1 + 8192;                 // b1 b2 b3 W4 as f32, 4 KB
constexpr int SM_PART = SM_BIAS + 4 * H * 4;          // [2 slots][3][128] partial logits of column groups 1..3
constexpr int SM_BAR = SM_PART + 2 * 3 * TILE * 4;    // mbarriers: ring full, ring empty, accumulator full, operand ready
constexpr int SM_NBAR = 2 * PP_RING + 4 + 1;          // ... and the MMA drain
constexpr int SM_FLAG = SM_BAR + 8 * SM_NBAR;         // abort flag
constexpr int SM_TMEM = SM_FLAG + 16;                 // TMEM base address written by tcgen05.alloc
constexpr int SM_TOTAL = SM_TMEM + 16;
static_assert(SM_TOTAL <= 227 * 1024, "shared memory of one CTA");
constexpr long long kWaitCycles = 4000000000LL;  // about 2 s at 2 GHz per wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start, leading and stride byte offsets
// (all >> 4), descriptor version 1, base offset 0, no swizzle.
__device__ __forceinline__ uint64_t make_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: D f32 (bits 4-5 = 1), A and B bf16
// (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17,
// M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Waits until the phase with parity `parity` of the mbarrier has completed;
// false when the cycle budget runs out first.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

// As mbar_wait, but also gives up at once when another role of the CTA has
// set *abort, and sets it when its own cycle budget runs out.
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t bar, uint32_t parity, volatile int* abort) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (*abort) return false;
    if (clock64() - t0 > kWaitCycles) {
      *abort = 1;
      return false;
    }
  }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

// Arrives on `bar` once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// Global -> shared bulk copy of `bytes` (a multiple of 16; 16-byte aligned
// ends) in 32 KB pieces, completing on `bar` (one arrival + the byte count).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  for (uint32_t off = 0; off < bytes; off += 32768) {
    const uint32_t n = bytes - off < 32768 ? bytes - off : 32768;
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst + off),
        "l"(static_cast<const char*>(src) + off), "r"(n), "r"(bar)
        : "memory");
  }
}

// 32 consecutive f32 columns of this thread's TMEM lane, without waiting
// (tmem_wait_ld completes every load issued before it).
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t r[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 32 consecutive f32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t r[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// SiLU a sigma(a) through the identity sigma(a) = (1 + tanh(a / 2)) / 2:
// silu(a) = h + h tanh(h), h = a / 2, with the special-function unit's
// tanh (tanh.approx.f32, relative error about 2^-11): one SFU operation per
// activation instead of an exponential and a reciprocal, on the path where
// the SFU sets the pace. The absolute error, below 2.5e-4 |a|, is under the
// bf16 rounding of the stored activation for a > -2 and of the order of the
// bf16 spacing of unit activations below that.
__device__ __forceinline__ float tanh_sfu(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float silu_f(float a) {
  const float h = 0.5f * a;
  return fmaf(h, tanh_sfu(h), h);
}
// The logistic for training, which also keeps SiLU'(a) = s (1 + a (1 - s)):
// the SFU's approximate exponential and reciprocal (relative error ~1e-6).
__device__ __forceinline__ float sigmoid_f(float a) { return __fdividef(1.f, 1.f + __expf(-a)); }
__device__ __forceinline__ float silu_grad_from(float a, float s) { return s * fmaf(a, 1.f - s, 1.f); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}


// Epilogue of layers 1 and 2 for one thread's row and its CW columns:
// TMEM -> + bias -> SiLU -> bf16 -> next A operand (canonical, K = 256); the
// next 32 columns are loaded from TMEM while the current ones are computed.
template <int CW>
__device__ __forceinline__ void epilogue_to_a(uint32_t taddr, const float* bias, uint8_t* sa, int row, int col0) {
  uint32_t r[2][32];
  tmem_ld32_async(taddr, r[0]);
  tmem_wait_ld();
#pragma unroll
  for (int c0 = 0; c0 < CW; c0 += 32) {
    const int cur = (c0 / 32) & 1;
    if (c0 + 32 < CW) tmem_ld32_async(taddr + c0 + 32, r[cur ^ 1]);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t w[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = col0 + c0 + q * 8 + 2 * j;
        const float p0 = __uint_as_float(r[cur][q * 8 + 2 * j]) + bias[c];
        const float p1 = __uint_as_float(r[cur][q * 8 + 2 * j + 1]) + bias[c + 1];
        w[j] = pack_bf16(silu_f(p0), silu_f(p1));
      }
      *reinterpret_cast<uint4*>(sa + canon_offset(row, col0 + c0 + q * 8, H)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    if (c0 + 32 < CW) tmem_wait_ld();
  }
}

// IO supplies the rows: rows() (the row count, read once), features(row, f)
// (the 9 raw features of a row < rows(), called by one thread per row) and
// emit(row, valid, logit) (called by every thread of warps 0..3, one row
// each, valid = row < rows(), so warp collectives may be used), and
// IO::kColGroups (2 or 4): 4 x kColGroups epilogue warps, warp w handling
// TMEM lanes 32 (w % 4) .. + 31 and columns (w / 4) H / kColGroups .. (more
// warps hide more of the epilogue's latency; fewer leave room on the SM for
// other kernels).
//
// One persistent CTA per SM keeps two of its tiles in flight, each in its
// own slot (a 64 KB operand buffer and 256 TMEM columns), so the tensor
// cores work on one slot while the epilogue warps work on the other: the
// epilogues go slot 0 layer 1, slot 1 layer 1, slot 0 layer 2, ... and the
// MMAs of a slot's next layer run under the other slot's epilogue. W2 and W3
// do not fit beside two operands, so one producer thread streams them
// through a ring of K-slices (64 inputs of all 256 outputs, 32 KB each, from
// the K-sliced weight copies) in the order one MMA thread consumes them, four
// M = 128, N = 256, K = 16 MMAs per slice; W1 stays resident. Roles meet on mbarriers: slice full (bulk
// copy) and empty (MMA commit), accumulator full (MMA commit), operand
// ready (every epilogue warp has written its part and finished its TMEM
// reads). Every wait is bounded; a role whose wait gives up sets a shared
// abort flag that ends the others' waits, and the CTA then latches
// kDevTimeout, waits (bounded) for its own copies and MMAs and frees TMEM.
template <class IO>
__global__ void __launch_bounds__(128 * IO::kColGroups + 64, 1) mlp_tc_kernel(MlpTcWeights w, IO io, int* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr int CG = IO::kColGroups, NE = 128 * CG, NT = NE + 64, CW = H / CG;
  static_assert(CG == 2 || CG == 4, "two or four column groups");
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = io.rows();
  const int ntiles = (n + TILE - 1) / TILE;
  if ((int)blockIdx.x >= ntiles) return;  // uniform for the CTA, before any allocation
  const int T = (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1;  // tiles blockIdx.x + i gridDim.x, i < T

  const uint32_t s0 = smem_u32(smem);
  float* sbias = reinterpret_cast<float*>(smem + SM_BIAS);  // b1 | b2 | b3 | W4
  float* spart = reinterpret_cast<float*>(smem + SM_PART);
  const uint32_t bar_full = s0 + SM_BAR, bar_empty = bar_full + 8 * PP_RING;
  const uint32_t bar_acc = bar_empty + 8 * PP_RING, bar_ready = bar_acc + 16, bar_drain = bar_ready + 16;
  volatile int* abort = reinterpret_cast<volatile int*>(smem + SM_FLAG);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + SM_TMEM);

  if (tid == 0) {
    for (int i = 0; i < PP_RING; ++i) {
      mbar_init(bar_full + 8 * i, 1);
      mbar_init(bar_empty + 8 * i, 1);
    }
    for (int p = 0; p < 2; ++p) {
      mbar_init(bar_acc + 8 * p, 1);
      mbar_init(bar_ready + 8 * p, NE / 32);
    }
    mbar_init(bar_drain, 1);
    *abort = 0;
  }
  for (int i = tid; i < 8192 / 16; i += NT)
    reinterpret_cast<uint4*>(smem + SM_W1)[i] = __ldg(reinterpret_cast<const uint4*>(w.W1c) + i);
  for (int i = tid; i < H; i += NT) {
    sbias[i] = __ldg(w.params + w.off_b1 + i);
    sbias[H + i] = __ldg(w.params + w.off_b2 + i);
    sbias[2 * H + i] = __ldg(w.params + w.off_b3 + i);
    sbias[3 * H + i] = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(w.W4)[i]);
  }
  const float b4 = __ldg(w.params + w.off_b4);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(2 * H)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_proxy_async();
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;  // slot p: columns 256 p .. + 255
  int issued = 0;                 // weight slices the producer issued (its thread only)

  if (warp < NE / 32) {
    // ---- epilogue warps
    const int quarter = warp & 3, cg = warp >> 2;
    const int trow = quarter * 32 + lane;  // this thread's row in the tile (= TMEM lane)
    const int col0 = cg * CW;              // this thread's columns
    // tile i's layer-1 operand (standardised features, bf16, K padded to 16)
    // into slot p, one row per thread of warps 0..3
    auto features = [&](int p, int i) {
      if (cg != 0) return;
      const int row = ((int)blockIdx.x + i * (int)gridDim.x) * TILE + trow;
      float x[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) x[k] = 0.f;
      if (row < n) {
        float f[9];
        io.features(row, f);
#pragma unroll
        for (int k = 0; k < 9; ++k) x[k] = (f[k] - __ldg(w.mu + k)) * __ldg(w.inv_sigma + k);
      }
      uint32_t xb[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) xb[k] = pack_bf16(x[2 * k], x[2 * k + 1]);
      uint8_t* sa = smem + SM_A + p * (TILE * H * 2);
#pragma unroll
      for (int q = 0; q < 2; ++q)
        *reinterpret_cast<uint4*>(sa + canon_offset(trow, q * 8, 16)) =
            make_uint4(xb[4 * q], xb[4 * q + 1], xb[4 * q + 2], xb[4 * q + 3]);
    };
    // this warp's part of slot p's operand is written and its TMEM reads are done
    auto ready = [&](int p) {
      fence_proxy_async();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_ready + 8 * p);
    };
    bool ok = true;
    uint32_t ph_acc[2] = {0u, 0u};
    for (int p = 0; p < 2 && p < T; ++p) {
      features(p, p);
      ready(p);
    }
    for (int i0 = 0; i0 < T && ok; i0 += 2)
      for (int layer = 0; layer < 3 && ok; ++layer)
        for (int p = 0; p < 2; ++p) {
          const int i = i0 + p;
          if (i >= T) break;
          ok = mbar_wait_or_abort(bar_acc + 8 * p, ph_acc[p], abort);
          if (!ok) break;
          ph_acc[p] ^= 1;
          tc_fence_after();
          const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(H * p + col0);
          uint8_t* sa = smem + SM_A + p * (TILE * H * 2);
          if (layer < 2) {
            epilogue_to_a<CW>(taddr, sbias + layer * H, sa, trow, col0);
            ready(p);
            continue;
          }
          // h3 = bf16(SiLU(acc + b3)); logit = W4 . h3 + b4
          const float* b3 = sbias + 2 * H + col0;
          const float* w4 = sbias + 3 * H + col0;
          float z = 0.f;
          uint32_t r[2][32];
          tmem_ld32_async(taddr, r[0]);
          tmem_wait_ld();
#pragma unroll
          for (int c0 = 0; c0 < CW; c0 += 32) {
            const int cur = (c0 / 32) & 1;
            if (c0 + 32 < CW) tmem_ld32_async(taddr + c0 + 32, r[cur ^ 1]);
#pragma unroll
            for (int j = 0; j < 32; j += 2) {
              const float p0 = __uint_as_float(r[cur][j]) + b3[c0 + j];
              const float p1 = __uint_as_float(r[cur][j + 1]) + b3[c0 + j + 1];
              const uint32_t hb = pack_bf16(silu_f(p0), silu_f(p1));
              z = fmaf(__uint_as_float(hb << 16), w4[c0 + j], z);
              z = fmaf(__uint_as_float(hb & 0xFFFF0000u), w4[c0 + j + 1], z);
            }
            if (c0 + 32 < CW) tmem_wait_ld();
          }
          float* sp = spart + p * 3 * TILE;
          if (cg > 0) sp[(cg - 1) * TILE + trow] = z;
          asm volatile("bar.sync 1, %0;" ::"r"(NE) : "memory");  // the column groups' partials (epilogue warps)
          // the next tile of this slot: its features, once this slot's TMEM is read
          if (i + 2 < T) features(p, i + 2);
          if (cg == 0) {  // column groups summed in order
#pragma unroll
            for (int g = 1; g < CG; ++g) z += sp[(g - 1) * TILE + trow];
            const int row = ((int)blockIdx.x + i * (int)gridDim.x) * TILE + trow;
            io.emit(row, row < n, z + b4);
          }
          if (i + 2 < T) ready(p);
        }
  } else if (warp == NE / 32) {
    // ---- producer: W2 and W3 slices, in the order the MMA thread takes them
    if (lane == 0) {
      bool ok = true;
      for (int i0 = 0; i0 < T && ok; i0 += 2)
        for (int layer = 1; layer < 3 && ok; ++layer)
          for (int p = 0; p < 2 && ok; ++p) {
            if (i0 + p >= T) break;
            const char* wl = static_cast<const char*>(layer == 1 ? w.W2k : w.W3k);
            for (int j = 0; j < H / PP_KS && ok; ++j) {
              const int r = issued % PP_RING;
              if (issued >= PP_RING)  // the MMAs that read this ring slot are done
                ok = mbar_wait_or_abort(bar_empty + 8 * r, (uint32_t)((issued / PP_RING - 1) & 1), abort);
              if (!ok) break;
              bulk_load(s0 + SM_WR + r * PP_SLICE, wl + (size_t)j * PP_SLICE, PP_SLICE, bar_full + 8 * r);
              ++issued;
            }
          }
    }
  } else {
    // ---- MMA thread
    if (lane == 0) {
      bool ok = true;
      int used = 0;
      uint32_t ph_ready[2] = {0u, 0u};
      for (int i0 = 0; i0 < T && ok; i0 += 2)
        for (int layer = 0; layer < 3 && ok; ++layer)
          for (int p = 0; p < 2 && ok; ++p) {
            if (i0 + p >= T) break;
            ok = mbar_wait_or_abort(bar_ready + 8 * p, ph_ready[p], abort);
            if (!ok) break;
            ph_ready[p] ^= 1;
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(H * p);
            const uint32_t a = s0 + SM_A + p * (TILE * H * 2);
            if (layer == 0) {
              tc_mma(d, make_desc(a, 128, 256), make_desc(s0 + SM_W1, 128, 256), make_idesc(TILE, H), 0);
            } else {
              for (int j = 0; j < H / PP_KS && ok; ++j, ++used) {
                const int r = used % PP_RING;
                ok = mbar_wait_or_abort(bar_full + 8 * r, (uint32_t)((used / PP_RING) & 1), abort);
                if (!ok) break;
                tc_fence_after();
                const uint32_t b = s0 + SM_WR + r * PP_SLICE;
#pragma unroll
                for (int k = 0; k < PP_KS / 16; ++k)
                  tc_mma(d, make_desc(a + (PP_KS / 16 * j + k) * 256, 128, 4096),
                         make_desc(b + 256 * k, 128, PP_KS / 8 * 128), make_idesc(TILE, H), (j > 0 || k > 0) ? 1u : 0u);
                tc_commit(bar_empty + 8 * r);
              }
            }
            if (ok) tc_commit(bar_acc + 8 * p);
          }
      // every MMA this thread issued has completed before TMEM is freed
      tc_commit(bar_drain);
      mbar_wait(bar_drain, 0);
    }
  }
  __syncthreads();
  if (*abort) {
    if (tid == 0) latch_error(status, kDevTimeout);
    if (warp == NE / 32 && lane == 0)  // this producer's copies have landed before the CTA leaves
      for (int u = issued > PP_RING ? issued - PP_RING : 0; u < issued; ++u)
        mbar_wait(bar_full + 8 * (u % PP_RING), (uint32_t)((u / PP_RING) & 1));
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * H) : "memory");
  }
}

}  // namespace

// Launches mlp_tc_kernel<IO> over at most n_cap rows (the kernel reads the
// actual count from io.rows()).
template <class IO>
cudaError_t launch_mlp_tc(const MlpTcWeights& w, const IO& io, int n_cap, int* status, int num_sms, cudaStream_t s) {
  if (n_cap <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(mlp_tc_kernel<IO>, cudaFuncAttributeMaxDynamicSharedMemorySize, SM_TOTAL);
  if (e) return e;
  const int tiles = (n_cap + TILE - 1) / TILE;
  const int grid = tiles < num_sms ? tiles : num_sms;
  mlp_tc_kernel<IO><<<grid, 128 * IO::kColGroups + 64, SM_TOTAL, s>>>(w, io, status);
  return cudaGetLastError();
}

}  // namespace sc
