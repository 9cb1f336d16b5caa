// Surrogate training on the 5th-generation tensor cores (tcgen05 + TMEM):
// one step of binary cross-entropy on logits for the learned reachability
// gate of Sec. IV-E, as three contractions per layer, all bf16 x bf16 -> f32
// in TMEM with operands in the canonical no-swizzle K-major layout:
//
//   forward   Z_l  = H_{l-1} W_l^T        mlp_train_fb_kernel, one cluster of
//   backward  dH_l = dA_{l+1} W_{l+1}     four CTAs per 128-row tile, each CTA
//             dA_l = bf16(dH_l * SiLU'(Z_l))   64 of the 256 features; B = W^T
//                                          copies in the backward pass
//   weights   dW_l = dA_l^T H_{l-1}       mlp_tc_wgrad_kernel: M = output
//   biases    db_l = dA_l^T 1             features (two 128-row tiles), N = input
//                                          features and a row of ones, K = the
//                                          batch split over the CTAs of a cluster,
//                                          the partials added in split order over
//                                          distributed shared memory
//
// Rounding points as in the FP64 reference: standardised input, SiLU outputs,
// weight copies, dL/dz before it meets W4 and every dL/da in bf16; biases,
// pre-activations, accumulations and gradients in FP32. Every mbarrier wait is
// bounded; on timeout the CTA latches kDevTimeout, drains its own copies and
// MMAs, frees TMEM and returns.
#include <cstring>

#include "mlp_adam.cuh"
#include "mlp_tc_core.cuh"

namespace sc {

namespace {

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float sigmoid_acc(float a) { return 1.f / (1.f + expf(-a)); }
__device__ __forceinline__ float bf16_lo(uint32_t x) { return __uint_as_float(x << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t x) { return __uint_as_float(x & 0xFFFF0000u); }

// ------------------------------------------- forward and backward, fused
//
// One 128-row tile per cluster of FB_CTAS CTAs. CTA rank j of the cluster owns
// hidden features [64 j, 64 j + 64) of every layer: its contractions are
// M = 128 (rows) x N = 64 (its features) x K = 256, with B = its 64-row slice
// of the weight copy (contiguous in the canonical layout). The A operands
// (h1, h2, dA3, dA2) are kept as four 16 KB blocks of 64 features, each in
// the canonical K-major layout with K = 64; a CTA writes its own block and
// sends it to the other CTAs of the cluster with one bulk shared-to-shared
// copy each (cp.async.bulk.shared::cluster), which completes on the
// receiver's mbarrier. Two operand buffers alternate, and a CTA sends the
// next layer's block only after it has received every block of the current
// one, so no block is overwritten while it is read. SiLU'(z) of the CTA's
// features stays in TMEM between the forward and the backward pass. The
// logit is the in-order sum of the four CTAs' partial dot products W4 . h3,
// exchanged the same way. Cluster barriers only bracket the kernel (every
// CTA has initialised its mbarriers before it is sent anything; none leaves
// while its copies may still be read), and every CTA passes both, whatever
// its bounded waits did.
constexpr int TS_LD = H + 2;  // per-tile sums: dW4 (256), db4, the BCE sum
constexpr int FB_CTAS = 4;
constexpr int FB_NS = H / FB_CTAS;                     // features per CTA
constexpr int FB_BLK = TILE * FB_NS * 2;               // one CTA's block of an operand, 16 KB
constexpr int FB_THREADS = 256;                        // 8 warps: TMEM lane quarter x 2 column halves
constexpr int FB_CW = FB_NS * TILE / FB_THREADS;       // 32 columns per thread
constexpr int FB_A0 = 0;                               // [4 blocks][128][64] bf16 operand, 64 KB
constexpr int FB_A1 = FB_A0 + FB_CTAS * FB_BLK;        // the other operand buffer
constexpr int FB_X = FB_A1 + FB_CTAS * FB_BLK;         // [128][16] bf16 canonical layer-1 operand
constexpr int FB_W1 = FB_X + TILE * 16 * 2;            // [64][16] slice of W1
constexpr int FB_WA = FB_W1 + FB_NS * 16 * 2;          // [64][256] slice of W2, then of W3^T
constexpr int FB_WB = FB_WA + FB_NS * H * 2;           // [64][256] slice of W3, then of W2^T
constexpr int FB_BIAS = FB_WB + FB_NS * H * 2;         // b1 b2 b3 W4 slices as f32
constexpr int FB_PART = FB_BIAS + 4 * FB_NS * 4;       // [FB_CTAS][128] partial logits
constexpr int FB_HALF = FB_PART + FB_CTAS * TILE * 4;  // [128] partial logit of column half 1
constexpr int FB_DZ = FB_HALF + TILE * 4;              // [128] bf16-rounded dz of the tile
constexpr int FB_DZF = FB_DZ + TILE * 4;               // [128] dz of the tile
constexpr int FB_RED = FB_DZF + TILE * 4;              // [4][64] partial sums of dW4
constexpr int FB_BAR = FB_RED + 4 * FB_NS * 4;         // 6 mbarriers
constexpr int FB_TMEM = FB_BAR + 48;
constexpr int FB_TOTAL = FB_TMEM + 16;
constexpr uint32_t FB_TCOLS = 4 * FB_NS;               // TMEM: accumulator, SiLU'(z1), SiLU'(z2), SiLU'(z3)
constexpr uint32_t FB_RECV = (FB_CTAS - 1) * FB_BLK;   // operand bytes received per layer
static_assert(FB_CW == 32, "one 32-column TMEM access per thread and epilogue");
static_assert(FB_TOTAL <= 227 * 1024, "shared memory of one CTA");

struct FbArgs {
  MlpTcWeights w;         // forward weights (W1c, W2c, W3c canonical [out][in]), biases, standardisation
  const void* W2tc;       // bf16 canonical [in][out]: B operand of dH1 = dA2 W2
  const void* W3tc;       // B operand of dH2 = dA3 W3
  const float* targets;
  const uint8_t* labels;  // [targets], through index
  const int32_t* index;   // batch row -> target / label (NULL: identity)
  int n;
  float inv_n;
  float* logits;          // [n]
  uint8_t* x16T;          // chunk-tiled (see below), 16 features: the standardised input and a row of ones
  uint8_t* hT[2];         // chunk-tiled, 256 features: h1, h2
  uint8_t* daT[3];        // chunk-tiled, 256 features: dL/da1, da2, da3
  float* dz;              // [n] dL/dz
  float* tsum;            // [tiles][TS_LD] over each tile's rows: dW4 = sum dz h3 (256), db4 = sum dz, the BCE sum
};

__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_shared_rank(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

// Programmatic dependent launch: the next kernel of the stream may be
// scheduled once every CTA of this one has signalled; griddep_wait blocks
// until the previous kernel has completed and its memory is visible (every
// global read or write of the training kernels comes after it).
__device__ __forceinline__ void griddep_signal() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// `bytes` at shared address `local` to the same address in every other CTA
// of the cluster, each copy completing on that CTA's mbarrier `bar` (one
// thread; the bytes were written before a proxy fence and a CTA barrier).
__device__ __forceinline__ void fb_send(uint32_t local, uint32_t bytes, uint32_t bar, uint32_t rank) {
#pragma unroll
  for (uint32_t r = 0; r < FB_CTAS; ++r) {
    if (r == rank) continue;
    asm volatile(
        "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            map_shared_rank(local, r)),
        "r"(local), "r"(bytes), "r"(map_shared_rank(bar, r))
        : "memory");
  }
}

// One arrival on `bar` that also expects `bytes` of copies for its phase.
__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t r[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
      "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
      "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// The weight gradients read the batch in 64-row chunks, so the caches they
// read are kept "chunk-tiled": chunk c holds rows [64 c, 64 c + 64) of every
// feature f in the canonical K-major layout with K = the 64 rows, at byte
// canon_offset(f, r % 64, 64) of a F x 128-byte tile (F = 256 or 16); the
// weight-gradient kernel stages a chunk with one bulk copy per operand.

// This CTA's 64-feature block of a 128-row tile (canonical, K = features)
// into the chunk-tiled layout, a core matrix per warp at a time: its 128
// contiguous bytes loaded as one 32-bit word per lane (row lane / 4,
// features 2 (lane % 4) and + 1), transposed across the warp
// (movmatrix.m8n8.trans), and stored as 128 contiguous bytes of the
// transposed core matrix (feature rows of 8 batch rows).
__device__ __forceinline__ void copy_out_tiled(const uint8_t* blk, uint8_t* dst, int tile, int fs, int warp,
                                               int lane) {
#pragma unroll 4
  for (int cm = warp; cm < (TILE / 8) * (FB_NS / 8); cm += FB_THREADS / 32) {
    const int rg = cm / (FB_NS / 8), kg = cm % (FB_NS / 8);  // rows 8 rg.., features 8 kg..
    const uint32_t v = *reinterpret_cast<const uint32_t*>(blk + rg * (FB_NS / 8) * 128 + kg * 128 + 4 * lane);
    uint32_t t;
    asm volatile("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;" : "=r"(t) : "r"(v));
    *reinterpret_cast<uint32_t*>(dst + (size_t)(2 * tile + (rg >> 3)) * (H * 128) + (size_t)(fs / 8 + kg) * 1024 +
                                 (rg & 7) * 128 + 4 * lane) = t;
  }
}

// The 16 MMAs (K = 16 each) of D[128 x 64] = A[128 x 256] B[64 x 256]^T, A
// in four 64-feature blocks, committed to `bar`; one thread.
__device__ __forceinline__ void fb_mma_k256(uint32_t tmem, uint32_t a, uint32_t b, uint32_t bar) {
  constexpr uint32_t idesc = make_idesc(TILE, FB_NS);
  tc_fence_after();
#pragma unroll 1
  for (int s = 0; s < H / 16; ++s)
    tc_mma(tmem, make_desc(a + (s >> 2) * FB_BLK + (s & 3) * 256, 128, FB_NS / 8 * 128),
           make_desc(b + 256 * s, 128, 4096), idesc, s > 0);
  tc_commit(bar);
}

// 32 bf16 values (16 packed pairs) of row `row`, block features [c0, c0 + 32),
// into the block at shared address `blk`.
__device__ __forceinline__ void fb_put_row(uint32_t blk, int row, int c0, const uint32_t hw[16]) {
#pragma unroll
  for (int q = 0; q < 4; ++q)
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(blk + canon_offset(row, c0 + 8 * q, FB_NS)),
                 "r"(hw[4 * q]), "r"(hw[4 * q + 1]), "r"(hw[4 * q + 2]), "r"(hw[4 * q + 3])
                 : "memory");
}

// Forward and backward of one 128-row tile, dz and the loss, for a cluster of
// FB_CTAS CTAs (see above). Writes the standardised input, h1, h2 and
// dA1..dA3 feature-major for the weight gradients, the logits, dz and the
// tile's sums of dz h3 and dz.
__global__ void __launch_bounds__(FB_THREADS, 1) mlp_train_fb_kernel(FbArgs A, int* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = A.n;
  const int row0 = (int)(blockIdx.x / FB_CTAS) * TILE;
  const uint32_t rank = cluster_ctarank();
  const int fs = (int)rank * FB_NS;  // first feature of this CTA
  float* sbias = reinterpret_cast<float*>(smem + FB_BIAS);  // b1 | b2 | b3 | W4 of this CTA's features
  float* spart = reinterpret_cast<float*>(smem + FB_PART);
  float* shalf = reinterpret_cast<float*>(smem + FB_HALF);
  float* sdz = reinterpret_cast<float*>(smem + FB_DZ);
  float* sdzf = reinterpret_cast<float*>(smem + FB_DZF);
  float* sred = reinterpret_cast<float*>(smem + FB_RED);
  const int tile = row0 / TILE;
  const uint32_t s0 = smem_u32(smem);
  const uint32_t bar_a = s0 + FB_BAR, bar_b = bar_a + 8, bar_m = bar_a + 16;  // weights, weights, MMAs
  const uint32_t bar_x0 = bar_a + 24, bar_x1 = bar_a + 32, bar_p = bar_a + 40;  // received: A0, A1, logits
  const uint32_t own0 = s0 + FB_A0 + rank * FB_BLK, own1 = s0 + FB_A1 + rank * FB_BLK;  // this CTA's blocks
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + FB_TMEM);
  const char* W2c = static_cast<const char*>(A.w.W2c) + (size_t)fs * H * 2;  // 64-row slices
  const char* W3c = static_cast<const char*>(A.w.W3c) + (size_t)fs * H * 2;
  const char* W2t = static_cast<const char*>(A.W2tc) + (size_t)fs * H * 2;
  const char* W3t = static_cast<const char*>(A.W3tc) + (size_t)fs * H * 2;

  if (tid == 0) {
    for (int i = 0; i < 6; ++i) mbar_init(bar_a + 8 * i, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  griddep_signal();
  griddep_wait();  // the previous step's weight update and its reads of the caches are done
  __syncthreads();
  // phases issued and completed on each mbarrier (the same in every thread)
  int iss_a = 1, iss_b = 1, iss_m = 0, iss_x0 = 1, iss_x1 = 1, iss_p = 1;
  int got_a = 0, got_b = 0, got_m = 0, got_x0 = 0, got_x1 = 0, got_p = 0;
  if (tid == 0) {
    mbar_expect(bar_x0, FB_RECV);
    mbar_expect(bar_x1, FB_RECV);
    mbar_expect(bar_p, (FB_CTAS - 1) * TILE * 4);
    bulk_load(s0 + FB_WA, W2c, FB_NS * H * 2, bar_a);
    bulk_load(s0 + FB_WB, W3c, FB_NS * H * 2, bar_b);
  }
  cluster_arrive();  // this CTA's mbarriers are ready for the others' copies
  for (int i = tid; i < FB_NS * 16 * 2 / 16; i += FB_THREADS)
    reinterpret_cast<uint4*>(smem + FB_W1)[i] =
        __ldg(reinterpret_cast<const uint4*>(static_cast<const char*>(A.w.W1c) + (size_t)fs * 16 * 2) + i);
  for (int i = tid; i < FB_NS; i += FB_THREADS) {
    sbias[i] = __ldg(A.w.params + A.w.off_b1 + fs + i);
    sbias[FB_NS + i] = __ldg(A.w.params + A.w.off_b2 + fs + i);
    sbias[2 * FB_NS + i] = __ldg(A.w.params + A.w.off_b3 + fs + i);
    sbias[3 * FB_NS + i] = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(A.w.W4)[fs + i]);
  }
  const float b4 = __ldg(A.w.params + A.w.off_b4);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(FB_TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // ---- layer-1 operand: standardised features, bf16, K padded to 16 (every
  // CTA forms all of it; rank 0 keeps it for dW1); each row's label
  float y = 0.f;
  if (tid < TILE) {
    const int row = row0 + tid;
    float x[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = 0.f;
    if (row < n) {
      const int ti = A.index ? __ldg(&A.index[row]) : row;
      const float* t = A.targets + 12 * (size_t)ti;
      const float f[9] = {__ldg(t + 9), __ldg(t + 10), __ldg(t + 11), __ldg(t + 0), __ldg(t + 3),
                          __ldg(t + 6), __ldg(t + 1), __ldg(t + 4), __ldg(t + 7)};
      y = __ldg(&A.labels[ti]) ? 1.f : 0.f;
#pragma unroll
      for (int i = 0; i < 9; ++i) x[i] = (f[i] - __ldg(A.w.mu + i)) * __ldg(A.w.inv_sigma + i);
    }
    uint32_t xb[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) xb[i] = pack_bf16(x[2 * i], x[2 * i + 1]);
#pragma unroll
    for (int q = 0; q < 2; ++q)
      *reinterpret_cast<uint4*>(smem + FB_X + canon_offset(tid, q * 8, 16)) =
          make_uint4(xb[4 * q], xb[4 * q + 1], xb[4 * q + 2], xb[4 * q + 3]);
    if (rank == 0) {  // the tile's two chunks of X, with input slot 9 = 1 on rows < n (bias gradients)
      uint16_t* xt = reinterpret_cast<uint16_t*>(A.x16T + (size_t)tile * 4096 + (tid >> 6) * 2048);
#pragma unroll
      for (int i = 0; i < 16; ++i)
        xt[canon_offset(i, tid & 63, 64) / 2] =
            i == 9 ? (row < n ? (uint16_t)0x3F80u : (uint16_t)0) : (uint16_t)(xb[i >> 1] >> (16 * (i & 1)));
    }
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int quarter = warp & 3, half = warp >> 2;
  const int trow = quarter * 32 + lane;  // this thread's row (= TMEM lane)
  const int cb = half * FB_CW;           // its first column among the CTA's features
  const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
  const uint32_t tacc = tl + (uint32_t)cb;  // accumulator
  const uint32_t tg1 = tacc + FB_NS, tg2 = tacc + 2 * FB_NS, tg3 = tacc + 3 * FB_NS;  // SiLU'(z1..z3)
  bool ok = true;

  // the next phase of an mbarrier, the outcome agreed by the CTA
  auto wait_bar = [&](uint32_t bar, int& got) {
    const bool w = mbar_wait(bar, (uint32_t)(got & 1));
    if (w) ++got;
    ok = __syncthreads_and(ok && w) != 0;
    tc_fence_after();
  };
  auto issue = [&](uint32_t a, uint32_t b) {  // D = A B^T, K = 256
    if (tid == 0) fb_mma_k256(tmem, s0 + a, s0 + b, bar_m);
    ++iss_m;
  };
  auto reload = [&](uint32_t dst, const char* src, uint32_t bar, int& iss) {
    if (tid == 0) bulk_load(s0 + dst, src, FB_NS * H * 2, bar);
    ++iss;
  };
  // this CTA's block written (by every thread): visible to the copies and
  // the tensor cores, then sent to the other CTAs
  auto publish = [&](uint32_t blk, uint32_t bytes, uint32_t bar) {
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) fb_send(blk, bytes, bar, rank);
  };
  // forward epilogue of layer l: bias, SiLU, SiLU' into TMEM, the bf16 h_l
  // block into `blk` (and, for l = 2, the partial logit of these features)
  auto fwd_epilogue = [&](int l, uint32_t blk) {
    uint32_t v[32], gw[32], hw[16];
    tmem_ld32(tacc, v);
    const float* bias = sbias + l * FB_NS + cb;
    const float* w4 = sbias + 3 * FB_NS + cb;
    float z = 0.f;
#pragma unroll
    for (int i = 0; i < 32; i += 2) {
      const float p0 = __uint_as_float(v[i]) + bias[i];
      const float p1 = __uint_as_float(v[i + 1]) + bias[i + 1];
      const float q0 = sigmoid_f(p0), q1 = sigmoid_f(p1);
      hw[i / 2] = pack_bf16(p0 * q0, p1 * q1);
      gw[i] = __float_as_uint(silu_grad_from(p0, q0));
      gw[i + 1] = __float_as_uint(silu_grad_from(p1, q1));
      if (l == 2) {
        z = fmaf(bf16_lo(hw[i / 2]), w4[i], z);
        z = fmaf(bf16_hi(hw[i / 2]), w4[i + 1], z);
      }
    }
    tmem_st32(l == 0 ? tg1 : l == 1 ? tg2 : tg3, gw);
    fb_put_row(blk, trow, cb, hw);
    return z;
  };
  // backward epilogue: the dA = bf16(dH * SiLU'(z)) block into `blk`
  auto bwd_epilogue = [&](uint32_t tg, uint32_t blk) {
    uint32_t v[32], g[32], hw[16];
    tmem_ld32_async(tacc, v);
    tmem_ld32_async(tg, g);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 32; i += 2)
      hw[i / 2] = pack_bf16(__uint_as_float(v[i]) * __uint_as_float(g[i]),
                            __uint_as_float(v[i + 1]) * __uint_as_float(g[i + 1]));
    fb_put_row(blk, trow, cb, hw);
  };

  // ---- forward. z1 = X W1^T (K = 16)
  if (tid == 0) {
    tc_mma(tmem, make_desc(s0 + FB_X, 128, 256), make_desc(s0 + FB_W1, 128, 256), make_idesc(TILE, FB_NS), 0);
    tc_commit(bar_m);
  }
  iss_m = 1;
  wait_bar(bar_m, got_m);
  if (ok) fwd_epilogue(0, own0);
  cluster_wait();  // every CTA's mbarriers are ready
  if (ok) publish(own0, FB_BLK, bar_x0);
  // z2 = h1 W2^T once every block of h1 is here; this CTA's h1 out meanwhile
  if (ok) copy_out_tiled(smem + FB_A0 + rank * FB_BLK, A.hT[0], tile, fs, warp, lane);
  if (ok) wait_bar(bar_x0, got_x0);
  if (ok && tid == 0) mbar_expect(bar_x0, FB_RECV);  // dA2 arrives in A0
  if (ok) ++iss_x0;
  if (ok) wait_bar(bar_a, got_a);
  if (ok) issue(FB_A0, FB_WA);
  if (ok) wait_bar(bar_m, got_m);
  if (ok) reload(FB_WA, W3t, bar_a, iss_a);  // the MMAs have read W2: bring in W3^T
  if (ok) fwd_epilogue(1, own1);
  if (ok) publish(own1, FB_BLK, bar_x1);
  // z3 = h2 W3^T
  if (ok) copy_out_tiled(smem + FB_A1 + rank * FB_BLK, A.hT[1], tile, fs, warp, lane);
  if (ok) wait_bar(bar_x1, got_x1);
  if (ok && tid == 0) mbar_expect(bar_x1, FB_RECV);  // dA3 arrives in A1
  if (ok) ++iss_x1;
  if (ok) wait_bar(bar_b, got_b);
  if (ok) issue(FB_A1, FB_WB);
  if (ok) wait_bar(bar_m, got_m);
  if (ok) reload(FB_WB, W2t, bar_b, iss_b);  // W3 read: bring in W2^T
  if (ok) {
    // h3 into this CTA's block of A0 (the others' blocks of h1 there stay
    // until dA2 replaces them); the partial logit of its features
    float z = fwd_epilogue(2, own0);
    if (half == 1) shalf[trow] = z;
    __syncthreads();
    if (half == 0) spart[rank * TILE + trow] = z + shalf[trow];
    publish(s0 + FB_PART + rank * TILE * 4, TILE * 4, bar_p);
  }
  // ---- logits, dz = (sigmoid(z) - y) / n, the loss
  if (ok) wait_bar(bar_p, got_p);
  if (tid < TILE) {
    const int row = row0 + tid;
    float dz = 0.f, loss = 0.f;
    if (ok && row < n) {
      float z = spart[tid];
#pragma unroll
      for (int r = 1; r < FB_CTAS; ++r) z += spart[r * TILE + tid];  // in rank order
      z += b4;
      dz = (sigmoid_acc(z) - y) * A.inv_n;
      loss = fmaxf(z, 0.f) - z * y + log1pf(expf(-fabsf(z)));
      if (rank == 0) {
        A.logits[row] = z;
        A.dz[row] = dz;
      }
    }
    sdz[tid] = bf16_round(dz);
    sdzf[tid] = dz;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xFFFFFFFFu, loss, o);
    if (lane == 0) shalf[warp] = loss;
  }
  __syncthreads();
  if (ok && rank == 0 && tid == 0)  // the tile's BCE sum, its four warps in order
    A.tsum[(size_t)tile * TS_LD + H + 1] = ((shalf[0] + shalf[1]) + shalf[2]) + shalf[3];
  // ---- backward. dA3 = bf16(bf16(dz) W4 * SiLU'(z3)) into A1
  if (ok) {
    uint32_t g[32], hw[16];
    tmem_ld32(tg3, g);
    const float d = sdz[trow];
    const float* w4 = sbias + 3 * FB_NS + cb;
#pragma unroll
    for (int i = 0; i < 32; i += 2)
      hw[i / 2] = pack_bf16(d * w4[i] * __uint_as_float(g[i]), d * w4[i + 1] * __uint_as_float(g[i + 1]));
    fb_put_row(own1, trow, cb, hw);
    publish(own1, FB_BLK, bar_x1);
  }
  if (ok) copy_out_tiled(smem + FB_A1 + rank * FB_BLK, A.daT[2], tile, fs, warp, lane);
  // dW4 = sum dz h3 and db4 = sum dz over the tile's rows, this CTA's
  // features of h3 (its block of A0): thread (row group set, 8 features,
  // row in group) with 16-byte loads, the 8 rows of a group added across
  // lanes, the 4 row-group sets in order
  if (ok) {
    const int kg = (lane >> 3) + 4 * (warp & 1), rl = lane & 7;
    const uint8_t* blk = smem + FB_A0 + rank * FB_BLK;
    float acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int rg = (warp >> 1) + 4 * i;
      const uint4 v = *reinterpret_cast<const uint4*>(blk + rg * (FB_NS / 8) * 128 + kg * 128 + rl * 16);
      const float d = sdzf[rg * 8 + rl];
      const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        acc[2 * j] = fmaf(bf16_lo(w[j]), d, acc[2 * j]);
        acc[2 * j + 1] = fmaf(bf16_hi(w[j]), d, acc[2 * j + 1]);
      }
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] += __shfl_xor_sync(0xFFFFFFFFu, acc[j], o);
    if (rl == 0)
#pragma unroll
      for (int j = 0; j < 8; ++j) sred[(warp >> 1) * FB_NS + kg * 8 + j] = acc[j];
    __syncthreads();
    float* ts = A.tsum + (size_t)tile * TS_LD;
    if (tid < FB_NS) ts[fs + tid] = ((sred[tid] + sred[FB_NS + tid]) + sred[2 * FB_NS + tid]) + sred[3 * FB_NS + tid];
    if (rank == 0 && tid == FB_NS) {
      float t = 0.f;
      for (int r = 0; r < TILE; ++r) t += sdzf[r];
      ts[H] = t;
    }
  }
  // dH2 = dA3 W3 -> dA2 into A0 (h3 there is read)
  if (ok) wait_bar(bar_x1, got_x1);
  if (ok) wait_bar(bar_a, got_a);
  if (ok) issue(FB_A1, FB_WA);
  if (ok) wait_bar(bar_m, got_m);
  if (ok) {
    bwd_epilogue(tg2, own0);
    publish(own0, FB_BLK, bar_x0);
  }
  // dH1 = dA2 W2 -> dA1 into this CTA's block of A1 (dA3 there is read)
  if (ok) copy_out_tiled(smem + FB_A0 + rank * FB_BLK, A.daT[1], tile, fs, warp, lane);
  if (ok) wait_bar(bar_x0, got_x0);
  if (ok) wait_bar(bar_b, got_b);
  if (ok) issue(FB_A0, FB_WB);
  if (ok) wait_bar(bar_m, got_m);
  if (ok) bwd_epilogue(tg1, own1);
  __syncthreads();
  if (ok) copy_out_tiled(smem + FB_A1 + rank * FB_BLK, A.daT[0], tile, fs, warp, lane);

  if (!ok) {
    if (tid == 0) latch_error(status, kDevTimeout);
    // drain what is still in flight into this CTA (bounded)
    while (got_a < iss_a && mbar_wait(bar_a, (uint32_t)(got_a & 1))) ++got_a;
    while (got_b < iss_b && mbar_wait(bar_b, (uint32_t)(got_b & 1))) ++got_b;
    while (got_m < iss_m && mbar_wait(bar_m, (uint32_t)(got_m & 1))) ++got_m;
    while (got_x0 < iss_x0 && mbar_wait(bar_x0, (uint32_t)(got_x0 & 1))) ++got_x0;
    while (got_x1 < iss_x1 && mbar_wait(bar_x1, (uint32_t)(got_x1 & 1))) ++got_x1;
    while (got_p < iss_p && mbar_wait(bar_p, (uint32_t)(got_p & 1))) ++got_p;
  }
  // every CTA has received what this one sent before any of them leaves
  cluster_arrive();
  cluster_wait();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(FB_TCOLS) : "memory");
  }
}

// -------------------------------------------------------- weight gradients
//
// dW_l = dA_l^T H_{l-1} and db_l = dA_l^T 1 as one contraction per output
// tile: M = 128 output features, K = the batch, and N = the input features
// followed by a row of ones over the batch (bf16 1.0 for rows < n, so the
// bias gradient is the sum of dA in FP32 on the tensor cores): for the first
// layer the ones take input slot 9 (slots 9..15 pad the 9 inputs to 16); for
// the others they are row 256 of a 16-row block, contracted by a second MMA
// of N = 16 (N stops at 256). The batch is split over the S CTAs of a
// cluster; each CTA accumulates its split in TMEM, copies it to its shared
// memory, and after a cluster barrier sums one slice of rows over all S
// partials in split order (distributed shared-memory loads), writing dW and
// db directly. The fused kernel's per-tile sums of dW4, db4 and the loss are
// added by a warp per output while the first chunk is staged. With Adam arguments, the CTA that writes a
// gradient also applies the Adam update to its parameter (a training step
// then needs no separate update launch).

struct WgJob {
  const uint8_t* A;   // dL/da, chunk-tiled (256 features): A operand rows = output features
  const uint8_t* B;   // activations, chunk-tiled (N features): B operand rows = input features
  int N;              // 256, or 16 for the first layer (9 inputs, the ones in slot 9, zeros)
  float* dW;          // [256][256], or [256][9]
  float* db;          // [256]
  int off_w, off_b;   // offsets of dW and db in the packed parameters
};

struct WgArgs {
  WgJob job[3];
  int n;         // batch rows
  int S;         // K splits = CTAs per cluster
  int chunks;    // 64-row chunks per split
  const float* tsum;  // [tiles][TS_LD] per-tile sums of dz h3 | dz | BCE
  int tiles;
  float* dW4;    // [256]
  float* db4;    // [1]
  float* loss;   // mean BCE
  float inv_n;
  mlpp::AdamArgs adam;  // params NULL: gradients only
};

constexpr int WG_CHUNK = 64;                            // batch rows per staged chunk (K)
constexpr int WG_NB = H + 16;                           // B rows staged: inputs, then the ones block
constexpr int WG_STAGE_A = 128 * WG_CHUNK * 2;          // 16 KB
constexpr int WG_STAGE = WG_STAGE_A + WG_NB * WG_CHUNK * 2;  // + 34 KB
constexpr int WG_NST = 4;                               // chunk stages in flight
constexpr int WG_LD = WG_NB + 4;                        // floats per row of a CTA's partial (padded)
constexpr int WG_RED = TILE * WG_LD * 4;                // the partial, over the stages once they are read
constexpr int WG_BAR = (WG_NST * WG_STAGE > WG_RED ? WG_NST * WG_STAGE : WG_RED);  // 2 x WG_NST mbarriers
constexpr int WG_TMEM = WG_BAR + 16 * WG_NST;
constexpr int WG_TOTAL = WG_TMEM + 16;
constexpr int WG_MAX_S = 16;
constexpr int WG_RB = 32;  // reduced rows held at a time, past the partial
static_assert(WG_TOTAL <= 227 * 1024, "shared memory of one CTA");
static_assert(WG_RED + WG_RB * WG_LD * 4 <= WG_BAR, "reduced rows fit past the partial");

// 16 consecutive f32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t r[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float4 ld_cluster_f4(uint32_t addr) {
  float4 v;
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(addr)
               : "memory");
  return v;
}

// Global -> shared bulk copy of `bytes` (a multiple of 16, at most 32 KB;
// 16-byte aligned ends) completing on `bar`, whose expected byte count the
// caller has already raised.
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// Rows [r0, r0 + rows) of a staged B chunk: row `ones` holds bf16 1.0 for
// batch columns < n (0 past n), the others zero.
__device__ __forceinline__ void stage_ones(uint8_t* dst, int r0, int rows, int ones, int k0, int n, int tid) {
  for (int v = tid; v < rows * (WG_CHUNK / 8); v += THREADS) {
    const int r = r0 + (v >> 3), kv = (v & 7) * 8;
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    if (r == ones)
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (k0 + kv + j < n) w[j >> 1] |= 0x3F80u << (16 * (j & 1));
    *reinterpret_cast<uint4*>(dst + canon_offset(r, kv, WG_CHUNK)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// One (layer, 128-row tile of output features) per cluster of G.S CTAs, CTA
// rank = split of the batch (see above).
__global__ void __launch_bounds__(THREADS, 1) mlp_tc_wgrad_kernel(WgArgs G, int* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int S = G.S;
  const int jb = blockIdx.x / (2 * S), mt = (blockIdx.x / S) % 2;
  const int split = (int)cluster_ctarank();
  const WgJob J = G.job[jb];
  const bool wide = J.N == H;
  const int NB = wide ? WG_NB : 16;                // B rows staged
  const int ones = wide ? H : 9;                   // the row of ones
  const uint32_t ncols = wide ? 512u : 32u;        // TMEM columns (a power of two >= NB)
  const int LDr = NB + 4;                          // row stride of the partial in shared memory
  const uint32_t s0 = smem_u32(smem);
  const uint32_t bar0 = s0 + WG_BAR;               // MMAs done with stage s: bar0 + 8 s
  const uint32_t barf = bar0 + 8 * WG_NST;          // stage s landed: barf + 8 s
  float* red = reinterpret_cast<float*>(smem);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + WG_TMEM);
  if (tid == 0)
    for (int i = 0; i < 2 * WG_NST; ++i) mbar_init(bar0 + 8 * i, 1);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  griddep_signal();
  griddep_wait();  // the fused kernel's caches and sums are written; its reads of the weights are done
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc_w = make_idesc(TILE, H), idesc_n = make_idesc(TILE, 16);
  const int c_first = split * G.chunks;
  const int c_end = min(c_first + G.chunks, (G.n + WG_CHUNK - 1) / WG_CHUNK);
  uint32_t commits[WG_NST] = {};  // MMA commits issued to each stage's barrier
  uint32_t waited[WG_NST] = {};   // phases of each barrier already waited for
  uint32_t fills[WG_NST] = {};    // copies issued into each stage
  uint32_t landed[WG_NST] = {};   // ... and waited for
  bool ok = true;
  int issued = 0;
  const uint32_t bytes_b = (uint32_t)J.N * WG_CHUNK * 2;
  // chunk c is staged in buffer (c - c_first) % WG_NST by two bulk copies
  // (its 128 features of dA, the N input features) and, for N = 256, the
  // block of ones written by the threads; up to WG_NST chunks in flight, a
  // buffer restaged once the MMAs that read it are done
  auto stage = [&](int cix) {
    const int s = (cix - c_first) % WG_NST;
    const uint32_t sa = s0 + s * WG_STAGE, sb = sa + WG_STAGE_A;
    if (tid == 0) {
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(barf + 8 * s),
                   "r"((uint32_t)WG_STAGE_A + bytes_b)
                   : "memory");
      bulk_copy(sa, J.A + (size_t)cix * (H * 128) + (size_t)mt * WG_STAGE_A, WG_STAGE_A, barf + 8 * s);
      bulk_copy(sb, J.B + (size_t)cix * bytes_b, bytes_b, barf + 8 * s);
    }
    ++fills[s];
    if (wide) stage_ones(smem + s * WG_STAGE + WG_STAGE_A, H, 16, ones, cix * WG_CHUNK, G.n, tid);
    fence_proxy_async();
  };
  const int nc = c_end > c_first ? c_end - c_first : 0;
  for (int i = 0; i < nc && i < WG_NST; ++i) stage(c_first + i);
  // meanwhile the last layer's dW4 and db4 and the mean BCE from the fused
  // kernel's per-tile sums: a warp per output, lanes over the tiles, a
  // butterfly across the lanes
  for (int o = blockIdx.x * (THREADS / 32) + warp; o < TS_LD; o += gridDim.x * (THREADS / 32)) {
    float t = 0.f;
    for (int i = lane; i < G.tiles; i += 32) t += G.tsum[(size_t)i * TS_LD + o];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, off);
    if (lane == 0) {
      if (o == H + 1) {
        *G.loss = t * G.inv_n;
      } else {
        if (o < H) G.dW4[o] = t;
        else *G.db4 = t;
        if (G.adam.params) mlpp::adam_update(G.adam, o < H ? mlpp::OFF_W4 + o : mlpp::OFF_B4, t);
      }
    }
  }
  for (int i = 0; i < nc && ok; ++i) {
    const int s = i % WG_NST;
    {  // chunk i landed
      const bool w = mbar_wait(barf + 8 * s, landed[s] & 1);
      if (w) ++landed[s];
      tc_fence_before();
      if (!__syncthreads_and(w)) {
        ok = false;
        break;
      }
    }
    const uint32_t sa = s0 + s * WG_STAGE, sb = sa + WG_STAGE_A;
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int k = 0; k < WG_CHUNK / 16; ++k) {
        const uint64_t ad = make_desc(sa + 256 * k, 128, WG_CHUNK / 8 * 128);
        const uint32_t acc = (issued > 0 || k > 0) ? 1u : 0u;
        if (wide) {
          tc_mma(tmem, ad, make_desc(sb + 256 * k, 128, WG_CHUNK / 8 * 128), idesc_w, acc);
          tc_mma(tmem + H, ad, make_desc(sb + H / 8 * 1024 + 256 * k, 128, WG_CHUNK / 8 * 128), idesc_n, acc);
        } else {
          tc_mma(tmem, ad, make_desc(sb + 256 * k, 128, WG_CHUNK / 8 * 128), idesc_n, acc);
        }
      }
      tc_commit(bar0 + 8 * s);
    }
    ++commits[s];
    ++issued;
    if (i + WG_NST < nc) {  // restage this buffer with chunk i + WG_NST once its MMAs are done
      ok = mbar_wait(bar0 + 8 * s, waited[s] & 1);
      if (ok) ++waited[s];
      if (!__syncthreads_and(ok)) {
        ok = false;
        break;
      }
      tc_fence_after();
      stage(c_first + i + WG_NST);
    }
  }
  // every copy and every commit made must be waited for before the shared
  // memory is reused or TMEM is read or freed
  for (int s = 0; s < WG_NST; ++s)
    while (fills[s] > landed[s]) {
      if (!mbar_wait(barf + 8 * s, landed[s] & 1)) ok = false;
      ++landed[s];
    }
  for (int s = 0; s < WG_NST; ++s)
    while (commits[s] > waited[s]) {
      if (!mbar_wait(bar0 + 8 * s, waited[s] & 1)) ok = false;
      ++waited[s];
    }
  tc_fence_after();
  ok = __syncthreads_and(ok) != 0;
  // this split's partial [128][NB] into shared memory (over the stages)
  if (ok) {
    const int quarter = warp & 3, half = warp >> 2;
    const int row = quarter * 32 + lane;
    const uint32_t tq = tmem + ((uint32_t)(quarter * 32) << 16);
    float* dst = red + row * LDr;
    auto put = [&](int c0, const uint32_t* r, int cnt) {
      for (int j = 0; j < cnt; j += 4)
        *reinterpret_cast<float4*>(dst + c0 + j) =
            issued ? make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]), __uint_as_float(r[j + 2]),
                                 __uint_as_float(r[j + 3]))
                   : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    if (wide) {
#pragma unroll 1
      for (int c0 = half * (H / 2); c0 < (half + 1) * (H / 2); c0 += 32) {
        uint32_t r[32];
        tmem_ld32(tq + (uint32_t)c0, r);
        put(c0, r, 32);
      }
      if (half == 1) {
        uint32_t r[16];
        tmem_ld16(tq + (uint32_t)H, r);
        put(H, r, 16);
      }
    } else if (half == 0) {
      uint32_t r[16];
      tmem_ld16(tq, r);
      put(0, r, 16);
    }
  }
  // every split's partial is in its CTA's shared memory
  tc_fence_before();
  cluster_arrive();
  cluster_wait();
  // rows [split R, split R + R) of the tile (R = 128 / S rounded up), up to
  // WG_RB at a time: the S partials added in split order into shared memory
  // past the partial, every thread with the loads of two float4 groups in
  // flight together
  float* rs = reinterpret_cast<float*>(smem + WG_RED);  // [WG_RB][LDr] reduced rows
  const int R = (TILE + S - 1) / S;
  const int rall = min(TILE, split * R + R) - split * R;  // this CTA's rows (none for a trailing split)
  for (int rb = 0; rb < rall; rb += WG_RB) {
    const int r1 = min(WG_RB, rall - rb);
    const int row0 = split * R + rb;
    if (ok) {
      // float4 groups: the 256 weight columns of a wide layer (its ones block
      // contributes only column H, summed below as a scalar), or all 16
      // columns of the first layer
      const int q4 = wide ? H / 4 : NB / 4;
      const int ng = r1 * q4;
      for (int g0 = tid; g0 < ng; g0 += 2 * THREADS) {
        float4 v[2][WG_MAX_S];
        float vb[WG_MAX_S];
        const bool bias = wide && g0 == tid && tid < r1;  // row tid's bias column, in the same round
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int g = g0 + u * THREADS;
          if (g >= ng) continue;
          const uint32_t a = s0 + (uint32_t)((row0 + g / q4) * LDr + (g % q4) * 4) * 4u;
#pragma unroll
          for (int q = 0; q < WG_MAX_S; ++q)
            if (q < S) v[u][q] = ld_cluster_f4(map_shared_rank(a, (uint32_t)q));
        }
        if (bias) {
          const uint32_t a = s0 + (uint32_t)((row0 + tid) * LDr + H) * 4u;
#pragma unroll
          for (int q = 0; q < WG_MAX_S; ++q)
            if (q < S)
              asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(vb[q]) : "r"(map_shared_rank(a, (uint32_t)q)) : "memory");
          float t = vb[0];
#pragma unroll
          for (int q = 1; q < WG_MAX_S; ++q)
            if (q < S) t += vb[q];
          rs[tid * LDr + H] = t;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int g = g0 + u * THREADS;
          if (g >= ng) continue;
          float4 t = v[u][0];
#pragma unroll
          for (int q = 1; q < WG_MAX_S; ++q)
            if (q < S) {
              t.x += v[u][q].x; t.y += v[u][q].y; t.z += v[u][q].z; t.w += v[u][q].w;
            }
          *reinterpret_cast<float4*>(rs + (g / q4) * LDr + (g % q4) * 4) = t;
        }
      }
    }
    __syncthreads();
    // the gradients out and, with Adam arguments, their parameters updated
    if (ok) {
      const int o0 = mt * TILE + row0;  // first output feature of this block
      if (wide) {
        __nv_bfloat16* Wc = jb == 1 ? G.adam.W2c : G.adam.W3c;
        __nv_bfloat16* Wk = jb == 1 ? G.adam.W2k : G.adam.W3k;
        __nv_bfloat16* Wtc = jb == 1 ? G.adam.W2tc : G.adam.W3tc;
        const int ng = r1 * (H / 4);
        for (int g0 = tid; g0 < ng; g0 += 2 * THREADS) {
          float4 t[2], m0[2], v0[2], p0[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int g = g0 + u * THREADS;
            if (g >= ng) continue;
            const int rl = g / (H / 4), c = (g % (H / 4)) * 4, o = o0 + rl;
            t[u] = *reinterpret_cast<const float4*>(rs + rl * LDr + c);
            *reinterpret_cast<float4*>(J.dW + (size_t)o * H + c) = t[u];
            if (G.adam.params) {
              const size_t i = (size_t)J.off_w + (size_t)o * H + c;
              m0[u] = *reinterpret_cast<const float4*>(G.adam.m + i);
              v0[u] = *reinterpret_cast<const float4*>(G.adam.v + i);
              p0[u] = *reinterpret_cast<const float4*>(G.adam.params + i);
            }
          }
          if (!G.adam.params) continue;
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int g = g0 + u * THREADS;
            if (g >= ng) continue;
            const int rl = g / (H / 4), c = (g % (H / 4)) * 4, o = o0 + rl;
            const size_t i = (size_t)J.off_w + (size_t)o * H + c;
            const float gs[4] = {t[u].x, t[u].y, t[u].z, t[u].w}, ms[4] = {m0[u].x, m0[u].y, m0[u].z, m0[u].w},
                        vs[4] = {v0[u].x, v0[u].y, v0[u].z, v0[u].w}, ps[4] = {p0[u].x, p0[u].y, p0[u].z, p0[u].w};
            float mn[4], vn[4], pn[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) mlpp::adam_core(G.adam, gs[j], ms[j], vs[j], ps[j], mn[j], vn[j], pn[j]);
            *reinterpret_cast<float4*>(G.adam.m + i) = make_float4(mn[0], mn[1], mn[2], mn[3]);
            *reinterpret_cast<float4*>(G.adam.v + i) = make_float4(vn[0], vn[1], vn[2], vn[3]);
            *reinterpret_cast<float4*>(G.adam.params + i) = make_float4(pn[0], pn[1], pn[2], pn[3]);
            // bf16 copies: 4 consecutive inputs of output o ([out][in] and
            // K-sliced, 8 bytes each) and the transposed copy's 4 rows
            const __nv_bfloat162 h01 = __floats2bfloat162_rn(pn[0], pn[1]), h23 = __floats2bfloat162_rn(pn[2], pn[3]);
            const uint2 h4 = make_uint2(*reinterpret_cast<const uint32_t*>(&h01), *reinterpret_cast<const uint32_t*>(&h23));
            *reinterpret_cast<uint2*>(Wc + canon_offset(o, c, H) / 2) = h4;
            *reinterpret_cast<uint2*>(Wk + mlpp::kslice_offset(o, c) / 2) = h4;
#pragma unroll
            for (int j = 0; j < 4; ++j) Wtc[canon_offset(c + j, o, H) / 2] = __float2bfloat16_rn(pn[j]);
          }
        }
        for (int rl = tid; rl < r1; rl += THREADS) {  // the bias gradients
          const int o = o0 + rl;
          const float t = rs[rl * LDr + H];
          J.db[o] = t;
          if (G.adam.params) mlpp::adam_update(G.adam, J.off_b + o, t);
        }
      } else {  // the first layer: 9 weights and the bias per output
        for (int e = tid; e < r1 * 10; e += THREADS) {
          const int rl = e / 10, c = e % 10, o = o0 + rl;
          const float t = rs[rl * LDr + c];
          int pi;
          if (c < 9) {
            J.dW[o * 9 + c] = t;
            pi = J.off_w + o * 9 + c;
          } else {
            J.db[o] = t;
            pi = J.off_b + o;
          }
          if (G.adam.params) mlpp::adam_update(G.adam, pi, t);
        }
      }
    }
    __syncthreads();  // the reduced rows are read before the next block replaces them
  }
  // no CTA leaves while another may still read its shared memory
  cluster_arrive();
  cluster_wait();
  if (!ok && tid == 0) latch_error(status, kDevTimeout);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

}  // namespace

size_t mlp_train_tc_tile_sum_bytes(int Bcap) { return (size_t)((Bcap + TILE - 1) / TILE) * TS_LD * 4; }

namespace {

// Per device: the kernels' attributes set, and the split count chosen for
// each chunk count up to WG_MAX_S (0: not yet), so that a training step
// makes no host calls beyond its two launches once a device has been seen.
constexpr int kMaxDevices = 64;
struct TrainLaunchCache {
  bool attrs = false;
  int splits[WG_MAX_S + 1] = {};
};
TrainLaunchCache g_train_cache[kMaxDevices];

cudaError_t train_launch_setup(TrainLaunchCache** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  TrainLaunchCache& c = g_train_cache[dev];
  if (!c.attrs) {
    if ((e = cudaFuncSetAttribute(mlp_train_fb_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, FB_TOTAL)) ||
        (e = cudaFuncSetAttribute(mlp_tc_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, WG_TOTAL)) ||
        (e = cudaFuncSetAttribute(mlp_tc_wgrad_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)))
      return e;
    c.attrs = true;
  }
  *out = &c;
  return cudaSuccess;
}

}  // namespace

cudaError_t mlp_train_tc_step(const TrainTcLaunch& L, int num_sms, cudaStream_t s) {
  if (L.n <= 0) return cudaSuccess;
  const int ntiles = (L.n + TILE - 1) / TILE;
  TrainLaunchCache* cache = nullptr;
  cudaError_t e = train_launch_setup(&cache);
  if (e) return e;
  // ---- forward and backward through the activations, a cluster per tile
  {
    FbArgs A;
    A.w = L.w;
    A.W2tc = L.W2tc;
    A.W3tc = L.W3tc;
    A.targets = L.targets;
    A.labels = L.labels;
    A.index = L.index;
    A.n = L.n;
    A.inv_n = 1.f / (float)L.n;
    A.logits = L.logits;
    A.x16T = L.x16T;
    for (int l = 0; l < 3; ++l) A.daT[l] = L.daT[l];
    for (int l = 0; l < 2; ++l) A.hT[l] = L.hT[l];
    A.dz = L.dz;
    A.tsum = L.tile_sums;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(FB_CTAS * ntiles));
    cfg.blockDim = dim3(FB_THREADS);
    cfg.dynamicSmemBytes = FB_TOTAL;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = FB_CTAS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    if ((e = cudaLaunchKernelEx(&cfg, mlp_train_fb_kernel, A, L.status))) return e;
  }
  // ---- weight and bias gradients, split-K over the CTAs of a cluster
  {
    WgArgs G;
    G.n = L.n;
    const int chunks = (L.n + WG_CHUNK - 1) / WG_CHUNK;
    G.job[0] = WgJob{L.daT[0], L.x16T, 16, L.dW1, L.db[0], mlpp::OFF_W1, mlpp::OFF_B1};
    G.job[1] = WgJob{L.daT[1], L.hT[0], H, L.dW2, L.db[1], mlpp::OFF_W2, mlpp::OFF_B2};
    G.job[2] = WgJob{L.daT[2], L.hT[1], H, L.dW3, L.db[2], mlpp::OFF_W3, mlpp::OFF_B3};
    if (L.adam) {
      G.adam = *L.adam;
    } else {
      std::memset(&G.adam, 0, sizeof(G.adam));
    }
    G.tsum = L.tile_sums;
    G.tiles = ntiles;
    G.dW4 = L.dW4;
    G.db4 = L.db4;
    G.loss = L.loss_sum;
    G.inv_n = 1.f / (float)L.n;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = WG_TOTAL;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    // the most splits (up to 16) whose six clusters can all be resident
    const int cmax = chunks < WG_MAX_S ? chunks : WG_MAX_S;
    int S = cache->splits[cmax];
    if (S == 0) {
      for (S = cmax; S > 1; S = S > 8 ? 8 : S / 2) {
        at[0].val.clusterDim.x = (unsigned)S;
        cfg.gridDim = dim3((unsigned)(3 * 2 * S));
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, mlp_tc_wgrad_kernel, &cfg) == cudaSuccess && clusters >= 6)
          break;
        (void)cudaGetLastError();
      }
      cache->splits[cmax] = S;
    }
    G.S = S;
    G.chunks = (chunks + S - 1) / S;
    at[0].val.clusterDim.x = (unsigned)S;
    cfg.gridDim = dim3((unsigned)(3 * 2 * S));
    if ((e = cudaLaunchKernelEx(&cfg, mlp_tc_wgrad_kernel, G, L.status))) return e;
  }
  return cudaSuccess;
}

}  // namespace sc
