// Surrogate training on the 5th-generation tensor cores (tcgen05 + TMEM):
// one step of binary cross-entropy on logits for the learned reachability
// gate of Sec. IV-E, as three contractions per layer, all bf16 x bf16 -> f32
// in TMEM with operands in the canonical no-swizzle K-major layout:
//
//   forward   Z_l  = H_{l-1} W_l^T        mlp_tc_kernel<TrainIO> (the inference
//                                          kernel, which here also keeps SiLU'(Z_l)
//                                          and, feature-major, every bf16
//                                          activation)
//   backward  dH_l = dA_{l+1} W_{l+1}     mlp_tc_bwd_kernel, B = W^T copies
//             dA_l = bf16(dH_l * SiLU'(Z_l))
//   weights   dW_l = dA_l^T H_{l-1}       mlp_tc_wgrad_kernel: M = output
//                                          features (two 128-row tiles), N = input
//                                          features, K = the batch, split over
//                                          CTAs; partial sums added in split
//                                          order by mlp_wgrad_reduce_kernel
//
// Rounding points as in the FP64 reference: standardised input, SiLU outputs,
// weight copies, dL/dz before it meets W4 and every dL/da in bf16; biases,
// pre-activations, accumulations and gradients in FP32. Every mbarrier wait is
// bounded; on timeout the CTA latches kDevTimeout, drains its own copies and
// MMAs, frees TMEM and returns.
#include "mlp_tc_core.cuh"

namespace sc {

namespace {

// Forward rows of a training batch: targets through an index, and the caches
// the backward pass and the weight gradients read.
// SiLU'(z) of every activation in a tile layout: float4 blocks of 4 columns,
// [64 column blocks][ld rows], so a warp's 32 consecutive rows touch 512
// contiguous bytes.
struct TrainIO {
  static constexpr int kColGroups = 4;
  static constexpr bool kStores = true;
  const float* targets;
  const int32_t* index;  // batch row -> target (NULL: identity)
  int n;
  float* logits;         // [n]
  uint16_t* x16T;        // [16][ld] standardised input, bf16, feature-major
  uint16_t* hT[3];       // [256][ld] h1, h2, h3, bf16, feature-major
  float4* g[3];          // [64][ld] SiLU'(z1), SiLU'(z2), SiLU'(z3)
  int ld;
  __device__ int rows() const { return n; }
  __device__ void features(int row, float f[9]) const {
    const int ti = index ? __ldg(&index[row]) : row;
    const float* t = targets + 12 * (size_t)ti;
    f[0] = __ldg(t + 9); f[1] = __ldg(t + 10); f[2] = __ldg(t + 11);
    f[3] = __ldg(t + 0); f[4] = __ldg(t + 3); f[5] = __ldg(t + 6);
    f[6] = __ldg(t + 1); f[7] = __ldg(t + 4); f[8] = __ldg(t + 7);
  }
  __device__ void emit(int row, bool valid, float logit) const {
    if (valid) logits[row] = logit;
  }
  __device__ void store_input(int row, const uint32_t* xb) const {
#pragma unroll
    for (int i = 0; i < 16; ++i) x16T[(size_t)i * ld + row] = (uint16_t)(xb[i >> 1] >> (16 * (i & 1)));
  }
  __device__ void store_grad(int layer, int row, int col8, const float* gg) const {
    g[layer][(size_t)(col8 / 4) * ld + row] = make_float4(gg[0], gg[1], gg[2], gg[3]);
    g[layer][(size_t)(col8 / 4 + 1) * ld + row] = make_float4(gg[4], gg[5], gg[6], gg[7]);
  }
  __device__ uint16_t* act_out(int layer) const { return hT[layer]; }
  __device__ int act_ld() const { return ld; }
};

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float sigmoid_acc(float a) { return 1.f / (1.f + expf(-a)); }

// ------------------------------------------------------------ backward pass

struct BwdArgs {
  const void* W3tc;        // bf16 [256 in][256 out] canonical: B operand of dH2 = dA3 W3
  const void* W2tc;        // bf16 canonical: B operand of dH1 = dA2 W2
  const uint16_t* W4;      // bf16 [256]
  const float* logits;     // [n]
  const uint8_t* labels;   // [targets], through index
  const int32_t* index;
  int n;
  float inv_n;
  const float4* g[3];      // SiLU'(z1), SiLU'(z2), SiLU'(z3) in TrainIO's tile layout
  uint16_t* daT[3];        // dL/da1, da2, da3, bf16 [256][ld]
  float* dz;               // [n] dL/dz
  float* loss_sum;         // mean BCE (sum / n)
  int ld;
};

constexpr int BW_THREADS = 512;              // 16 warps: TMEM lane quarter x 4 column groups of 64
constexpr int BW_CW = H / 4;
constexpr int BW_W = 0;                      // [256][256] bf16 canonical weights, 128 KB
constexpr int BW_A = BW_W + 131072;          // [128][256] bf16 canonical dA operand, 64 KB
constexpr int BW_W4 = BW_A + 65536;          // W4 as f32, 1 KB
constexpr int BW_DZ = BW_W4 + 4 * H;         // [128] bf16-rounded dz of the tile
constexpr int BW_BAR = BW_DZ + 4 * TILE;     // 2 mbarriers
constexpr int BW_TMEM = BW_BAR + 16;
constexpr int BW_TOTAL = BW_TMEM + 16;

// Epilogue of one backward contraction for one thread's row and 64 columns:
// dA = bf16(TMEM * SiLU'(z)) (zero on rows past the batch) into the shared
// operand buffer, from where it is copied out feature-major.
__device__ __forceinline__ void bwd_epilogue(uint32_t taddr, const float4* g, int ld, uint8_t* sa, int trow, int col0,
                                             int grow, bool valid) {
  uint32_t r[2][32];
  tmem_ld32_async(taddr, r[0]);
  tmem_wait_ld();
#pragma unroll
  for (int c0 = 0; c0 < BW_CW; c0 += 32) {
    const int cur = (c0 / 32) & 1;
    if (c0 + 32 < BW_CW) tmem_ld32_async(taddr + c0 + 32, r[cur ^ 1]);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = col0 + c0 + q * 8;
      float4 ga = make_float4(0.f, 0.f, 0.f, 0.f), gb = ga;
      if (valid) {
        ga = g[(size_t)(c / 4) * ld + grow];
        gb = g[(size_t)(c / 4 + 1) * ld + grow];
      }
      const float* v = reinterpret_cast<const float*>(&r[cur][q * 8]);
      const uint4 w = make_uint4(pack_bf16(v[0] * ga.x, v[1] * ga.y), pack_bf16(v[2] * ga.z, v[3] * ga.w),
                                 pack_bf16(v[4] * gb.x, v[5] * gb.y), pack_bf16(v[6] * gb.z, v[7] * gb.w));
      *reinterpret_cast<uint4*>(sa + canon_offset(trow, c, H)) = w;
    }
    if (c0 + 32 < BW_CW) tmem_wait_ld();
  }
}

// Backward through the activations, one persistent CTA of 16 warps per SM over
// 128-row tiles: dz = (sigmoid(z) - y) / n and the loss; dA3 = bf16(bf16(dz)
// W4 * SiLU'(z3)) formed by the threads into the A operand; dH2 = dA3 W3 and
// dH1 = dA2 W2 on the tensor cores (the W^T copies arrive by bulk copy, the
// next one overlapping the epilogue).
__global__ void __launch_bounds__(BW_THREADS, 1) mlp_tc_bwd_kernel(BwdArgs A, int* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = A.n;
  const int ntiles = (n + TILE - 1) / TILE;
  if ((int)blockIdx.x >= ntiles) return;
  uint8_t* sw = smem + BW_W;
  uint8_t* sa = smem + BW_A;
  float* sw4 = reinterpret_cast<float*>(smem + BW_W4);
  float* sdz = reinterpret_cast<float*>(smem + BW_DZ);
  const uint32_t bar_w = smem_u32(smem + BW_BAR), bar_m = bar_w + 8;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + BW_TMEM);
  if (tid == 0) {
    mbar_init(bar_w, 1);
    mbar_init(bar_m, 1);
  }
  for (int i = tid; i < H; i += BW_THREADS) sw4[i] = __uint_as_float((uint32_t)__ldg(&A.W4[i]) << 16);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)), "r"(H)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_proxy_async();
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int quarter = warp & 3, cg = warp >> 2;
  const int trow = quarter * 32 + lane;
  const int col0 = cg * BW_CW;
  const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)col0;
  constexpr uint32_t idesc = make_idesc(TILE, H);

  uint32_t ph_w = 0, ph_m = 0;
  bool w_pending = true, m_pending = false, ok = true;
  if (tid == 0) bulk_load(smem_u32(sw), A.W3tc, 131072, bar_w);

  for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    // ---- dz and the loss (one thread per row)
    if (tid < TILE) {
      const int row = tile * TILE + tid;
      float dz = 0.f, loss = 0.f;
      if (row < n) {
        const float z = A.logits[row];
        const float y = A.labels[A.index ? __ldg(&A.index[row]) : row] ? 1.f : 0.f;
        dz = (sigmoid_acc(z) - y) * A.inv_n;
        loss = fmaxf(z, 0.f) - z * y + log1pf(expf(-fabsf(z)));
        A.dz[row] = dz;
      }
      sdz[tid] = bf16_round(dz);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xFFFFFFFFu, loss, o);
      if (lane == 0) atomicAdd(A.loss_sum, loss * A.inv_n);
    }
    __syncthreads();
    // ---- dA3 = bf16(bf16(dz) W4 * SiLU'(z3)): thread (row, 64 columns)
    {
      const int r = tid & (TILE - 1), cb = (tid >> 7) * BW_CW;
      const int grow = tile * TILE + r;
      const bool valid = grow < n;
      const float d = sdz[r];
#pragma unroll 4
      for (int c = cb; c < cb + BW_CW; c += 8) {
        float4 ga = make_float4(0.f, 0.f, 0.f, 0.f), gb = ga;
        if (valid) {
          ga = A.g[2][(size_t)(c / 4) * A.ld + grow];
          gb = A.g[2][(size_t)(c / 4 + 1) * A.ld + grow];
        }
        const float* w4 = sw4 + c;
        *reinterpret_cast<uint4*>(sa + canon_offset(r, c, H)) =
            make_uint4(pack_bf16(d * w4[0] * ga.x, d * w4[1] * ga.y), pack_bf16(d * w4[2] * ga.z, d * w4[3] * ga.w),
                       pack_bf16(d * w4[4] * gb.x, d * w4[5] * gb.y), pack_bf16(d * w4[6] * gb.z, d * w4[7] * gb.w));
      }
    }
    // ---- dH2 = dA3 W3 -> dA2; dH1 = dA2 W2 -> dA1. Each dA is copied out
    // feature-major from the operand buffer (dA3, dA2 while the tensor cores
    // read them; dA1 after the last contraction).
    const int grow = tile * TILE + trow;
    for (int layer = 0; layer < 2; ++layer) {
      fence_proxy_async();
      tc_fence_before();
      ok = mbar_wait(bar_w, ph_w);
      if (ok) {
        ph_w ^= 1;
        w_pending = false;
      }
      if (!__syncthreads_and(ok)) {
        ok = false;
        break;
      }
      if (tid == 0) {
        tc_fence_after();
#pragma unroll 1
        for (int s = 0; s < H / 16; ++s)
          tc_mma(tmem, make_desc(smem_u32(sa) + 256 * s, 128, 4096), make_desc(smem_u32(sw) + 256 * s, 128, 4096),
                 idesc, s > 0);
        tc_commit(bar_m);
      }
      copy_out_transposed(sa, A.daT[2 - layer], A.ld, tile * TILE, n - tile * TILE, tid, BW_THREADS);
      m_pending = true;
      ok = mbar_wait(bar_m, ph_m);
      if (ok) {
        ph_m ^= 1;
        m_pending = false;
      }
      tc_fence_after();
      if (!__syncthreads_and(ok)) {
        ok = false;
        break;
      }
      // the MMAs have read the weights and the operand; the copy is done
      if (layer == 0 || tile + (int)gridDim.x < ntiles) {
        if (tid == 0) bulk_load(smem_u32(sw), layer == 0 ? A.W2tc : A.W3tc, 131072, bar_w);
        w_pending = true;
      }
      bwd_epilogue(taddr, A.g[1 - layer], A.ld, sa, trow, col0, grow, grow < n);
      tc_fence_before();
      __syncthreads();  // TMEM read and the operand written before the next MMA or copy
    }
    if (!ok) break;
    copy_out_transposed(sa, A.daT[0], A.ld, tile * TILE, n - tile * TILE, tid, BW_THREADS);
    __syncthreads();  // the operand is read before the next tile's dA3 overwrites it
  }
  if (!ok) {
    if (tid == 0) latch_error(status, kDevTimeout);
    if (w_pending) mbar_wait(bar_w, ph_w);
    if (m_pending) mbar_wait(bar_m, ph_m);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(H) : "memory");
  }
}

// -------------------------------------------------------- weight gradients

struct WgJob {
  const uint16_t* A;  // dL/da feature-major [256][ld]: A operand rows = output features
  const uint16_t* B;  // activations feature-major [N][ld]: B operand rows = input features
  int N;              // 256, or 16 for the first layer (inputs padded to 16)
  float* part;        // [S][256][N] partial sums
};

struct WgArgs {
  WgJob job[3];
  int n;         // batch rows
  int ld;
  int S;         // K splits
  int chunks;    // 64-row chunks per split
};

constexpr int WG_CHUNK = 64;                       // batch rows per staged chunk (K)
constexpr int WG_STAGE_A = 128 * WG_CHUNK * 2;     // 16 KB
constexpr int WG_STAGE = WG_STAGE_A + H * WG_CHUNK * 2;  // + 32 KB
constexpr int WG_BAR = 2 * WG_STAGE;               // 2 mbarriers
constexpr int WG_TMEM = WG_BAR + 16;
constexpr int WG_TOTAL = WG_TMEM + 16;

// 16 consecutive f32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t r[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Rows [row0, row0 + rows) x batch columns [k0, k0 + 64) of a feature-major
// bf16 matrix into the canonical K-major layout (K = 64) by asynchronous
// 16-byte copies (cp.async; whole vectors past n are zero-filled by the copy,
// a vector that straddles n is assembled by the thread); batch columns at or
// past n read as zero.
__device__ __forceinline__ void stage_chunk_async(uint8_t* dst, const uint16_t* src, int row0, int rows, int k0,
                                                  int n, int ld, int tid) {
  for (int v = tid; v < rows * (WG_CHUNK / 8); v += THREADS) {
    const int r = v >> 3, kv = (v & 7) * 8;
    const int k = k0 + kv;
    const uint16_t* p = src + (size_t)(row0 + r) * ld + k;
    uint8_t* d = dst + canon_offset(r, kv, WG_CHUNK);
    if (k + 8 <= n || k >= n) {
      const uint32_t bytes = k < n ? 16u : 0u;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(d)), "l"(k < n ? p : src),
                   "r"(bytes)
                   : "memory");
    } else {
      uint16_t e[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) e[j] = k + j < n ? p[j] : (uint16_t)0;
      *reinterpret_cast<uint4*>(d) = make_uint4(e[0] | ((uint32_t)e[1] << 16), e[2] | ((uint32_t)e[3] << 16),
                                                e[4] | ((uint32_t)e[5] << 16), e[6] | ((uint32_t)e[7] << 16));
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// dW (one 128-row tile of output features) over one split of the batch:
// 64-row chunks staged in two buffers, the next chunk loading while the
// tensor cores work on the current one.
__global__ void __launch_bounds__(THREADS, 1) mlp_tc_wgrad_kernel(WgArgs G, int* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int per_job = 2 * G.S;
  const int jb = blockIdx.x / per_job, mt = (blockIdx.x / G.S) % 2, split = blockIdx.x % G.S;
  const WgJob J = G.job[jb];
  const int N = J.N;
  const uint32_t ncols = N >= 32 ? (uint32_t)N : 32u;  // TMEM columns (a power of two >= 32)
  const uint32_t bar0 = smem_u32(smem + WG_BAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + WG_TMEM);
  if (tid == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar0 + 8, 1);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = make_idesc(TILE, N);
  const int c_first = split * G.chunks;
  const int c_end = min(c_first + G.chunks, (G.n + WG_CHUNK - 1) / WG_CHUNK);
  uint32_t commits[2] = {0u, 0u};  // MMA commits issued to each stage's barrier
  uint32_t waited[2] = {0u, 0u};   // phases of each barrier already waited for
  bool ok = true;
  int issued = 0;
  // chunk c is staged in buffer (c - c_first) & 1; chunk c + 1 is copied in
  // while the tensor cores work on chunk c
  auto stage = [&](int cix) {
    uint8_t* sa = smem + ((cix - c_first) & 1) * WG_STAGE;
    stage_chunk_async(sa, J.A, mt * TILE, TILE, cix * WG_CHUNK, G.n, G.ld, tid);
    stage_chunk_async(sa + WG_STAGE_A, J.B, 0, N, cix * WG_CHUNK, G.n, G.ld, tid);
  };
  if (c_first < c_end) stage(c_first);
  for (int cix = c_first; cix < c_end && ok; ++cix) {
    const int s = (cix - c_first) & 1;
    const bool more = cix + 1 < c_end;
    if (more) {
      const int s1 = s ^ 1;
      if (commits[s1] > waited[s1]) {  // the MMAs that last read the next buffer are done
        ok = mbar_wait(bar0 + 8 * s1, waited[s1] & 1);
        if (ok) ++waited[s1];
      }
      if (!__syncthreads_and(ok)) {
        ok = false;
        break;
      }
      tc_fence_after();
      stage(cix + 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");  // this thread's copies of chunk cix landed
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    uint8_t* sa = smem + s * WG_STAGE;
    uint8_t* sb = sa + WG_STAGE_A;
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int k = 0; k < WG_CHUNK / 16; ++k)
        tc_mma(tmem, make_desc(smem_u32(sa) + 256 * k, 128, WG_CHUNK / 8 * 128),
               make_desc(smem_u32(sb) + 256 * k, 128, WG_CHUNK / 8 * 128), idesc, (issued > 0 || k > 0) ? 1u : 0u);
      tc_commit(bar0 + 8 * s);
    }
    ++commits[s];
    ++issued;
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");  // nothing of this thread's left in flight
  // every commit made must be waited for before TMEM is read or freed
  for (int s = 0; s < 2; ++s)
    while (commits[s] > waited[s]) {
      if (!mbar_wait(bar0 + 8 * s, waited[s] & 1)) ok = false;
      ++waited[s];
    }
  tc_fence_after();
  ok = __syncthreads_and(ok) != 0;
  if (!ok) {
    if (tid == 0) latch_error(status, kDevTimeout);
  } else {
    // D row = output feature mt * 128 + lane quarter; columns = input features
    const int quarter = warp & 3, half = warp >> 2;
    const int o = mt * TILE + quarter * 32 + lane;
    float* dst = J.part + ((size_t)split * H + o) * N;
    const uint32_t tq = tmem + ((uint32_t)(quarter * 32) << 16);
    if (N == H) {
#pragma unroll 1
      for (int c0 = half * (H / 2); c0 < (half + 1) * (H / 2); c0 += 32) {
        uint32_t r[32];
        tmem_ld32(tq + (uint32_t)c0, r);
        if (issued == 0) {
#pragma unroll
          for (int j = 0; j < 32; ++j) r[j] = 0u;
        }
#pragma unroll
        for (int j = 0; j < 32; j += 4)
          *reinterpret_cast<float4*>(dst + c0 + j) = make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                                                  __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
      }
    } else if (half == 0) {  // N = 16
      uint32_t r[16];
      tmem_ld16(tq, r);
#pragma unroll
      for (int j = 0; j < 16; ++j) dst[j] = issued ? __uint_as_float(r[j]) : 0.f;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

// The rest of the gradients, one launch: the weight gradients as sums over
// the splits in split order (dW1 [256][9], inputs 9..15 dropped; dW2, dW3
// [256][256]), from blocks [0, red_blocks); then, one warp per output, the
// bias gradients (sums of dA over the batch), dW4 = sum dz h3 and
// db4 = sum dz, four bf16 per lane and load (rows are 32-byte aligned: ld is a
// multiple of 16), four independent partial sums per lane.
struct FinishArgs {
  float* dW[3];
  float* db[3];
  float* dW4;
  float* db4;
  const uint16_t* daT[3];
  const uint16_t* h3T;
  const float* dz;
  int red_blocks;
};

__device__ __forceinline__ float bf16_lo(uint32_t x) { return __uint_as_float(x << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t x) { return __uint_as_float(x & 0xFFFF0000u); }

__global__ void mlp_grad_finish_kernel(WgArgs G, FinishArgs F) {
  if ((int)blockIdx.x < F.red_blocks) {
    const int n1 = H * 16, n2 = H * H;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n1 + 2 * n2; e += F.red_blocks * blockDim.x) {
      const int jb = e < n1 ? 0 : e < n1 + n2 ? 1 : 2;
      const int idx = jb == 0 ? e : jb == 1 ? e - n1 : e - n1 - n2;
      const int N = jb == 0 ? 16 : H;
      const float* part = jb == 0 ? G.job[0].part : jb == 1 ? G.job[1].part : G.job[2].part;
      const int o = idx / N, i = idx % N;
      if (jb == 0 && i >= 9) continue;
      float v[16];
#pragma unroll
      for (int s = 0; s < 16; ++s) v[s] = s < G.S ? part[((size_t)s * H + o) * N + i] : 0.f;  // loads in flight together
      float acc = 0.f;
#pragma unroll
      for (int s = 0; s < 16; ++s) acc += v[s];  // split order
      if (jb == 0) F.dW[0][o * 9 + i] = acc;
      else F.dW[jb][o * H + i] = acc;
    }
    return;
  }
  // rows 0..H-1: db1, H..2H-1: db2, 2H..3H-1: db3, 3H..4H-1: dW4, 4H: db4
  const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
  const int w = ((int)blockIdx.x - F.red_blocks) * warps + (threadIdx.x >> 5);
  const int B = G.n, B4 = G.n & ~3;
  for (int row = w; row <= 4 * H; row += ((int)gridDim.x - F.red_blocks) * warps) {
    float acc = 0.f;
    if (row < 4 * H) {
      const bool dot = row >= 3 * H;
      const uint16_t* src = row < H ? F.daT[0] : row < 2 * H ? F.daT[1] : row < 3 * H ? F.daT[2] : F.h3T;
      const uint16_t* p = src + (size_t)(row % H) * G.ld;
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
      for (int s = 4 * lane; s < B4; s += 128) {
        const uint2 v = *reinterpret_cast<const uint2*>(p + s);
        if (dot) {
          const float4 d = *reinterpret_cast<const float4*>(F.dz + s);
          a0 = fmaf(bf16_lo(v.x), d.x, a0); a1 = fmaf(bf16_hi(v.x), d.y, a1);
          a2 = fmaf(bf16_lo(v.y), d.z, a2); a3 = fmaf(bf16_hi(v.y), d.w, a3);
        } else {
          a0 += bf16_lo(v.x); a1 += bf16_hi(v.x); a2 += bf16_lo(v.y); a3 += bf16_hi(v.y);
        }
      }
      for (int s = B4 + lane; s < B; s += 32) {
        const float x = __uint_as_float((uint32_t)p[s] << 16);
        a0 = dot ? fmaf(x, F.dz[s], a0) : a0 + x;
      }
      acc = (a0 + a1) + (a2 + a3);
    } else {
      for (int s = lane; s < B; s += 32) acc += F.dz[s];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, off);
    if (lane == 0) {
      if (row < 3 * H) F.db[row / H][row % H] = acc;
      else if (row < 4 * H) F.dW4[row - 3 * H] = acc;
      else *F.db4 = acc;
    }
  }
}

}  // namespace

size_t mlp_train_tc_part_bytes(int Bcap) {
  const int S = mlp_train_tc_splits(Bcap);
  return (size_t)S * H * (16 + 2 * H) * 4;
}

int mlp_train_tc_splits(int Bcap) {
  const int chunks = (Bcap + WG_CHUNK - 1) / WG_CHUNK;
  return chunks < 16 ? chunks : 16;
}

cudaError_t mlp_train_tc_step(const TrainTcLaunch& L, int num_sms, cudaStream_t s) {
  if (L.n <= 0) return cudaSuccess;
  const int ntiles = (L.n + TILE - 1) / TILE;
  cudaError_t e;
  // ---- forward with caches
  {
    TrainIO io;
    io.targets = L.targets;
    io.index = L.index;
    io.n = L.n;
    io.logits = L.logits;
    io.x16T = L.x16T;
    for (int l = 0; l < 3; ++l) {
      io.hT[l] = L.hT[l];
      io.g[l] = L.g[l];
    }
    io.ld = L.ld;
    if ((e = launch_mlp_tc(L.w, io, L.n, L.status, num_sms, s))) return e;
  }
  // ---- backward through the activations
  {
    BwdArgs A;
    A.W3tc = L.W3tc;
    A.W2tc = L.W2tc;
    A.W4 = static_cast<const uint16_t*>(L.w.W4);
    A.logits = L.logits;
    A.labels = L.labels;
    A.index = L.index;
    A.n = L.n;
    A.inv_n = 1.f / (float)L.n;
    for (int l = 0; l < 3; ++l) {
      A.g[l] = L.g[l];
      A.daT[l] = L.daT[l];
    }
    A.dz = L.dz;
    A.loss_sum = L.loss_sum;
    A.ld = L.ld;
    if ((e = cudaFuncSetAttribute(mlp_tc_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, BW_TOTAL))) return e;
    const int grid = ntiles < num_sms ? ntiles : num_sms;
    mlp_tc_bwd_kernel<<<grid, BW_THREADS, BW_TOTAL, s>>>(A, L.status);
    if ((e = cudaGetLastError())) return e;
  }
  // ---- weight gradients: dW1 = dA1^T X, dW2 = dA2^T H1, dW3 = dA3^T H2
  {
    WgArgs G;
    G.n = L.n;
    G.ld = L.ld;
    G.S = mlp_train_tc_splits(L.n);
    const int chunks = (L.n + WG_CHUNK - 1) / WG_CHUNK;
    G.chunks = (chunks + G.S - 1) / G.S;
    float* part = L.wg_part;
    G.job[0] = WgJob{L.daT[0], L.x16T, 16, part};
    G.job[1] = WgJob{L.daT[1], L.hT[0], H, part + (size_t)G.S * H * 16};
    G.job[2] = WgJob{L.daT[2], L.hT[1], H, part + (size_t)G.S * H * (16 + H)};
    if ((e = cudaFuncSetAttribute(mlp_tc_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, WG_TOTAL))) return e;
    mlp_tc_wgrad_kernel<<<3 * 2 * G.S, THREADS, WG_TOTAL, s>>>(G, L.status);
    if ((e = cudaGetLastError())) return e;
    FinishArgs F;
    F.dW[0] = L.dW1;
    F.dW[1] = L.dW2;
    F.dW[2] = L.dW3;
    for (int l = 0; l < 3; ++l) {
      F.db[l] = L.db[l];
      F.daT[l] = L.daT[l];
    }
    F.dW4 = L.dW4;
    F.db4 = L.db4;
    F.h3T = L.hT[2];
    F.dz = L.dz;
    F.red_blocks = 2 * num_sms;
    const int bias_blocks = (4 * H + 1 + 7) / 8;  // one warp per output, 8 warps per block
    mlp_grad_finish_kernel<<<F.red_blocks + bias_blocks, 256, 0, s>>>(G, F);
    if ((e = cudaGetLastError())) return e;
  }
  return cudaSuccess;
}

}  // namespace sc
