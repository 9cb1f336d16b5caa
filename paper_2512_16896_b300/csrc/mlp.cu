// Reachability surrogate: an MLP 9 -> 256 -> 256 -> 256 -> 1 with SiLU,
// BF16 weights and activations, FP32 accumulation, trained with
// binary-cross-entropy on logits and Adam (the learned gate in front of the
// exact IK check of Sec. IV-E). Features of a target (R row-major, p):
// x = (p, R[:,0], R[:,1]), standardised by the stored mean / std.
//
// Products run on the tensor cores with mma.sync m16n8k16 (bf16 x bf16 ->
// f32). Layouts are chosen so every operand is read in its natural order:
//   forward   out[s][n]  = sum_k h[s][k] W[n][k]     (A = h row-major, B = W [out][in])
//   backward  dh[s][k]   = sum_n da[s][n] W[n][k]    (B = W^T copy [in][out])
//   weights   dW[n][k]   = sum_s daT[n][s] hT[k][s]  (activations kept feature-major)
// Rounding points (matching the FP64 reference): standardised input, every
// SiLU output, W copies, and every dL/da are rounded to bf16; biases,
// pre-activations, accumulations, gradients and Adam state are FP32.
#include <cstring>

#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace sc {

namespace {

constexpr int H = 256;     // hidden width
constexpr int KIN = 16;    // 9 input features padded to one k16 step
constexpr int AST = H + 8; // activation row stride in shared memory (bank spread)

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float sigmoidf_(float a) { return 1.f / (1.f + expf(-a)); }
__device__ __forceinline__ float silu(float a) { return a * sigmoidf_(a); }
__device__ __forceinline__ float silu_grad(float a) {
  const float s = sigmoidf_(a);
  return s * (1.f + a * (1.f - s));
}
__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

struct MlpDev {
  const float* params;        // FP32 masters, packed (see sc_mlp_param_count)
  const __nv_bfloat16* W1;    // [H][KIN] (inputs 9..15 zero)
  const __nv_bfloat16* W2;    // [H][H]   [out][in]
  const __nv_bfloat16* W3;    // [H][H]
  const __nv_bfloat16* W4;    // [H]
  const __nv_bfloat16* W2t;   // [H][H]   [in][out]
  const __nv_bfloat16* W3t;   // [H][H]
  const float* mu;            // [9]
  const float* inv_sigma;     // [9]
};

// packed parameter offsets
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * 9, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + H * H, OFF_W4 = OFF_B3 + H, OFF_B4 = OFF_W4 + H,
              N_PARAMS = OFF_B4 + 1;

// Features of one target (12 floats) for row `row` of a warp's 16-row tile.
__device__ __forceinline__ void features(const float* t, float x[9]) {
  x[0] = t[9]; x[1] = t[10]; x[2] = t[11];
  x[3] = t[0]; x[4] = t[3]; x[5] = t[6];  // R[:,0]
  x[6] = t[1]; x[7] = t[4]; x[8] = t[7];  // R[:,1]
}

// Training caches (feature-major transposes for the weight-gradient products).
struct TrainCache {
  __nv_bfloat16* x16T;  // [KIN][B]
  __nv_bfloat16* h1T;   // [H][B]
  __nv_bfloat16* h2T;
  __nv_bfloat16* h3T;
  float* a1;            // [B][H] pre-activations
  float* a2;
  float* a3;
  int B;                // batch rows (stride of the transposes)
};

// Rows [row0, row0 + 16) of the batch: warp-level forward pass.
// idx(i) maps batch row i to the target index.
template <bool TRAIN>
__device__ void warp_forward(const MlpDev& M, const float* targets, const int32_t* index, int n_rows, int row0,
                             __nv_bfloat16* act0, __nv_bfloat16* act1, float* logits, TrainCache tc, int lane) {
  const int g = lane >> 2, t4 = lane & 3;
  // ---- input features, standardised, bf16, padded to 16
  if (lane < 16) {
    const int row = row0 + lane;
    float x[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (row < n_rows) {
      const int ti = index ? index[row] : row;
      float tt[12];
#pragma unroll
      for (int i = 0; i < 12; ++i) tt[i] = __ldg(targets + 12 * (size_t)ti + i);
      features(tt, x);
#pragma unroll
      for (int i = 0; i < 9; ++i) x[i] = (x[i] - M.mu[i]) * M.inv_sigma[i];
    }
#pragma unroll
    for (int i = 0; i < KIN; ++i) {
      const __nv_bfloat16 v = __float2bfloat16_rn(i < 9 ? x[i] : 0.f);
      act0[lane * AST + i] = v;
      if (TRAIN && row < n_rows) tc.x16T[(size_t)i * tc.B + row] = v;
    }
  }
  __syncwarp();
  const float* b1 = M.params + OFF_B1;
  const float* b2 = M.params + OFF_B2;
  const float* b3 = M.params + OFF_B3;
  // ---- layer 1 (K = 16): act0 -> act1
  {
    uint32_t a[4];
    a[0] = ld32(act0 + g * AST + 2 * t4);
    a[1] = ld32(act0 + (g + 8) * AST + 2 * t4);
    a[2] = ld32(act0 + g * AST + 2 * t4 + 8);
    a[3] = ld32(act0 + (g + 8) * AST + 2 * t4 + 8);
    for (int nt = 0; nt < H / 8; ++nt) {
      const int n = nt * 8 + g;
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      mma_bf16(c, a, ld32(M.W1 + n * KIN + 2 * t4), ld32(M.W1 + n * KIN + 2 * t4 + 8));
      const int col = nt * 8 + 2 * t4;
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int r = g + (h >> 1) * 8, cc = col + (h & 1);
        const float pre = c[h] + b1[cc];
        const __nv_bfloat16 v = __float2bfloat16_rn(silu(pre));
        act1[r * AST + cc] = v;
        if (TRAIN && row0 + r < n_rows) {
          tc.a1[(size_t)(row0 + r) * H + cc] = pre;
          tc.h1T[(size_t)cc * tc.B + row0 + r] = v;
        }
      }
    }
  }
  __syncwarp();
  // ---- layers 2 and 3 (K = 256): act1 -> act0 -> act1
  for (int layer = 0; layer < 2; ++layer) {
    const __nv_bfloat16* W = layer == 0 ? M.W2 : M.W3;
    const float* bias = layer == 0 ? b2 : b3;
    const __nv_bfloat16* src = layer == 0 ? act1 : act0;
    __nv_bfloat16* dst = layer == 0 ? act0 : act1;
    float* a_out = layer == 0 ? tc.a2 : tc.a3;
    __nv_bfloat16* hT = layer == 0 ? tc.h2T : tc.h3T;
    for (int chunk = 0; chunk < H / 64; ++chunk) {
      float c[8][4];
#pragma unroll
      for (int j = 0; j < 8; ++j) c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.f;
#pragma unroll 4
      for (int ks = 0; ks < H / 16; ++ks) {
        const int k0 = ks * 16;
        uint32_t a[4];
        a[0] = ld32(src + g * AST + k0 + 2 * t4);
        a[1] = ld32(src + (g + 8) * AST + k0 + 2 * t4);
        a[2] = ld32(src + g * AST + k0 + 2 * t4 + 8);
        a[3] = ld32(src + (g + 8) * AST + k0 + 2 * t4 + 8);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int n = chunk * 64 + j * 8 + g;
          mma_bf16(c[j], a, __ldg(reinterpret_cast<const unsigned int*>(W + n * H + k0 + 2 * t4)),
                   __ldg(reinterpret_cast<const unsigned int*>(W + n * H + k0 + 2 * t4 + 8)));
        }
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int col = chunk * 64 + j * 8 + 2 * t4;
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const int r = g + (h >> 1) * 8, cc = col + (h & 1);
          const float pre = c[j][h] + bias[cc];
          const __nv_bfloat16 v = __float2bfloat16_rn(silu(pre));
          dst[r * AST + cc] = v;
          if (TRAIN && row0 + r < n_rows) {
            a_out[(size_t)(row0 + r) * H + cc] = pre;
            hT[(size_t)cc * tc.B + row0 + r] = v;
          }
        }
      }
    }
    __syncwarp();
  }
  // ---- layer 4 (K = 256, one output): act1 . W4 + b4 on the CUDA cores
  {
    const int r = lane & 15, half = lane >> 4;
    float acc = 0.f;
    for (int k = half * 128; k < half * 128 + 128; ++k)
      acc = fmaf(__bfloat162float(act1[r * AST + k]), __bfloat162float(M.W4[k]), acc);
    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 16);
    if (half == 0 && row0 + r < n_rows) logits[row0 + r] = acc + M.params[OFF_B4];
  }
  __syncwarp();
}

// Shared memory per warp: two 16 x AST bf16 activation tiles (+ 16 floats
// of dL/dz in the backward kernel).
constexpr int kWarpSmem = 2 * 16 * AST * 2;
constexpr int kWarpSmemBwd = kWarpSmem + 64;

// n_rows_dev (optional): the row count is read from device memory (lists
// produced on the device), n_rows is then only an upper bound.
template <bool TRAIN>
__global__ void __launch_bounds__(128) mlp_forward_kernel(MlpDev M, const float* targets, const int32_t* index,
                                                          int n_rows, const int* n_rows_dev, float* logits,
                                                          TrainCache tc) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, warps = blockDim.x >> 5;
  if (n_rows_dev) n_rows = min(n_rows, *(volatile const int*)n_rows_dev);
  __nv_bfloat16* act0 = reinterpret_cast<__nv_bfloat16*>(smem + w * kWarpSmem);
  __nv_bfloat16* act1 = act0 + 16 * AST;
  for (int row0 = (blockIdx.x * warps + w) * 16; row0 < n_rows; row0 += gridDim.x * warps * 16)
    warp_forward<TRAIN>(M, targets, index, n_rows, row0, act0, act1, logits, tc, lane);
}

// Backward through the activations for rows [row0, row0 + 16): dz, then
// da3 = bf16(bf16(dz) W4 * silu'(a3)), da2 = bf16((da3 W3) * silu'(a2)),
// da1 = bf16((da2 W2) * silu'(a1)); the da are stored feature-major.
struct BwdOut {
  float* dz;             // [B]
  __nv_bfloat16* da1T;   // [H][B]
  __nv_bfloat16* da2T;
  __nv_bfloat16* da3T;
  float* loss_sum;       // scalar (mean BCE accumulated as sum / B)
};

__global__ void __launch_bounds__(128) mlp_backward_act_kernel(MlpDev M, const float* logits, const uint8_t* labels,
                                                               const int32_t* index, int n_rows, float inv_n,
                                                               TrainCache tc, BwdOut o) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, warps = blockDim.x >> 5;
  const int g = lane >> 2, t4 = lane & 3;
  __nv_bfloat16* da = reinterpret_cast<__nv_bfloat16*>(smem + w * kWarpSmemBwd);  // [16][AST] current dL/da
  __nv_bfloat16* dn = da + 16 * AST;                                              // [16][AST] next dL/da
  float* dzs = reinterpret_cast<float*>(smem + w * kWarpSmemBwd + 2 * 16 * AST * 2);  // [16]
  for (int row0 = (blockIdx.x * warps + w) * 16; row0 < n_rows; row0 += gridDim.x * warps * 16) {
    // dz and the loss
    float loss = 0.f;
    if (lane < 16) {
      const int row = row0 + lane;
      float dz = 0.f;
      if (row < n_rows) {
        const float z = logits[row];
        const float y = labels[index ? index[row] : row] ? 1.f : 0.f;
        dz = (sigmoidf_(z) - y) * inv_n;
        loss = fmaxf(z, 0.f) - z * y + log1pf(expf(-fabsf(z)));
        o.dz[row] = dz;
      }
      dzs[lane] = dz;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) loss += __shfl_xor_sync(0xFFFFFFFFu, loss, off);
    if (lane == 0) atomicAdd(o.loss_sum, loss * inv_n);
    __syncwarp();
    // da3 (CUDA cores): element (r, n)
    for (int e = lane; e < 16 * H; e += 32) {
      const int r = e / H, n = e % H;
      const bool in = row0 + r < n_rows;
      float v = 0.f;
      if (in) {
        const float dh = bf16r(dzs[r]) * __bfloat162float(M.W4[n]);
        v = dh * silu_grad(tc.a3[(size_t)(row0 + r) * H + n]);
      }
      const __nv_bfloat16 b = __float2bfloat16_rn(v);
      da[r * AST + n] = b;
      if (in) o.da3T[(size_t)n * tc.B + row0 + r] = b;
    }
    __syncwarp();
    // da2 from da3 W3, then da1 from da2 W2 (tensor cores), 64 columns at a time
    for (int layer = 0; layer < 2; ++layer) {
      const __nv_bfloat16* Wt = layer == 0 ? M.W3t : M.W2t;
      const float* a_pre = layer == 0 ? tc.a2 : tc.a1;
      __nv_bfloat16* outT = layer == 0 ? o.da2T : o.da1T;
      const __nv_bfloat16* src = layer == 0 ? da : dn;
      __nv_bfloat16* dst = layer == 0 ? dn : da;
      for (int chunk = 0; chunk < H / 64; ++chunk) {
        float acc[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll 4
        for (int ks = 0; ks < H / 16; ++ks) {
          const int k0 = ks * 16;
          uint32_t a[4];
          a[0] = ld32(src + g * AST + k0 + 2 * t4);
          a[1] = ld32(src + (g + 8) * AST + k0 + 2 * t4);
          a[2] = ld32(src + g * AST + k0 + 2 * t4 + 8);
          a[3] = ld32(src + (g + 8) * AST + k0 + 2 * t4 + 8);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int n = chunk * 64 + j * 8 + g;
            mma_bf16(acc[j], a, __ldg(reinterpret_cast<const unsigned int*>(Wt + n * H + k0 + 2 * t4)),
                     __ldg(reinterpret_cast<const unsigned int*>(Wt + n * H + k0 + 2 * t4 + 8)));
          }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int col = chunk * 64 + j * 8 + 2 * t4;
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const int r = g + (h >> 1) * 8, cc = col + (h & 1);
            const bool in = row0 + r < n_rows;
            const float v = in ? acc[j][h] * silu_grad(a_pre[(size_t)(row0 + r) * H + cc]) : 0.f;
            const __nv_bfloat16 b = __float2bfloat16_rn(v);
            dst[r * AST + cc] = b;
            if (in) outT[(size_t)cc * tc.B + row0 + r] = b;
          }
        }
      }
      __syncwarp();
    }
  }
}

// dW[n][k] = sum_s daT[n][s] hT[k][s] for one layer; one CTA per 16 x 64
// tile (n0, k0), K = batch rows padded to a multiple of 16 with zeros. The
// CTA's kWgSplit warps take every kWgSplit-th 16-row step of the batch, so a
// tile's serial chain is kWgSplit times shorter; their partial sums are added
// in warp order through shared memory (the same order on every run).
constexpr int kWgSplit = 8;

__global__ void __launch_bounds__(32 * kWgSplit) mlp_weight_grad_kernel(const __nv_bfloat16* daT,
                                                                         const __nv_bfloat16* hT, int n_out, int n_in,
                                                                         int B, int Bpad, float* dW, int dW_stride,
                                                                         int n_in_store) {
  __shared__ float part[kWgSplit][16 * 64];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int g = lane >> 2, t4 = lane & 3;
  const int tiles_n = n_out / 16, tiles_k = (n_in + 63) / 64;
  for (int tile = blockIdx.x; tile < tiles_n * tiles_k; tile += gridDim.x) {
    const int n0 = (tile / tiles_k) * 16, k0 = (tile % tiles_k) * 64;
    const int nk = min(64, n_in - k0) / 8;  // n-tiles of 8 in this chunk (n_in is a multiple of 8)
    float c[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.f;
    for (int s0 = w * 16; s0 < Bpad; s0 += 16 * kWgSplit) {
      uint32_t a[4];
      a[0] = ld32(daT + (size_t)(n0 + g) * B + s0 + 2 * t4);
      a[1] = ld32(daT + (size_t)(n0 + g + 8) * B + s0 + 2 * t4);
      a[2] = ld32(daT + (size_t)(n0 + g) * B + s0 + 2 * t4 + 8);
      a[3] = ld32(daT + (size_t)(n0 + g + 8) * B + s0 + 2 * t4 + 8);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (j < nk) {
          const int k = k0 + j * 8 + g;
          mma_bf16(c[j], a, ld32(hT + (size_t)k * B + s0 + 2 * t4), ld32(hT + (size_t)k * B + s0 + 2 * t4 + 8));
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (j < nk) {
#pragma unroll
        for (int h = 0; h < 4; ++h) part[w][(g + (h >> 1) * 8) * 64 + j * 8 + 2 * t4 + (h & 1)] = c[j][h];
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 16 * 64; e += blockDim.x) {
      const int r = e >> 6, cc = e & 63;
      if (cc < nk * 8 && k0 + cc < n_in_store) {
        float v = part[0][e];
#pragma unroll
        for (int q = 1; q < kWgSplit; ++q) v += part[q][e];
        dW[(size_t)(n0 + r) * dW_stride + k0 + cc] = v;
      }
    }
    __syncthreads();  // part is reused by the CTA's next tile
  }
}

// Bias gradients (row sums of daT), dW4 = hT3 . dz and db4 = sum dz.
__global__ void mlp_bias_grad_kernel(const __nv_bfloat16* da1T, const __nv_bfloat16* da2T, const __nv_bfloat16* da3T,
                                     const __nv_bfloat16* h3T, const float* dz, int B, int ld, float* grads) {
  // rows 0..H-1: db1, H..2H-1: db2, 2H..3H-1: db3, 3H..4H-1: dW4, 4H: db4
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, warps = blockDim.x >> 5;
  for (int row = blockIdx.x * warps + w; row <= 4 * H; row += gridDim.x * warps) {
    float acc = 0.f;
    if (row < 3 * H) {
      const __nv_bfloat16* src = row < H ? da1T : row < 2 * H ? da2T : da3T;
      const __nv_bfloat16* p = src + (size_t)(row % H) * ld;
      for (int s = lane; s < B; s += 32) acc += __bfloat162float(p[s]);
    } else if (row < 4 * H) {
      const __nv_bfloat16* p = h3T + (size_t)(row - 3 * H) * ld;
      for (int s = lane; s < B; s += 32) acc = fmaf(__bfloat162float(p[s]), dz[s], acc);
    } else {
      for (int s = lane; s < B; s += 32) acc += dz[s];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, off);
    if (lane == 0) {
      const int dst = row < H ? OFF_B1 + row : row < 2 * H ? OFF_B2 + row - H : row < 3 * H ? OFF_B3 + row - 2 * H
                      : row < 4 * H ? OFF_W4 + row - 3 * H : OFF_B4;
      grads[dst] = acc;
    }
  }
}

// Adam on the FP32 masters (step t, 1-based), then the bf16 compute copies.
__global__ void mlp_adam_kernel(float* params, const float* grads, float* m, float* v, int n, float lr, float b1,
                                float b2, float eps, float bc1, float bc2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = grads[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    params[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

// bf16 copies of the weights: row-major [out][in] (training forward), the
// transposes (backward) and the canonical tensor-core layout (inference).
__global__ void mlp_copies_kernel(const float* params, __nv_bfloat16* W1, __nv_bfloat16* W2, __nv_bfloat16* W3,
                                  __nv_bfloat16* W4, __nv_bfloat16* W2t, __nv_bfloat16* W3t, __nv_bfloat16* W1c,
                                  __nv_bfloat16* W2c, __nv_bfloat16* W3c) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < H * H; i += gridDim.x * blockDim.x) {
    const int n = i / H, k = i % H;
    const __nv_bfloat16 w2 = __float2bfloat16_rn(params[OFF_W2 + i]);
    const __nv_bfloat16 w3 = __float2bfloat16_rn(params[OFF_W3 + i]);
    W2[i] = w2;
    W3[i] = w3;
    W2t[k * H + n] = w2;
    W3t[k * H + n] = w3;
    W2c[canon_offset(n, k, H) / 2] = w2;
    W3c[canon_offset(n, k, H) / 2] = w3;
    if (i < H * KIN) {
      const int n1 = i / KIN, k1 = i % KIN;
      const __nv_bfloat16 w1 = __float2bfloat16_rn(k1 < 9 ? params[OFF_W1 + n1 * 9 + k1] : 0.f);
      W1[i] = w1;
      W1c[canon_offset(n1, k1, KIN) / 2] = w1;
    }
    if (i < H) W4[i] = __float2bfloat16_rn(params[OFF_W4 + i]);
  }
}

// Per-feature sums and sums of squares (double) of the training targets.
__global__ void feature_moments_kernel(const float* targets, int n, double* acc /*[18]*/) {
  double s[9] = {0}, s2[9] = {0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float tt[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) tt[j] = targets[12 * (size_t)i + j];
    float x[9];
    features(tt, x);
#pragma unroll
    for (int j = 0; j < 9; ++j) { s[j] += x[j]; s2[j] += (double)x[j] * x[j]; }
  }
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    for (int off = 16; off > 0; off >>= 1) {
      s[j] += __shfl_xor_sync(0xFFFFFFFFu, s[j], off);
      s2[j] += __shfl_xor_sync(0xFFFFFFFFu, s2[j], off);
    }
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int j = 0; j < 9; ++j) { atomicAdd(&acc[j], s[j]); atomicAdd(&acc[9 + j], s2[j]); }
  }
}

__global__ void feature_norm_kernel(const double* acc, int n, float* mu, float* inv_sigma) {
  const int j = threadIdx.x;
  if (j < 9) {
    const double m = acc[j] / n;
    const double var = acc[9 + j] / n - m * m;
    const double sd = var > 1e-12 ? sqrt(var) : 1.0;  // a constant feature keeps unit scale
    mu[j] = (float)m;
    inv_sigma[j] = (float)(1.0 / sd);
  }
}

// Batch rows of an epoch: an affine permutation i -> (a i + c) mod n with
// gcd(a, n) = 1, a and c drawn from Philox (epoch-wise shuffling).
__global__ void epoch_index_kernel(int n, uint64_t a, uint64_t c, int32_t* index) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    index[i] = (int32_t)((a * (uint64_t)i + c) % (uint64_t)n);
}

// U(-1/sqrt(fan_in), 1/sqrt(fan_in)) initial weights and biases from Philox.
__global__ void mlp_init_kernel(float* params, uint64_t seed) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N_PARAMS; i += gridDim.x * blockDim.x) {
    const int fan_in = i < OFF_W2 ? 9 : i < OFF_W4 ? H : H;
    const float kk = rsqrtf((float)fan_in);
    const float4 u = draw_uniform4(seed, (uint32_t)i, 0x4D4C50u, 0u, 0u);
    params[i] = kk * (2.f * u.x - 1.f);
  }
}

}  // namespace

// ------------------------------------------------------------------ host side

int mlp_param_count() { return N_PARAMS; }

struct MlpState {
  float* params = nullptr;  // device, FP32 masters
  float* m = nullptr;
  float* v = nullptr;
  float* grads = nullptr;
  __nv_bfloat16 *W1 = nullptr, *W2 = nullptr, *W3 = nullptr, *W4 = nullptr, *W2t = nullptr, *W3t = nullptr;
  __nv_bfloat16 *W1c = nullptr, *W2c = nullptr, *W3c = nullptr;  // canonical tensor-core layout (inference)
  float* mu = nullptr;
  float* inv_sigma = nullptr;
  double* moments = nullptr;
  int64_t step = 0;
  // training scratch for a batch of Bcap rows
  int Bcap = 0;
  void* train_buf = nullptr;
};

static MlpDev dev_view(const MlpState& S) {
  MlpDev d;
  d.params = S.params;
  d.W1 = S.W1; d.W2 = S.W2; d.W3 = S.W3; d.W4 = S.W4; d.W2t = S.W2t; d.W3t = S.W3t;
  d.mu = S.mu;
  d.inv_sigma = S.inv_sigma;
  return d;
}

cudaError_t mlp_alloc(MlpState** out) {
  MlpState* S = new (std::nothrow) MlpState;
  if (!S) return cudaErrorMemoryAllocation;
  const size_t nf = N_PARAMS;
  cudaError_t e;
  if ((e = cudaMalloc(&S->params, nf * 4)) || (e = cudaMalloc(&S->m, nf * 4)) || (e = cudaMalloc(&S->v, nf * 4)) ||
      (e = cudaMalloc(&S->grads, nf * 4)) || (e = cudaMalloc(&S->W1, H * KIN * 2)) ||
      (e = cudaMalloc(&S->W2, H * H * 2)) || (e = cudaMalloc(&S->W3, H * H * 2)) || (e = cudaMalloc(&S->W4, H * 2)) ||
      (e = cudaMalloc(&S->W2t, H * H * 2)) || (e = cudaMalloc(&S->W3t, H * H * 2)) ||
      (e = cudaMalloc(&S->W1c, H * KIN * 2)) || (e = cudaMalloc(&S->W2c, H * H * 2)) ||
      (e = cudaMalloc(&S->W3c, H * H * 2)) || (e = cudaMalloc(&S->mu, 64)) ||
      (e = cudaMalloc(&S->inv_sigma, 64)) || (e = cudaMalloc(&S->moments, 18 * 8))) {
    mlp_free(S);
    return e;
  }
  *out = S;
  return cudaSuccess;
}

void mlp_free(MlpState* S) {
  if (!S) return;
  void* ptrs[] = {S->params, S->m,   S->v,   S->grads, S->W1, S->W2,        S->W3,      S->W4,
                  S->W2t,    S->W3t, S->W1c, S->W2c, S->W3c,  S->mu, S->inv_sigma, S->moments, S->train_buf};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete S;
}

cudaError_t mlp_refresh_copies(MlpState* S, cudaStream_t s) {
  mlp_copies_kernel<<<128, 256, 0, s>>>(S->params, S->W1, S->W2, S->W3, S->W4, S->W2t, S->W3t, S->W1c, S->W2c,
                                         S->W3c);
  return cudaGetLastError();
}

cudaError_t mlp_init(MlpState* S, uint64_t seed, cudaStream_t s) {
  mlp_init_kernel<<<128, 256, 0, s>>>(S->params, seed);
  cudaError_t e;
  if ((e = cudaMemsetAsync(S->m, 0, N_PARAMS * 4, s)) || (e = cudaMemsetAsync(S->v, 0, N_PARAMS * 4, s))) return e;
  const float zeros[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, ones[9] = {1, 1, 1, 1, 1, 1, 1, 1, 1};
  if ((e = cudaMemcpyAsync(S->mu, zeros, 36, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(S->inv_sigma, ones, 36, cudaMemcpyHostToDevice, s)))
    return e;
  S->step = 0;
  return mlp_refresh_copies(S, s);
}

cudaError_t mlp_set_norm_from(MlpState* S, const float* targets, int n, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(S->moments, 0, 18 * 8, s);
  if (e) return e;
  feature_moments_kernel<<<256, 256, 0, s>>>(targets, n, S->moments);
  feature_norm_kernel<<<1, 32, 0, s>>>(S->moments, n, S->mu, S->inv_sigma);
  return cudaGetLastError();
}

// Kernels that take more than 48 KB of dynamic shared memory opt in once.
static cudaError_t smem_opt_in() {
  cudaError_t e =
      cudaFuncSetAttribute(mlp_forward_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * kWarpSmem);
  if (!e)
    e = cudaFuncSetAttribute(mlp_backward_act_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * kWarpSmemBwd);
  return e;
}

static MlpTcWeights tc_view(const MlpState& S);
MlpTcWeights mlp_tc_weights(const MlpState* S) { return tc_view(*S); }

static MlpTcWeights tc_view(const MlpState& S) {
  MlpTcWeights w;
  w.params = S.params;
  w.W1c = S.W1c;
  w.W2c = S.W2c;
  w.W3c = S.W3c;
  w.W4 = S.W4;
  w.mu = S.mu;
  w.inv_sigma = S.inv_sigma;
  w.off_b1 = OFF_B1;
  w.off_b2 = OFF_B2;
  w.off_b3 = OFF_B3;
  w.off_b4 = OFF_B4;
  return w;
}

// Inference runs on tcgen05 (mlp_tc.cu); the mma.sync forward above serves
// training, where the pre-activations and transposed caches are written too.
cudaError_t mlp_infer(const MlpState* S, const float* targets, int n, float* logits, int* status, int num_sms,
                      cudaStream_t s) {
  return mlp_forward_tc(tc_view(*S), targets, n, nullptr, logits, status, num_sms, s);
}

cudaError_t mlp_infer_counted(const MlpState* S, const float* targets, const int* n_dev, int n_cap, float* logits,
                              int* status, int num_sms, cudaStream_t s) {
  return mlp_forward_tc(tc_view(*S), targets, n_cap, n_dev, logits, status, num_sms, s);
}

// Batch buffers: caches + backward outputs for Bcap rows.
static size_t train_bytes(int Bcap) {
  const size_t Bp = (size_t)Bcap;
  return Bp * KIN * 2 + 3 * Bp * H * 2 + 3 * Bp * H * 4 + 3 * Bp * H * 2 + Bp * 4 + Bp * 4 + 1024;
}

struct TrainViews {
  TrainCache tc;
  BwdOut bo;
  float* logits;
};

static TrainViews carve(MlpState* S, int Bcap) {
  char* p = static_cast<char*>(S->train_buf);
  auto take = [&](size_t bytes) { char* r = p; p += (bytes + 255) & ~size_t(255); return r; };
  TrainViews v;
  v.tc.B = Bcap;
  v.tc.x16T = reinterpret_cast<__nv_bfloat16*>(take((size_t)Bcap * KIN * 2));
  v.tc.h1T = reinterpret_cast<__nv_bfloat16*>(take((size_t)Bcap * H * 2));
  v.tc.h2T = reinterpret_cast<__nv_bfloat16*>(take((size_t)Bcap * H * 2));
  v.tc.h3T = reinterpret_cast<__nv_bfloat16*>(take((size_t)Bcap * H * 2));
  v.tc.a1 = reinterpret_cast<float*>(take((size_t)Bcap * H * 4));
  v.tc.a2 = reinterpret_cast<float*>(take((size_t)Bcap * H * 4));
  v.tc.a3 = reinterpret_cast<float*>(take((size_t)Bcap * H * 4));
  v.bo.da1T = reinterpret_cast<__nv_bfloat16*>(take((size_t)Bcap * H * 2));
  v.bo.da2T = reinterpret_cast<__nv_bfloat16*>(take((size_t)Bcap * H * 2));
  v.bo.da3T = reinterpret_cast<__nv_bfloat16*>(take((size_t)Bcap * H * 2));
  v.bo.dz = reinterpret_cast<float*>(take((size_t)Bcap * 4));
  v.logits = reinterpret_cast<float*>(take((size_t)Bcap * 4));
  v.bo.loss_sum = reinterpret_cast<float*>(take(256));
  return v;
}

cudaError_t mlp_reserve(MlpState* S, int Bcap) {
  Bcap = (Bcap + 15) & ~15;
  if (Bcap <= S->Bcap) return cudaSuccess;
  if (S->train_buf) cudaFree(S->train_buf);
  S->train_buf = nullptr;
  S->Bcap = 0;
  cudaError_t e = cudaMalloc(&S->train_buf, train_bytes(Bcap) + 16 * 256);
  if (e) return e;
  S->Bcap = Bcap;
  return cudaSuccess;
}

// Gradients of the mean BCE over rows index[0..B) into S->grads (packed).
// Caches are zero-filled past B so the padded rows contribute nothing.
cudaError_t mlp_gradients(MlpState* S, const float* targets, const uint8_t* labels, const int32_t* index, int B,
                          float* loss_dev, int num_sms, cudaStream_t s) {
  const int Bpad = (B + 15) & ~15;
  if (Bpad > S->Bcap) return cudaErrorInvalidValue;
  if (cudaError_t e = smem_opt_in()) return e;
  TrainViews v = carve(S, S->Bcap);
  v.tc.B = S->Bcap;
  cudaError_t e;
  // zero the transposed caches (padded rows must read as zero)
  if ((e = cudaMemsetAsync(S->train_buf, 0, train_bytes(S->Bcap), s))) return e;
  v.bo.loss_sum = loss_dev ? loss_dev : v.bo.loss_sum;
  if (loss_dev && (e = cudaMemsetAsync(loss_dev, 0, 4, s))) return e;
  const int warps = 4, rows_per_block = warps * 16;
  int blocks = (B + rows_per_block - 1) / rows_per_block;
  if (blocks > num_sms * 8) blocks = num_sms * 8;
  const MlpDev M = dev_view(*S);
  mlp_forward_kernel<true><<<blocks, warps * 32, warps * kWarpSmem, s>>>(M, targets, index, B, nullptr, v.logits,
                                                                          v.tc);
  mlp_backward_act_kernel<<<blocks, warps * 32, warps * kWarpSmemBwd, s>>>(M, v.logits, labels, index, B, 1.f / B,
                                                                            v.tc, v.bo);
  const int ld = S->Bcap;
  // dW1 [256][9] from da1T . x16T, dW2, dW3
  // one CTA per 16 x 64 tile of each weight gradient
  const int wg_tiles_1 = (H / 16) * ((KIN + 63) / 64), wg_tiles_h = (H / 16) * ((H + 63) / 64);
  mlp_weight_grad_kernel<<<wg_tiles_1, 32 * kWgSplit, 0, s>>>(v.bo.da1T, v.tc.x16T, H, KIN, ld, Bpad,
                                                              S->grads + OFF_W1, 9, 9);
  mlp_weight_grad_kernel<<<wg_tiles_h, 32 * kWgSplit, 0, s>>>(v.bo.da2T, v.tc.h1T, H, H, ld, Bpad,
                                                              S->grads + OFF_W2, H, H);
  mlp_weight_grad_kernel<<<wg_tiles_h, 32 * kWgSplit, 0, s>>>(v.bo.da3T, v.tc.h2T, H, H, ld, Bpad,
                                                              S->grads + OFF_W3, H, H);
  mlp_bias_grad_kernel<<<64, 256, 0, s>>>(v.bo.da1T, v.bo.da2T, v.bo.da3T, v.tc.h3T, v.bo.dz, B, ld, S->grads);
  return cudaGetLastError();
}

cudaError_t mlp_adam(MlpState* S, float lr, float b1, float b2, float eps, cudaStream_t s) {
  S->step += 1;
  const double t = (double)S->step;
  mlp_adam_kernel<<<128, 256, 0, s>>>(S->params, S->grads, S->m, S->v, N_PARAMS, lr, b1, b2, eps,
                                      (float)(1.0 - pow((double)b1, t)), (float)(1.0 - pow((double)b2, t)));
  cudaError_t e = cudaGetLastError();
  if (e) return e;
  return mlp_refresh_copies(S, s);
}

// Epoch shuffle: i -> (a i + c) mod n, a odd and coprime with n, both taken
// from a 64-bit mix of (seed, epoch).
cudaError_t mlp_epoch_index(int n, uint64_t seed, int epoch, int32_t* index, cudaStream_t s) {
  uint64_t x = seed * 0x9E3779B97F4A7C15ull + (uint64_t)(epoch + 1) * 0xBF58476D1CE4E5B9ull;
  x ^= x >> 31;
  x *= 0x94D049BB133111EBull;
  x ^= x >> 29;
  auto gcd = [](uint64_t p, uint64_t q) {
    while (q) { const uint64_t r = p % q; p = q; q = r; }
    return p;
  };
  uint64_t a = (x % (uint64_t)n) | 1u;
  while (gcd(a, (uint64_t)n) != 1) a = ((a + 2) % (uint64_t)n) | 1u;
  const uint64_t c = (x >> 23) % (uint64_t)n;
  epoch_index_kernel<<<256, 256, 0, s>>>(n, a, c, index);
  return cudaGetLastError();
}

float* mlp_params_ptr(MlpState* S) { return S->params; }
float* mlp_grads_ptr(MlpState* S) { return S->grads; }
float* mlp_mu_ptr(MlpState* S) { return S->mu; }
float* mlp_inv_sigma_ptr(MlpState* S) { return S->inv_sigma; }
float* mlp_m_ptr(MlpState* S) { return S->m; }
float* mlp_v_ptr(MlpState* S) { return S->v; }
int64_t mlp_step(const MlpState* S) { return S->step; }
void mlp_set_step(MlpState* S, int64_t t) { S->step = t; }

}  // namespace sc
