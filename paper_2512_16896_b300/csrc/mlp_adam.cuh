#pragma once
// Packed parameter layout of the reachability surrogate (9 -> 256 -> 256 ->
// 256 -> 1) and its Adam step (Kingma and Ba, Algorithm 1, with the bias
// corrections 1 - beta^t), shared by the standalone Adam kernel and by the
// weight-gradient kernel, which applies the same update to each gradient it
// has just reduced, so both paths give the same bits.
#include <cuda_bf16.h>

#include "common.cuh"

namespace sc {
namespace mlpp {

constexpr int H = 256;   // hidden width
constexpr int KIN = 16;  // 9 input features padded to one k16 step

constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * 9, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + H * H, OFF_W4 = OFF_B3 + H, OFF_B4 = OFF_W4 + H,
              N_PARAMS = OFF_B4 + 1;

// Byte offset of W[o][k] (256 x 256) in the K-sliced copy the inference
// kernel streams: 4 slices of 64 inputs, each 32 KB in the canonical K-major
// layout with K = 64.
__host__ __device__ __forceinline__ uint32_t kslice_offset(int o, int k) {
  return (uint32_t)(k >> 6) * 32768u + canon_offset(o, k & 63, 64);
}

// Adam state and the bf16 weight copies one update writes: W1c, W2c, W3c
// ([out][in], canonical K-major), W2k, W3k (the same, K-sliced), W2tc, W3tc
// ([in][out]), W4 plain.
struct AdamArgs {
  float* params;  // FP32 masters; NULL: no update
  float* m;
  float* v;
  float lr, b1, b2, eps;
  float ibc1, ibc2;  // 1 / (1 - b1^t), 1 / (1 - b2^t) of this step
  __nv_bfloat16* W4;
  __nv_bfloat16* W1c;
  __nv_bfloat16* W2c;
  __nv_bfloat16* W3c;
  __nv_bfloat16* W2k;
  __nv_bfloat16* W3k;
  __nv_bfloat16* W2tc;
  __nv_bfloat16* W3tc;
};

// The Adam arithmetic of one parameter: new moments and value from the
// gradient and the current ones. Every operation is an explicitly rounded
// intrinsic (no contraction left to the compiler), so the update has the
// same bits in every kernel it is inlined into.
__device__ __forceinline__ void adam_core(const AdamArgs& a, float gi, float m0, float v0, float p0, float& mi,
                                          float& vi, float& p) {
  mi = __fmaf_rn(a.b1, m0, __fmul_rn(__fsub_rn(1.f, a.b1), gi));
  vi = __fmaf_rn(a.b2, v0, __fmul_rn(__fmul_rn(__fsub_rn(1.f, a.b2), gi), gi));
  const float mhat = __fmul_rn(mi, a.ibc1), vhat = __fmul_rn(vi, a.ibc2);
  p = __fsub_rn(p0, __fdiv_rn(__fmul_rn(a.lr, mhat), __fadd_rn(__fsqrt_rn(vhat), a.eps)));
}

// The bf16 copies of updated parameter i with value p.
__device__ __forceinline__ void adam_copies(const AdamArgs& a, int i, float p) {
  const __nv_bfloat16 h = __float2bfloat16_rn(p);
  if (i < OFF_B1) {  // W1 [256][9] -> canonical [256][16] (columns 9..15 stay zero)
    a.W1c[canon_offset(i / 9, i % 9, KIN) / 2] = h;
  } else if (i >= OFF_W2 && i < OFF_B2) {
    const int o = (i - OFF_W2) / H, k = (i - OFF_W2) % H;
    a.W2c[canon_offset(o, k, H) / 2] = h;
    a.W2k[kslice_offset(o, k) / 2] = h;
    a.W2tc[canon_offset(k, o, H) / 2] = h;
  } else if (i >= OFF_W3 && i < OFF_B3) {
    const int o = (i - OFF_W3) / H, k = (i - OFF_W3) % H;
    a.W3c[canon_offset(o, k, H) / 2] = h;
    a.W3k[kslice_offset(o, k) / 2] = h;
    a.W3tc[canon_offset(k, o, H) / 2] = h;
  } else if (i >= OFF_W4 && i < OFF_B4) {
    a.W4[i - OFF_W4] = h;
  }
}

// Adam on parameter i with gradient gi, given its current moments and value
// (loaded by the caller, so that several updates can have their loads in
// flight together); stores them and the updated weight's bf16 copies.
__device__ __forceinline__ void adam_apply(const AdamArgs& a, int i, float gi, float m0, float v0, float p0) {
  float mi, vi, p;
  adam_core(a, gi, m0, v0, p0, mi, vi, p);
  a.m[i] = mi;
  a.v[i] = vi;
  a.params[i] = p;
  adam_copies(a, i, p);
}

// Adam on parameter i with gradient gi.
__device__ __forceinline__ void adam_update(const AdamArgs& a, int i, float gi) {
  adam_apply(a, i, gi, a.m[i], a.v[i], a.params[i]);
}

}  // namespace mlpp
}  // namespace sc
