// Device-side helpers shared by the kernels of libsceniris_b300.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sceniris.h"

namespace sc {

constexpr float kBand = 1e-5f;                       // decision band (metres)
constexpr float kTwoPi = 6.28318530717958647692f;
constexpr float kFarSentinel = 1e18f;                // "no distance seen yet"
constexpr float kBroadMargin = 1e-3f;                // object-level culling slack (metres), >> kBand + FP32 error
constexpr int kMaxObj = 256;                         // object ids fit in a byte
constexpr int kMaxSph = 8192;                        // spheres of one template
constexpr int kMaxSphPerObj = 256;                   // spheres of one object (generation)
constexpr int kMaxPolyVerts = 64;
constexpr int kMaxObbPerTemplate = 64;
constexpr int kMaxParts = 16;                        // articulated parts of one template

// Device status codes latched into the context's status word (first error wins).
enum DeviceError : int {
  kDevOk = 0,
  kDevBadTemplate = 1,   // candidate index outside every template range
  kDevTooManySpheres = 2,
  kDevTooManyObjects = 3,
  kDevTooManyBoxes = 4,
  kDevBadPolygon = 5,
  kDevBadRelation = 6,  // relation refers to itself or a later object
  kDevTimeout = 7,      // a bounded wait on a tensor-core MMA or bulk copy gave up
  kDevBadPart = 8,      // a box or an INSIDE relation names a part its template does not have
  kDevTooManyTriangles = 9,
};

// Byte offset of element (r, k) of a [rows][K] bf16 matrix in the canonical
// no-swizzle K-major layout of the tensor cores: core matrices of 8 rows x 16
// bytes, adjacent core matrices along K 128 bytes apart, 8-row groups
// K / 8 * 128 bytes apart.
__host__ __device__ __forceinline__ uint32_t canon_offset(int r, int k, int K) {
  return (uint32_t)((r >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void latch_error(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// Philox4x32-10 as published by Salmon, Moraes, Dror and Shaw (SC'11): ten
// rounds of two 32x32->64 multiplications whose high halves are mixed with the
// other counter words and the round key, the key advanced by the Weyl
// constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
    uint32_t hi_a = __umulhi(m0, x.x), lo_a = m0 * x.x;
    uint32_t hi_b = __umulhi(m1, x.z), lo_b = m1 * x.z;
    x = make_uint4(hi_b ^ x.y ^ k0, lo_b, hi_a ^ x.w ^ k1, lo_a);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return x;
}

// sin and cos of a bounded angle (the callers pass yaws the sampler drew in
// [0, 2 pi) and joint angles clamped to their limits; valid for |x| < 2^20): Cody
// and Waite's additive range reduction x = j (pi/2) + r with pi/2 split into
// its float value and the remainder, |r| <= pi/4, then minimax polynomials
// on that interval, sin r = r + r^3 (s1 + s2 r^2 + s3 r^4) (relative error
// 3.8e-9) and cos r = 1 + r^2 (c1 + ... + c4 r^6) (absolute error 5.4e-11),
// from a Remez exchange (sincos_minimax.py), and the quadrant rotation by j.
// Error within 1.5 float ulps of the result.
namespace cw {
constexpr float kTwoOverPi = 0.63661977236758134f;
constexpr float kPio2Hi = 1.57079637050628662f;  // float(pi/2) = pi/2 + 4.371139e-8
constexpr float kPio2Lo = 4.37113900630947700e-8f;
constexpr float kS1 = -0.16666654609547418f, kS2 = 0.0083321607618011673f, kS3 = -0.00019515283185388041f;
constexpr float kC1 = -0.49999999725108215f, kC2 = 0.041666623324343622f, kC3 = -0.0013886763794352274f,
                kC4 = 2.4390450701653411e-5f;

// sin and cos of j (pi/2) + r from sin r, cos r.
__device__ __forceinline__ void quadrant(float j, float sn, float cs, float* s, float* c) {
  const int q = (int)j;
  const float s1 = (q & 1) ? cs : sn, c1 = (q & 1) ? sn : cs;
  *s = (q & 2) ? -s1 : s1;
  *c = ((q + 1) & 2) ? -c1 : c1;
}
}  // namespace cw

__device__ __forceinline__ void sincos_cw(float x, float* s, float* c) {
  const float j = rintf(x * cw::kTwoOverPi);  // nearest multiple of pi/2
  float r = fmaf(j, -cw::kPio2Hi, x);
  r = fmaf(j, cw::kPio2Lo, r);
  const float r2 = r * r;
  float ps = fmaf(cw::kS3, r2, cw::kS2);
  ps = fmaf(ps, r2, cw::kS1);
  const float sn = fmaf(ps * r2, r, r);
  float pc = fmaf(cw::kC4, r2, cw::kC3);
  pc = fmaf(pc, r2, cw::kC2);
  pc = fmaf(pc, r2, cw::kC1);
  const float cs = fmaf(pc, r2, 1.f);
  cw::quadrant(j, sn, cs, s, c);
}

// sincos_cw of two angles at once: the reduction and both series on the
// packed two-lane FP32 instructions, each lane rounding as the scalar form
// (the same bits as two sincos_cw calls).
__device__ __forceinline__ void sincos_cw2(float2 x, float2* s, float2* c) {
  float2 j = __fmul2_rn(x, make_float2(cw::kTwoOverPi, cw::kTwoOverPi));
  j.x = rintf(j.x);
  j.y = rintf(j.y);
  float2 r = __ffma2_rn(j, make_float2(-cw::kPio2Hi, -cw::kPio2Hi), x);
  r = __ffma2_rn(j, make_float2(cw::kPio2Lo, cw::kPio2Lo), r);
  const float2 r2 = __fmul2_rn(r, r);
  float2 ps = __ffma2_rn(make_float2(cw::kS3, cw::kS3), r2, make_float2(cw::kS2, cw::kS2));
  ps = __ffma2_rn(ps, r2, make_float2(cw::kS1, cw::kS1));
  const float2 sn = __ffma2_rn(__fmul2_rn(ps, r2), r, r);
  float2 pc = __ffma2_rn(make_float2(cw::kC4, cw::kC4), r2, make_float2(cw::kC3, cw::kC3));
  pc = __ffma2_rn(pc, r2, make_float2(cw::kC2, cw::kC2));
  pc = __ffma2_rn(pc, r2, make_float2(cw::kC1, cw::kC1));
  const float2 cs = __ffma2_rn(pc, r2, make_float2(1.f, 1.f));
  cw::quadrant(j.x, sn.x, cs.x, &s->x, &c->x);
  cw::quadrant(j.y, sn.y, cs.y, &s->y, &c->y);
}

// Uniform float in [0, 1) from the top 24 bits of a word (exact in FP32).
__device__ __forceinline__ float unit_float(uint32_t w) { return (float)(w >> 8) * 5.9604644775390625e-8f; }

__device__ __forceinline__ float4 draw_uniform4(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3) {
  uint4 w = philox4x32_10(make_uint4(c0, c1, c2, c3), (uint32_t)seed, (uint32_t)(seed >> 32));
  return make_float4(unit_float(w.x), unit_float(w.y), unit_float(w.z), unit_float(w.w));
}

// Template owning candidate c: last t with cand_tmpl_off[t] <= c (binary search).
__device__ __forceinline__ int template_of(const sc_scene_batch& b, int c) {
  int lo = 0, hi = b.n_templates;  // invariant: off[lo] <= c < off[hi]
  if (c < 0 || c >= b.cand_tmpl_off[b.n_templates]) return -1;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(&b.cand_tmpl_off[mid]) <= c) lo = mid; else hi = mid;
  }
  return lo;
}

// Displacement q * axis of world box `box` (a batch index) for candidate c of
// template t: nonzero only for a box of an articulated part (obb_part >= 0),
// q being that part's joint value of the candidate. A part index outside the
// template's parts latches kDevBadPart (when status is given), sets *bad
// (when given) and leaves the box where it is.
__device__ __forceinline__ float3 box_shift(const sc_scene_batch& b, int t, int c, int box, int* status,
                                            bool* bad = nullptr) {
  float3 s = make_float3(0.f, 0.f, 0.f);
  if (!b.obb_part || b.max_parts <= 0) return s;
  const int p = __ldg(&b.obb_part[box]);
  if (p < 0) return s;
  const int p0 = __ldg(&b.tmpl_part_off[t]);
  if (p >= __ldg(&b.tmpl_part_off[t + 1]) - p0 || p >= b.max_parts) {
    latch_error(status, kDevBadPart);
    if (bad) *bad = true;
    return s;
  }
  const float q = __ldg(&b.part_q[(int64_t)c * b.max_parts + p]);
  const float* a = b.part_param + 12 * (int64_t)(p0 + p);
  s.x = q * __ldg(a);
  s.y = q * __ldg(a + 1);
  s.z = q * __ldg(a + 2);
  return s;
}

// Order-preserving map of a float onto a signed int (for atomicMin on floats).
__device__ __forceinline__ int float_key(float f) {
  int i = __float_as_int(f);
  return i >= 0 ? i : (i ^ 0x7FFFFFFF);
}
__device__ __forceinline__ float key_float(int k) {
  return __int_as_float(k >= 0 ? k : (k ^ 0x7FFFFFFF));
}

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
  return v;
}

}  // namespace sc
