// Sphere against world triangle meshes: the squared distance from a point to
// a filled triangle, shared by the collision kernel and the generation step.
#pragma once

#include "common.cuh"

namespace sc {

constexpr int kMaxTriPerTemplate = 65536;

struct Tri {
  float3 a, b, c;
};

// Triangles are also grouped per template in chunks of 32 consecutive ones;
// chunk j of template t (first triangle tq0) has the table slot
// tq0 / 32 + t + j, a layout without collisions in at most
// n_tri / 32 + n_templates + 1 slots (template t's chunks touch at most as
// many 32-aligned blocks as they cover, so its last slot stays below the
// next template's first).
__host__ __device__ __forceinline__ int tri_chunk_slot(int tq0, int t, int j) { return tq0 / 32 + t + j; }
__host__ __device__ __forceinline__ size_t tri_chunk_slots(const sc_scene_batch& b) {
  return b.n_tri > 0 ? (size_t)b.n_tri / 32 + (size_t)b.n_templates + 1 : 0;
}

// Triangle q of the batch, its vertices relative to `ref`.
__device__ __forceinline__ Tri load_tri(const float* tri, int q, float3 ref) {
  const float4* t = reinterpret_cast<const float4*>(tri) + 3 * (int64_t)q;
  const float4 a = __ldg(t), b = __ldg(t + 1), c = __ldg(t + 2);
  Tri r;
  r.a = make_float3(a.x - ref.x, a.y - ref.y, a.z - ref.z);
  r.b = make_float3(b.x - ref.x, b.y - ref.y, b.z - ref.z);
  r.c = make_float3(c.x - ref.x, c.y - ref.y, c.z - ref.z);
  return r;
}

__device__ __forceinline__ float dot3(float3 u, float3 v) { return u.x * v.x + u.y * v.y + u.z * v.z; }
__device__ __forceinline__ float3 sub3(float3 u, float3 v) { return make_float3(u.x - v.x, u.y - v.y, u.z - v.z); }

// |u - t v|^2
__device__ __forceinline__ float off_d2(float3 u, float t, float3 v) {
  const float3 w = make_float3(u.x - t * v.x, u.y - t * v.y, u.z - t * v.z);
  return dot3(w, w);
}

// Squared distance from p to segment [a, a + e].
__device__ __forceinline__ float seg_d2(float3 p, float3 a, float3 e) {
  const float3 ap = sub3(p, a);
  const float l2 = dot3(e, e);
  const float t = l2 > 0.f ? fminf(fmaxf(dot3(ap, e) / l2, 0.f), 1.f) : 0.f;
  return off_d2(ap, t, e);
}

// Squared distance from p to the filled triangle T. The nearest point is found
// by locating p among the triangle's Voronoi regions (three vertices, three
// edges, the face) with the dot-product tests of Ericson, Real-Time
// Collision Detection (2005), Sec. 5.1.5: vertex a when p projects before
// both edges leaving a; edge ab when the signed area term for c is not
// positive and p projects within ab; the face when all three terms are
// positive (then the barycentric weights are those terms over their sum).
// A zero-area triangle (no positive sum) is its three edges.
__device__ __forceinline__ float point_tri_d2(float3 p, const Tri& T) {
  const float3 ab = sub3(T.b, T.a), ac = sub3(T.c, T.a), ap = sub3(p, T.a);
  const float d1 = dot3(ab, ap), d2 = dot3(ac, ap);
  if (d1 <= 0.f && d2 <= 0.f) return dot3(ap, ap);
  const float3 bp = sub3(p, T.b);
  const float d3 = dot3(ab, bp), d4 = dot3(ac, bp);
  if (d3 >= 0.f && d4 <= d3) return dot3(bp, bp);
  const float vc = d1 * d4 - d3 * d2;
  if (vc <= 0.f && d1 >= 0.f && d3 <= 0.f) return off_d2(ap, d1 / (d1 - d3), ab);
  const float3 cp = sub3(p, T.c);
  const float d5 = dot3(ab, cp), d6 = dot3(ac, cp);
  if (d6 >= 0.f && d5 <= d6) return dot3(cp, cp);
  const float vb = d5 * d2 - d1 * d6;
  if (vb <= 0.f && d2 >= 0.f && d6 <= 0.f) return off_d2(ap, d2 / (d2 - d6), ac);
  const float va = d3 * d6 - d5 * d4;
  const float e43 = d4 - d3, e56 = d5 - d6;
  if (va <= 0.f && e43 >= 0.f && e56 >= 0.f) return off_d2(bp, e43 / (e43 + e56), sub3(T.c, T.b));
  const float s = va + vb + vc;
  if (!(s > 0.f))
    return fminf(seg_d2(p, T.a, ab), fminf(seg_d2(p, T.a, ac), seg_d2(p, T.b, sub3(T.c, T.b))));
  const float v = vb / s, w = vc / s;
  const float3 q = make_float3(ap.x - v * ab.x - w * ac.x, ap.y - v * ab.y - w * ac.y, ap.z - v * ab.z - w * ac.z);
  return dot3(q, q);
}

}  // namespace sc
