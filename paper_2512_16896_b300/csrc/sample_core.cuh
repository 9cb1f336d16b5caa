// Warp-level sampling of one object's pose (Sec. III position sampling,
// Sec. IV-C batch sampling with the canonical polygon moved per instance,
// Sec. IV-F relations and ratio_on_support erosion). Shared by the sampling
// kernel and the fused generation step.
#pragma once

#include "common.cuh"

namespace sc {

struct PolyView {
  const float2* v;
  int n;
};

// Crossing-number point-in-polygon (boundary counts as inside) and the
// Euclidean distance to the boundary (minimum over the edge segments).
__device__ __forceinline__ bool pip_with_distance(const PolyView& P, float px, float py, float* dist) {
  bool odd = false;
  float d2 = 3.0e38f;
  float2 a = __ldg(&P.v[P.n - 1]);
  for (int i = 0; i < P.n; ++i) {
    float2 b = __ldg(&P.v[i]);
    // distance to segment a-b
    float ex = b.x - a.x, ey = b.y - a.y;
    float wx = px - a.x, wy = py - a.y;
    float len2 = ex * ex + ey * ey;
    float t = len2 > 0.f ? (wx * ex + wy * ey) / len2 : 0.f;
    t = fminf(fmaxf(t, 0.f), 1.f);
    float qx = wx - t * ex, qy = wy - t * ey;
    d2 = fminf(d2, qx * qx + qy * qy);
    // does edge a-b cross the ray from p towards +x?
    if ((a.y > py) != (b.y > py)) {
      float xc = a.x + (py - a.y) * (b.x - a.x) / (b.y - a.y);
      if (px < xc) odd = !odd;
    }
    a = b;
  }
  *dist = sqrtf(d2);
  return odd || d2 == 0.f;
}

// Support polygon of template t and its bounding box (computed by the warp).
struct Support {
  PolyView P;
  float xmin, xmax, ymin, ymax, z;
  bool ok;
};

__device__ __forceinline__ Support warp_support(const sc_scene_batch& b, int t, int lane) {
  Support s;
  const int v0 = __ldg(&b.tmpl_poly_off[t]);
  s.P.v = reinterpret_cast<const float2*>(b.poly_verts) + v0;
  s.P.n = __ldg(&b.tmpl_poly_off[t + 1]) - v0;
  s.ok = s.P.n >= 3 && s.P.n <= kMaxPolyVerts;
  s.z = __ldg(&b.tmpl_support_z[t]);
  float xmin = 3e38f, xmax = -3e38f, ymin = 3e38f, ymax = -3e38f;
  if (s.ok) {
    for (int i = lane; i < s.P.n; i += 32) {
      float2 v = __ldg(&s.P.v[i]);
      xmin = fminf(xmin, v.x); xmax = fmaxf(xmax, v.x);
      ymin = fminf(ymin, v.y); ymax = fmaxf(ymax, v.y);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    xmin = fminf(xmin, __shfl_xor_sync(0xFFFFFFFFu, xmin, o));
    xmax = fmaxf(xmax, __shfl_xor_sync(0xFFFFFFFFu, xmax, o));
    ymin = fminf(ymin, __shfl_xor_sync(0xFFFFFFFFu, ymin, o));
    ymax = fmaxf(ymax, __shfl_xor_sync(0xFFFFFFFFu, ymax, o));
  }
  s.xmin = xmin; s.xmax = xmax; s.ymin = ymin; s.ymax = ymax;
  return s;
}

struct SampleResult {
  float4 pose;
  bool placed;
  bool band;
};

// Sample template-local object k of candidate c for try `retry`; the whole
// warp calls this (uniform arguments). Earlier objects' poses are read from
// poses[pbase + ref] (written before this call; the caller orders the
// accesses). Attempts run one per lane; the lowest accepted attempt wins,
// which equals trying them in order. Lane 0's result is the valid one; every
// lane gets the same values.
__device__ __forceinline__ SampleResult warp_sample_object(const sc_scene_batch& b, const Support& sup,
                                                          uint64_t seed, int max_attempts, int retry, int c, int k,
                                                          int o0, const float4* poses, int64_t pbase, int* status,
                                                          int lane) {
  SampleResult R;
  R.band = false;
  R.placed = false;
  R.pose = make_float4(0.f, 0.f, 0.f, 0.f);
  const int o = o0 + k;
  const int rel = __ldg(&b.obj_rel[o]);
  int kind = rel & SC_REL_KIND_MASK;
  const int ref = rel >> 8;
  if (kind != SC_REL_FREE && (ref < 0 || ref >= k || kind > SC_REL_NEXT_TO)) {
    // a relation must refer to an earlier object: report, sample it as free
    if (lane == 0) latch_error(status, kDevBadRelation);
    kind = SC_REL_FREE;
  }
  const float4 H = __ldg(reinterpret_cast<const float4*>(b.obj_half) + o);
  const float4 RP = __ldg(reinterpret_cast<const float4*>(b.obj_rel_param) + o);
  if (kind == SC_REL_ON_TOP) {
    const float4 u = draw_uniform4(seed, (uint32_t)c, (uint32_t)k, (uint32_t)retry, 0u);
    const float4 pp = poses[pbase + ref];
    const float4 pH = __ldg(reinterpret_cast<const float4*>(b.obj_half) + (o0 + ref));
    const float xl = pH.x * (2.f * u.x - 1.f), yl = pH.y * (2.f * u.y - 1.f);
    float sy, cy;
    sincosf(pp.w, &sy, &cy);
    R.pose = make_float4(pp.x + cy * xl - sy * yl, pp.y + sy * xl + cy * yl, pp.z + pH.z + H.z, kTwoPi * u.z);
    R.placed = true;
    return R;
  }
  const float e = RP.z * fminf(H.x, H.y);  // ratio_on_support erosion
  float4 anchor = make_float4(0.f, 0.f, 0.f, 0.f);
  float rho_sum = 0.f;
  if (kind == SC_REL_NEXT_TO) {
    anchor = poses[pbase + ref];
    rho_sum = __ldg(&b.obj_half[4 * (o0 + ref) + 3]) + H.w;
  }
  for (int a0 = 0; a0 < max_attempts && !R.placed; a0 += 32) {
    const int a = a0 + lane;
    const bool valid = a < max_attempts;
    float x = 0.f, y = 0.f, yaw = 0.f;
    bool acc = false, bnd = false;
    if (valid) {
      const float4 u = draw_uniform4(seed, (uint32_t)c, (uint32_t)k, (uint32_t)retry, (uint32_t)a);
      if (kind == SC_REL_NEXT_TO) {
        float sp, cp;
        sincosf(kTwoPi * u.x, &sp, &cp);
        const float r = rho_sum + RP.x + (RP.y - RP.x) * u.y;
        x = anchor.x + r * cp;
        y = anchor.y + r * sp;
      } else {
        x = sup.xmin + (sup.xmax - sup.xmin) * u.x;
        y = sup.ymin + (sup.ymax - sup.ymin) * u.y;
      }
      yaw = kTwoPi * u.z;
      float dist;
      const bool inside = pip_with_distance(sup.P, x, y, &dist);
      acc = inside && dist >= e;
      bnd = dist <= kBand || (inside && fabsf(dist - e) <= kBand);
    }
    const unsigned acc_mask = __ballot_sync(0xFFFFFFFFu, acc);
    const unsigned bnd_mask = __ballot_sync(0xFFFFFFFFu, bnd);
    int src;
    if (acc_mask) {
      src = __ffs(acc_mask) - 1;
      const unsigned upto = (src == 31) ? 0xFFFFFFFFu : ((2u << src) - 1u);
      R.band = R.band || (bnd_mask & upto);
      R.placed = true;
    } else {
      R.band = R.band || bnd_mask;
      src = min(31, max_attempts - 1 - a0);  // last attempt of this chunk
    }
    R.pose.x = __shfl_sync(0xFFFFFFFFu, x, src);
    R.pose.y = __shfl_sync(0xFFFFFFFFu, y, src);
    R.pose.w = __shfl_sync(0xFFFFFFFFu, yaw, src);
  }
  R.pose.z = sup.z + H.z;
  return R;
}

}  // namespace sc
