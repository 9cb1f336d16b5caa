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
  const float* inv;  // optional: 1 / |v_i - v_{i-1}|^2 per vertex (0 for a zero-length edge)
};

// Crossing-number point-in-polygon (boundary counts as inside) and the
// Euclidean distance to the boundary (minimum over the edge segments). The
// crossing test compares (px - ax) * ey with (py - ay) * ex instead of
// dividing by ey, which is the same test for every point off the boundary.
__device__ __forceinline__ bool pip_with_distance(const PolyView& P, float px, float py, float* dist) {
  bool odd = false;
  float d2 = 3.0e38f;
  float2 a = __ldg(&P.v[P.n - 1]);
#pragma unroll 1
  for (int i = 0; i < P.n; ++i) {
    const float2 b = __ldg(&P.v[i]);
    // distance to segment a-b
    const float ex = b.x - a.x, ey = b.y - a.y;
    const float wx = px - a.x, wy = py - a.y;
    const float dot = wx * ex + wy * ey;
    float t;
    if (P.inv) {
      t = dot * __ldg(&P.inv[i]);
    } else {
      const float len2 = ex * ex + ey * ey;
      t = len2 > 0.f ? dot / len2 : 0.f;
    }
    t = fminf(fmaxf(t, 0.f), 1.f);
    const float qx = wx - t * ex, qy = wy - t * ey;
    d2 = fminf(d2, qx * qx + qy * qy);
    // does edge a-b cross the ray from p towards +x? (ey != 0 here)
    if ((a.y > py) != (b.y > py)) {
      const float lhs = wx * ey, rhs = wy * ex;
      if (ey > 0.f ? lhs < rhs : lhs > rhs) odd = !odd;
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
  s.P.inv = nullptr;
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

constexpr int kMaxAnchors = 16;

// What sampling object k needs besides the support: its relation, half
// extents (w: rho), relation parameters and, for a relation, the reference
// object's pose and half extents; for DIRECTIONAL the direction angle (the
// anchor's yaw added under SC_REL_LOCAL), for MIDDLE where its anchors are.
// Loaded by load_object_spec so a caller can issue these loads early.
struct ObjectSpec {
  int kind, ref, face_to;
  float4 H, RP;
  float4 ref_pose, ref_half;
  float dir;      // DIRECTIONAL: direction angle
  int an0, n_an;  // MIDDLE: anchors obj_anchor[an0 .. an0 + n_an)
};

// Relation of template-local object k of candidate c (template t). A
// reference (parent, anchor, faced object) must be an earlier object, a
// DIRECTIONAL object needs obj_rel_dir, a MIDDLE one 2..16 earlier anchors, an
// INSIDE one a part of its template: otherwise kDevBadRelation is latched and
// the object is sampled as free. The reference pose is read from
// poses[pbase + ref], written before this call (the caller orders the
// accesses). INSIDE becomes ON_TOP of a flat reference: the part's support
// rectangle moved by q * axis, its half extents shrunk by the erosion e (not
// below 0), the face-to flag dropped as for ON_TOP. EXT = false compiles only
// FREE / ON_TOP / NEXT_TO (any other kind or flag is refused the same way) for
// batches known to use no more.
template <bool EXT = true>
__device__ __forceinline__ ObjectSpec load_object_spec(const sc_scene_batch& b, int o0, int k, int rel,
                                                       const float4* poses, int64_t pbase, int* status, int lane,
                                                       int t, int c) {
  ObjectSpec S;
  const int o = o0 + k;
  S.kind = rel & SC_REL_KIND_MASK;
  S.face_to = EXT && (rel & SC_REL_FACE_TO) != 0;
  S.ref = (rel >> 8) & 0xFF;
  S.an0 = 0;
  S.n_an = 0;
  S.dir = 0.f;
  const bool inside = EXT && S.kind == SC_REL_INSIDE;
  int part0 = 0;
  if (inside) {
    S.face_to = 0;
    bool ok = b.part_param && b.part_q && b.tmpl_part_off && b.max_parts > 0;
    if (ok) {
      part0 = __ldg(&b.tmpl_part_off[t]);
      ok = S.ref < __ldg(&b.tmpl_part_off[t + 1]) - part0 && S.ref < b.max_parts;
    }
    if (!ok && lane == 0) latch_error(status, kDevBadPart);
    if (!ok) S.kind = SC_REL_FREE;
  }
  bool bad = (S.kind != SC_REL_FREE || S.face_to) && S.ref >= k && !inside;
  bad = bad || S.kind > (EXT ? SC_REL_INSIDE : SC_REL_NEXT_TO) || (EXT && S.kind == SC_REL_DIRECTIONAL && !b.obj_rel_dir);
  if (EXT && S.kind == SC_REL_MIDDLE) {
    if (!b.obj_anchor_off) {
      bad = true;
    } else {
      S.an0 = __ldg(&b.obj_anchor_off[o]);
      S.n_an = __ldg(&b.obj_anchor_off[o + 1]) - S.an0;
      bool ok = S.n_an >= 2 && S.n_an <= kMaxAnchors;
      if (ok) {
        const int j = lane < S.n_an ? __ldg(&b.obj_anchor[S.an0 + lane]) : 0;
        ok = __all_sync(0xFFFFFFFFu, j >= 0 && j < k);
      }
      bad = bad || !ok;
    }
  }
  if (bad) {
    if (lane == 0) latch_error(status, kDevBadRelation);
    S.kind = SC_REL_FREE;
    S.face_to = 0;
  }
  S.H = __ldg(reinterpret_cast<const float4*>(b.obj_half) + o);
  S.RP = __ldg(reinterpret_cast<const float4*>(b.obj_rel_param) + o);
  S.ref_pose = make_float4(0.f, 0.f, 0.f, 0.f);
  S.ref_half = make_float4(0.f, 0.f, 0.f, 0.f);
  if (EXT && S.kind == SC_REL_INSIDE) {
    // part_param rows: (axis, qmin), (qmax, centre), (half extents, yaw, -)
    const float4* pp = reinterpret_cast<const float4*>(b.part_param) + 3 * (int64_t)(part0 + S.ref);
    const float4 ax = __ldg(pp), ce = __ldg(pp + 1), hh = __ldg(pp + 2);
    const float q = __ldg(&b.part_q[(int64_t)c * b.max_parts + S.ref]);
    const float e = S.RP.z * fminf(S.H.x, S.H.y);
    S.ref_pose = make_float4(ce.y + q * ax.x, ce.z + q * ax.y, ce.w + q * ax.z, hh.z);
    S.ref_half = make_float4(fmaxf(hh.x - e, 0.f), fmaxf(hh.y - e, 0.f), 0.f, 0.f);
    S.kind = SC_REL_ON_TOP;
  } else if (S.kind != SC_REL_FREE || S.face_to) {
    S.ref_pose = poses[pbase + S.ref];
    S.ref_half = __ldg(reinterpret_cast<const float4*>(b.obj_half) + (o0 + S.ref));
  }
  if (EXT && S.kind == SC_REL_DIRECTIONAL)
    S.dir = __ldg(&b.obj_rel_dir[o]) + ((rel & SC_REL_LOCAL) ? S.ref_pose.w : 0.f);
  return S;
}

// Lowest accepted attempt of a 32-attempt chunk (or the chunk's last attempt
// when none is accepted), folded into R: placed, band of the deciding
// attempts, and the chosen attempt's x, y, yaw.
__device__ __forceinline__ void take_attempt(SampleResult& R, bool acc, bool bnd, float x, float y, float yaw,
                                             int max_attempts, int a0) {
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

// FREE, NEXT_TO and ON_TOP objects (Sec. III, IV-C, IV-F). Attempts run one
// per lane; the lowest accepted attempt wins, which equals trying them in
// order. Every lane gets the same result.
__device__ __forceinline__ SampleResult warp_sample_basic(const Support& sup, const ObjectSpec& S, uint64_t seed,
                                                         int max_attempts, int retry, int c, int k, int lane) {
  SampleResult R;
  R.band = false;
  R.placed = false;
  R.pose = make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 H = S.H, RP = S.RP;
  const bool on_top = S.kind == SC_REL_ON_TOP;
  const float e = RP.z * fminf(H.x, H.y);  // ratio_on_support erosion
  float4 anchor = make_float4(0.f, 0.f, 0.f, 0.f);
  float rho_sum = 0.f;
  if (S.kind == SC_REL_NEXT_TO) {
    anchor = S.ref_pose;
    rho_sum = S.ref_half.w + H.w;
  }
#pragma unroll 1
  for (int a0 = 0; a0 < max_attempts && !R.placed; a0 += 32) {
    const int a = a0 + lane;
    const bool valid = a < max_attempts;
    const float4 u = draw_uniform4(seed, (uint32_t)c, (uint32_t)k, (uint32_t)retry, (uint32_t)a);
    if (on_top) {
      // attempt 0 (lane 0's draw) places the object on the reference's top face
      const float4 pp = S.ref_pose;
      const float4 pH = S.ref_half;
      const float ux = __shfl_sync(0xFFFFFFFFu, u.x, 0), uy = __shfl_sync(0xFFFFFFFFu, u.y, 0),
                  uz = __shfl_sync(0xFFFFFFFFu, u.z, 0);
      const float xl = pH.x * (2.f * ux - 1.f), yl = pH.y * (2.f * uy - 1.f);
      float sy, cy;
      sincosf(pp.w, &sy, &cy);
      R.pose = make_float4(pp.x + cy * xl - sy * yl, pp.y + sy * xl + cy * yl, pp.z + pH.z + H.z, kTwoPi * uz);
      R.placed = true;
      return R;
    }
    float x = 0.f, y = 0.f, yaw = 0.f;
    bool acc = false, bnd = false;
    if (valid) {
      if (S.kind == SC_REL_NEXT_TO) {
        float sp, cp;
        sincos_cw(kTwoPi * u.x, &sp, &cp);
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
    take_attempt(R, acc, bnd, x, y, yaw, max_attempts, a0);
  }
  R.pose.z = sup.z + H.z;
  return R;
}

// Position of object j of the candidate (anchors of a MIDDLE relation).
__device__ __forceinline__ float2 object_xy(const float4* poses, int j) {
  const float4 p = poses[j];
  return make_float2(p.x, p.y);
}

// DIRECTIONAL and MIDDLE objects (Sec. IV-F), out of line so the common
// kinds do not carry this code. Attempts as in warp_sample_spec, with the
// proposal:
//   DIRECTIONAL: area-uniform in the sector of half-angle RP.w around S.dir
//     between radii RP.x and min(RP.y, the farthest support-box corner from
//     the anchor), measured from the anchor's position;
//   MIDDLE: on the segment between two anchors, or uniform in the bounding
//     box of 3+ anchors and kept inside their polygon (crossing number,
//     boundary inside; within the band of its boundary flags the attempt).
// anchors: the batch's obj_anchor; poses: the candidate's object poses.
static __device__ __noinline__ SampleResult warp_sample_special(const Support& sup, const ObjectSpec& S, uint64_t seed,
                                                                int max_attempts, int retry, int c, int k, int lane,
                                                                const int32_t* anchors, const float4* poses) {
  SampleResult R;
  R.band = false;
  R.placed = false;
  R.pose = make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 H = S.H, RP = S.RP;
  const float e = RP.z * fminf(H.x, H.y);  // ratio_on_support erosion
  const bool directional = S.kind == SC_REL_DIRECTIONAL;
  const int n = S.n_an;
  const int32_t* an = anchors + S.an0;
  float r1 = 0.f;
  float4 box = make_float4(3e38f, -3e38f, 3e38f, -3e38f);
  if (directional) {
    const float dx = fmaxf(fabsf(sup.xmin - S.ref_pose.x), fabsf(sup.xmax - S.ref_pose.x));
    const float dy = fmaxf(fabsf(sup.ymin - S.ref_pose.y), fabsf(sup.ymax - S.ref_pose.y));
    r1 = fminf(RP.y, sqrtf(dx * dx + dy * dy));
  } else {
    for (int i = 0; i < n; ++i) {
      const float2 a = object_xy(poses, __ldg(&an[i]));
      box.x = fminf(box.x, a.x); box.y = fmaxf(box.y, a.x);
      box.z = fminf(box.z, a.y); box.w = fmaxf(box.w, a.y);
    }
  }
  for (int a0 = 0; a0 < max_attempts && !R.placed; a0 += 32) {
    const int a = a0 + lane;
    const float4 u = draw_uniform4(seed, (uint32_t)c, (uint32_t)k, (uint32_t)retry, (uint32_t)a);
    float x = 0.f, y = 0.f;
    bool acc = false, bnd = false;
    if (a < max_attempts) {
      bool in_rel = true;
      if (directional) {
        const float r0 = RP.x;
        const float rho = sqrtf(fmaxf(0.f, r0 * r0 + (r1 * r1 - r0 * r0) * u.x));
        float sn, cs;
        sincosf(S.dir + RP.w * (2.f * u.y - 1.f), &sn, &cs);
        x = S.ref_pose.x + rho * cs;
        y = S.ref_pose.y + rho * sn;
      } else if (n == 2) {
        const float2 p = object_xy(poses, __ldg(&an[0])), q = object_xy(poses, __ldg(&an[1]));
        x = p.x + u.x * (q.x - p.x);
        y = p.y + u.x * (q.y - p.y);
      } else {
        x = box.x + (box.y - box.x) * u.x;
        y = box.z + (box.w - box.z) * u.y;
        bool odd = false;
        float d2 = 3.0e38f;
        float2 p = object_xy(poses, __ldg(&an[n - 1]));
        for (int i = 0; i < n; ++i) {
          const float2 q = object_xy(poses, __ldg(&an[i]));
          const float ex = q.x - p.x, ey = q.y - p.y, wx = x - p.x, wy = y - p.y;
          const float len2 = ex * ex + ey * ey;
          float t = len2 > 0.f ? (wx * ex + wy * ey) / len2 : 0.f;
          t = fminf(fmaxf(t, 0.f), 1.f);
          const float qx = wx - t * ex, qy = wy - t * ey;
          d2 = fminf(d2, qx * qx + qy * qy);
          if ((p.y > y) != (q.y > y)) {
            const float lhs = wx * ey, rhs = wy * ex;
            if (ey > 0.f ? lhs < rhs : lhs > rhs) odd = !odd;
          }
          p = q;
        }
        in_rel = odd || d2 == 0.f;
        bnd = sqrtf(d2) <= kBand;
      }
      float dist;
      const bool inside = pip_with_distance(sup.P, x, y, &dist);
      acc = in_rel && inside && dist >= e;
      bnd = bnd || dist <= kBand || (inside && fabsf(dist - e) <= kBand);
    }
    take_attempt(R, acc, bnd, x, y, kTwoPi * u.z, max_attempts, a0);
  }
  R.pose.z = sup.z + H.z;
  return R;
}

// Sample object k (spec S) of candidate c for try `retry`; the whole warp
// calls this (uniform arguments). Attempts run one per lane; the lowest
// accepted attempt wins, which equals trying them in order. Every lane gets
// the same result. With SC_REL_FACE_TO the yaw of the chosen attempt faces
// the reference object (the yaw takes no part in acceptance). anchors: the
// batch's obj_anchor; poses: the candidate's object poses (MIDDLE anchors).
// EXT = false: the basic kinds only (see load_object_spec).
template <bool EXT = true>
__device__ __forceinline__ SampleResult warp_sample_spec(const Support& sup, const ObjectSpec& S, uint64_t seed,
                                                        int max_attempts, int retry, int c, int k, int lane,
                                                        const int32_t* anchors, const float4* poses) {
  if (!EXT) return warp_sample_basic(sup, S, seed, max_attempts, retry, c, k, lane);
  SampleResult R;
  if (S.kind >= SC_REL_DIRECTIONAL) {
    R = warp_sample_special(sup, S, seed, max_attempts, retry, c, k, lane, anchors, poses);
  } else {
    R = warp_sample_basic(sup, S, seed, max_attempts, retry, c, k, lane);
  }
  if (S.face_to && S.kind != SC_REL_ON_TOP) R.pose.w = atan2f(S.ref_pose.y - R.pose.y, S.ref_pose.x - R.pose.x);
  return R;
}

// Sample template-local object k of candidate c for try `retry` (loads the
// object's spec, then samples it).
__device__ __forceinline__ SampleResult warp_sample_object(const sc_scene_batch& b, const Support& sup,
                                                          uint64_t seed, int max_attempts, int retry, int c, int k,
                                                          int o0, const float4* poses, int64_t pbase, int* status,
                                                          int lane, int t) {
  const ObjectSpec S = load_object_spec(b, o0, k, __ldg(&b.obj_rel[o0 + k]), poses, pbase, status, lane, t, c);
  return warp_sample_spec(sup, S, seed, max_attempts, retry, c, k, lane, b.obj_anchor, poses + pbase);
}

}  // namespace sc
