// Collision kernel of sc_collide / sc_collide_ex (Sec. IV-B one transform
// per instance, Sec. IV-D batched collision checking). Persistent CTAs take
// candidates from the caller's list through a global atomic counter (list the
// heaviest first); one CTA reduces one candidate's minimum signed distance
// (exact minimum, or decide-only mode) at a time:
//  * stage_*: the candidate's objects [0, n) are moved to shared memory once,
//    spheres in the world frame relative to the position of object 0, with
//    each object's bounding ball, and the template's world boxes;
//  * box_units: sphere vs world box, culled per (object, box) by the ball;
//  * seed_pairs: the first two spheres of every object pair, a first upper
//    bound on the minimum;
//  * build_units / pair_units: the pair set {(i, j): obj(i) < obj(j),
//    obj(j) >= f} is cut into units (A block of 32*APL consecutive spheres,
//    one per lane per slot) x (B segment of up to seg_len spheres); warps
//    pull units from a CTA-local counter and sweep them one B object at a
//    time (object-pair ball cull) with the prune test of collide_core.cuh.
#include "collide_core.cuh"
#include "kernels.h"
#include "tri_core.cuh"

namespace sc {

namespace {

using namespace core;

struct Layout {
  int W, beta, oid, off, opose, osc, obb, blk_lo, blk_pref, total, nb_max, cap;
};

__host__ __device__ inline Layout make_layout(int max_sph, int max_obj, int apl) {
  Layout L;
  L.cap = ((max_sph + kPad + 7) / 8) * 8;
  L.nb_max = L.cap / (32 * apl) + 2;
  L.W = 0;
  L.beta = align16(L.W + 16 * L.cap);
  L.oid = align16(L.beta + 4 * L.cap);
  L.off = align16(L.oid + L.cap);
  L.opose = align16(L.off + 4 * (max_obj + 1));
  L.osc = align16(L.opose + 16 * max_obj);
  L.obb = align16(L.osc + 8 * max_obj);
  L.blk_lo = align16(L.obb + 4 * 16 * kMaxObbPerTemplate);
  L.blk_pref = align16(L.blk_lo + 4 * L.nb_max);
  L.total = align16(L.blk_pref + 4 * (L.nb_max + 1));
  return L;
}

struct Smem {
  float4* W;
  float* beta;
  uint8_t* oid;
  int* off;
  float4* opose;
  float2* osc;  // sin, cos of each object's yaw; once the spheres are staged,
                // (radius of its bounding ball about its position, 0)
  float* obbd;
  int* blk_lo;
  int* blk_pref;
};

__device__ __forceinline__ Smem smem_view(unsigned char* base, const Layout& L) {
  Smem s;
  s.W = reinterpret_cast<float4*>(base + L.W);
  s.beta = reinterpret_cast<float*>(base + L.beta);
  s.oid = base + L.oid;
  s.off = reinterpret_cast<int*>(base + L.off);
  s.opose = reinterpret_cast<float4*>(base + L.opose);
  s.osc = reinterpret_cast<float2*>(base + L.osc);
  s.obbd = reinterpret_cast<float*>(base + L.obb);
  s.blk_lo = reinterpret_cast<int*>(base + L.blk_lo);
  s.blk_pref = reinterpret_cast<int*>(base + L.blk_pref);
  return s;
}

// CTA-wide scalars (a static __shared__ object of the kernel).
struct CtaShared {
  int item;
  int unit_next, total_units, nb;
  int best_key;            // MIN: CTA-wide running minimum (float_key)
  int r2max_key, rmax_key;
  int hit;                 // DECIDE: a certain collision was found
  int bad_box;             // a staged box names a part its template lacks
  unsigned long long bar;  // mbarrier of the bulk copy of the local spheres
  float warp_min[32];
};

// largest k in [0, n) with arr[k] <= v, for non-decreasing arr with arr[0] <= v
__device__ __forceinline__ int upper_index(const int* arr, int n, int v) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (arr[mid] <= v) lo = mid; else hi = mid;
  }
  return lo;
}

// Poses, sin/cos of yaw and sphere offsets of objects [0, n).
__device__ __forceinline__ void stage_objects(const sc_scene_batch& b, const float4* poses, int64_t pbase, int o0,
                                              int s0, int n, const Smem& sm, int tid, int nthr) {
  for (int k = tid; k < n; k += nthr) {
    const float4 p = poses[pbase + k];
    float sn, cs;
    sincosf(p.w, &sn, &cs);
    sm.opose[k] = p;
    sm.osc[k] = make_float2(sn, cs);
    sm.off[k] = __ldg(&b.obj_sph_off[o0 + k]) - s0;
  }
  if (tid == 0) sm.off[n] = __ldg(&b.obj_sph_off[o0 + n]) - s0;
}

// Spheres [0, S) of the staged objects in the world frame relative to object
// 0's position, plus |c|^2 - r^2; kPad far-away dummies after them; and each
// object's bounding-ball radius about its position, max |l| + r over its
// local spheres l, in place of its (no longer needed) sin/cos. Groups of gl lanes (8, 16 or 32, from the mean spheres
// per object) take one object at a time, so a sphere's object needs no search
// and each object's pose is read once per group.
__device__ __forceinline__ void stage_spheres(const sc_scene_batch& b, int s0, int n, int S, const Smem& sm,
                                              CtaShared& sh, int tid, int nthr, int lane, bool in_smem) {
  const float4 ref = sm.opose[0];
  float r2max = 0.f, rmx = 0.f;
  const int mean = S / n;
  const int gl = mean > 16 ? 32 : mean > 8 ? 16 : 8;
  const int ngrp = nthr / gl;
  // the local spheres: in global memory, or already copied into W (in_smem;
  // each sphere is then read and overwritten by the same lane)
  const float4* local = in_smem ? sm.W : reinterpret_cast<const float4*>(b.sph_local) + s0;
#pragma unroll 1
  for (int k0 = 0; k0 < n; k0 += ngrp) {  // same trip count in every lane (group shuffles below)
    const int k = k0 + tid / gl;
    float rad = 0.f;
    if (k < n) {
      const int lo = sm.off[k], hi = sm.off[k + 1];
      const float4 p = sm.opose[k];
      const float2 sc2 = sm.osc[k];
      const float tx = p.x - ref.x, ty = p.y - ref.y, tz = p.z - ref.z;
#pragma unroll 2
      for (int q = lo + (tid & (gl - 1)); q < hi; q += gl) {
        const float4 l = in_smem ? local[q] : __ldg(local + q);
        const float x = tx + (sc2.y * l.x - sc2.x * l.y);
        const float y = ty + (sc2.x * l.x + sc2.y * l.y);
        const float z = tz + l.z;
        const float c2 = x * x + y * y + z * z;
        sm.W[q] = make_float4(x, y, z, l.w);
        sm.beta[q] = c2 - l.w * l.w;
        sm.oid[q] = (uint8_t)k;
        r2max = fmaxf(r2max, c2);
        rmx = fmaxf(rmx, l.w);
        rad = fmaxf(rad, sqrtf(l.x * l.x + l.y * l.y + l.z * l.z) + l.w);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      if (o < gl) rad = fmaxf(rad, __shfl_xor_sync(0xFFFFFFFFu, rad, o));
    // the group's lanes read osc[k] before the shuffles above
    if (k < n && (tid & (gl - 1)) == 0) sm.osc[k] = make_float2(rad, 0.f);
  }
  for (int q = S + tid; q < S + kPad; q += nthr) {
    sm.W[q] = make_float4(1e6f, 1e6f, 1e6f, 0.f);
    sm.beta[q] = 3e12f;
    sm.oid[q] = 255;
  }
  r2max = -warp_min(-r2max);
  rmx = -warp_min(-rmx);
  if (lane == 0) {
    atomicMax(&sh.r2max_key, __float_as_int(r2max));  // non-negative floats order as ints
    atomicMax(&sh.rmax_key, __float_as_int(rmx));
  }
}

// World boxes: columns of R, minus R^T (centre - object 0's position), half
// extents. A sphere centre w (relative to object 0) has box-frame
// coordinates p = R^T w - R^T (centre - ref): three FMAs per axis.
__device__ __forceinline__ void stage_boxes(const sc_scene_batch& b, int t, int c, int bx0, int nobb, const Smem& sm,
                                            int tid, int nthr, int* status, int* bad_box) {
  const float4 ref = sm.opose[0];
  for (int k = tid; k < nobb; k += nthr) {
    bool bad = false;
    const float3 sh = box_shift(b, t, c, bx0 + k, status, &bad);  // an articulated part's box moves with its joint
    if (bad) *(volatile int*)bad_box = 1;
    const float* o = b.obb + 12 * (bx0 + k);
    float qx = __ldg(o + 4), qy = __ldg(o + 5), qz = __ldg(o + 6), qw = __ldg(o + 7);
    const float inv = rsqrtf(qx * qx + qy * qy + qz * qz + qw * qw);
    qx *= inv; qy *= inv; qz *= inv; qw *= inv;
    float* d = sm.obbd + 16 * k;
    // R (row-major) of the unit quaternion; stored by columns
    d[0] = 1.f - 2.f * (qy * qy + qz * qz); d[1] = 2.f * (qx * qy + qz * qw); d[2] = 2.f * (qx * qz - qy * qw);
    d[3] = 2.f * (qx * qy - qz * qw); d[4] = 1.f - 2.f * (qx * qx + qz * qz); d[5] = 2.f * (qy * qz + qx * qw);
    d[6] = 2.f * (qx * qz + qy * qw); d[7] = 2.f * (qy * qz - qx * qw); d[8] = 1.f - 2.f * (qx * qx + qy * qy);
    const float cx = (__ldg(o + 0) + sh.x) - ref.x, cy = (__ldg(o + 1) + sh.y) - ref.y,
                cz = (__ldg(o + 2) + sh.z) - ref.z;
    d[9] = -(d[0] * cx + d[1] * cy + d[2] * cz);
    d[10] = -(d[3] * cx + d[4] * cy + d[5] * cz);
    d[11] = -(d[6] * cx + d[7] * cy + d[8] * cz);
    d[12] = __ldg(o + 8); d[13] = __ldg(o + 9); d[14] = __ldg(o + 10); d[15] = 0.f;
  }
}

// Warp 0: work units for pairs (i, j), obj(i) < obj(j), obj(j) in [f, n):
// A blocks of BA spheres, each lane one block at a time, unit counts summed
// by a warp scan.
__device__ __forceinline__ void build_units(int f, int n, int S, int BA, int seg_len, const Smem& sm, CtaShared& sh,
                                            int lane) {
  int total = 0, nb = 0;
  if (f < n && sm.off[n - 1] > 0) nb = (sm.off[n - 1] + BA - 1) / BA;
  for (int bk0 = 0; bk0 < nb; bk0 += 32) {
    const int bk = bk0 + lane;
    int cnt = 0;
    if (bk < nb) {
      const int lo = max(sm.off[f], sm.off[sm.oid[bk * BA] + 1]);
      sm.blk_lo[bk] = lo;
      if (S > lo) cnt = (S - lo + seg_len - 1) / seg_len;
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += v;
    }
    if (bk < nb) sm.blk_pref[bk] = total + incl - cnt;
    total += __shfl_sync(0xFFFFFFFFu, incl, 31);
  }
  if (lane == 0) {
    sm.blk_pref[nb] = total;
    sh.total_units = total;
    sh.nb = nb;
    sh.unit_next = 0;
  }
}

// Box-frame excess q = |R^T (c - centre)| - h of a point c (relative to
// object 0) against a staged box (c0..c3, see stage_boxes), and its largest
// component: a lower bound on the box's signed distance, 1-Lipschitz in c.
struct BoxQ {
  float x, y, z, m;
};

__device__ __forceinline__ BoxQ box_q(const float4& c0, const float4& c1, const float4& c2, const float4& c3,
                                      float wx, float wy, float wz) {
  // c0 = R col 0 | col 1 x; c1 = col 1 yz | col 2 xy; c2 = col 2 z | -R^T centre; c3 = half extents
  const float px = fmaf(c0.x, wx, fmaf(c0.y, wy, fmaf(c0.z, wz, c2.y)));
  const float py = fmaf(c0.w, wx, fmaf(c1.x, wy, fmaf(c1.y, wz, c2.z)));
  const float pz = fmaf(c1.z, wx, fmaf(c1.w, wy, fmaf(c2.x, wz, c2.w)));
  BoxQ q;
  q.x = fabsf(px) - c3.x;
  q.y = fabsf(py) - c3.y;
  q.z = fabsf(pz) - c3.z;
  q.m = fmaxf(q.x, fmaxf(q.y, q.z));
  return q;
}

// Sphere vs world box for the objects [f, n), one (object, box) unit at a
// time. Broad phase: the object's bounding ball (centre c, radius R) gives
// L = max(q(c)) - R, below every sphere's max(q) - r and hence below every
// sphere's distance to the box; a unit is skipped when L (with kBroadMargin
// for FP32 rounding) cannot reach the threshold. Narrow phase: the warp's
// lanes take the object's spheres; the exact box SDF minus r is computed
// where max(q) - r beats the threshold thr (m in MIN, the band in DECIDE),
// tested as max(q) < t with t = thr + r rounded up: a computed distance is
// never below the computed max(q) - r (the sqrt of a sum holding max(q)^2 is
// at least max(q); rounding is monotone), so a skipped pair cannot beat thr.
// PASS 0 (DECIDE): units with L < band; stops at the first certain collision
// (below -band), its own or one another warp raised in `hit`.
// PASS 1 (MIN): units whose balls come within kBroadMargin of the box, which
// is where a collision's depth is found. PASS 2 (MIN): the other units with L below the
// CTA-wide minimum so far (read once per 32 units).
template <int PASS>
__device__ __forceinline__ float box_units(const Smem& sm, CtaShared& sh, int f, int n, int nobb, float m, int lane,
                                           int warp, int nwarps, unsigned long long& my_box) {
  constexpr bool DECIDE = PASS == 0;
  const float4* bd = reinterpret_cast<const float4*>(sm.obbd);
  const float4 ref = sm.opose[0];
  const int nu = (n - f) * nobb;
#pragma unroll 1
  for (int u0 = warp * 32; u0 < nu; u0 += nwarps * 32) {
    float lim = (DECIDE ? kBand : 0.f) + kBroadMargin;
    if (PASS == 2) lim = fminf(m, key_float(*(volatile int*)&sh.best_key)) + kBroadMargin;
    const int u = u0 + lane;
    bool need = false;
    if (u < nu) {
      const int o = f + u / nobb, k = u - (o - f) * nobb;
      const float4 p = sm.opose[o];
      const BoxQ q = box_q(bd[4 * k], bd[4 * k + 1], bd[4 * k + 2], bd[4 * k + 3], p.x - ref.x, p.y - ref.y,
                           p.z - ref.z);
      const float L = q.m - sm.osc[o].x;
      need = PASS == 2 ? (L >= kBroadMargin && L < lim) : L < lim;
    }
    unsigned mask = __ballot_sync(0xFFFFFFFFu, need);
#pragma unroll 1
    while (mask) {
      const int uu = u0 + __ffs(mask) - 1;
      mask &= mask - 1;
      const int o = f + uu / nobb, k = uu - (o - f) * nobb;
      const float4 c0 = bd[4 * k], c1 = bd[4 * k + 1], c2 = bd[4 * k + 2], c3 = bd[4 * k + 3];
      const int lo = sm.off[o], hi = sm.off[o + 1];
#pragma unroll 2
      for (int i = lo + lane; i < hi; i += 32) {
        const float4 w = sm.W[i];
        const BoxQ q = box_q(c0, c1, c2, c3, w.x, w.y, w.z);
        if (q.m < __fadd_ru(DECIDE ? kBand : m, w.w)) {
          const float ox = fmaxf(q.x, 0.f), oy = fmaxf(q.y, 0.f), oz = fmaxf(q.z, 0.f);
          m = fminf(m, sqrtf(ox * ox + oy * oy + oz * oz) + fminf(q.m, 0.f) - w.w);
        }
      }
      if (lane == 0) my_box += (unsigned long long)(hi - lo);
      if (DECIDE) {
        if (__any_sync(0xFFFFFFFFu, m < -kBand)) {
          if (lane == 0) *(volatile int*)&sh.hit = 1;
          return m;
        }
        // another warp's certain collision (the vote keeps the exit warp-uniform)
        if (__any_sync(0xFFFFFFFFu, *(volatile int*)&sh.hit != 0)) return m;
      }
    }
    if (DECIDE && __any_sync(0xFFFFFFFFu, *(volatile int*)&sh.hit != 0)) return m;
    if (PASS == 2) {
      const float wm = warp_min(m);
      if (lane == 0 && wm < kFarSentinel) atomicMin(&sh.best_key, float_key(wm));
    }
  }
  return m;
}

// Sphere vs world triangle for the objects [f, n), one (object, triangle)
// unit at a time, the passes and thresholds of box_units: the unit's bound is
// L = dist(ball centre, triangle) - R, below every sphere's distance to the
// triangle minus its radius (the triangle is a convex set, its distance
// 1-Lipschitz), with kBroadMargin for FP32 rounding; the narrow phase
// computes each sphere's exact distance. tri: the template's first triangle.
template <int PASS>
__device__ __forceinline__ float tri_units(const Smem& sm, CtaShared& sh, const float* tri, int f, int n, int ntri,
                                           float m, int lane, int warp, int nwarps, unsigned long long& my_tri) {
  constexpr bool DECIDE = PASS == 0;
  const float4 r4 = sm.opose[0];
  const float3 ref = make_float3(r4.x, r4.y, r4.z);
  const int nu = (n - f) * ntri;
#pragma unroll 1
  for (int u0 = warp * 32; u0 < nu; u0 += nwarps * 32) {
    float lim = (DECIDE ? kBand : 0.f) + kBroadMargin;
    if (PASS == 2) lim = fminf(m, key_float(*(volatile int*)&sh.best_key)) + kBroadMargin;
    const int u = u0 + lane;
    bool need = false;
    if (u < nu) {
      const int o = f + u / ntri, k = u - (o - f) * ntri;
      const float4 p = sm.opose[o];
      const Tri T = load_tri(tri, k, ref);
      const float L = sqrtf(point_tri_d2(make_float3(p.x - ref.x, p.y - ref.y, p.z - ref.z), T)) - sm.osc[o].x;
      need = PASS == 2 ? (L >= kBroadMargin && L < lim) : L < lim;
    }
    if (lane == 0) my_tri += (unsigned long long)min(32, nu - u0);
    unsigned mask = __ballot_sync(0xFFFFFFFFu, need);
#pragma unroll 1
    while (mask) {
      const int uu = u0 + __ffs(mask) - 1;
      mask &= mask - 1;
      const int o = f + uu / ntri, k = uu - (o - f) * ntri;
      const Tri T = load_tri(tri, k, ref);
      const int lo = sm.off[o], hi = sm.off[o + 1];
#pragma unroll 1
      for (int i = lo + lane; i < hi; i += 32) {
        const float4 w = sm.W[i];
        m = fminf(m, sqrtf(point_tri_d2(make_float3(w.x, w.y, w.z), T)) - w.w);
      }
      if (lane == 0) my_tri += (unsigned long long)(hi - lo);
      if (DECIDE) {
        if (__any_sync(0xFFFFFFFFu, m < -kBand)) {
          if (lane == 0) *(volatile int*)&sh.hit = 1;
          return m;
        }
        if (__any_sync(0xFFFFFFFFu, *(volatile int*)&sh.hit != 0)) return m;
      }
    }
    if (DECIDE && __any_sync(0xFFFFFFFFu, *(volatile int*)&sh.hit != 0)) return m;
    if (PASS == 2) {
      const float wm = warp_min(m);
      if (lane == 0 && wm < kFarSentinel) atomicMin(&sh.best_key, float_key(wm));
    }
  }
  return m;
}

// Seed pairs: the first two spheres of every object against those of every
// later object (the later one new, obj >= f), before the pair sweep. They
// are real pairs, so their minimum is an upper bound on the result that the
// sweep's culls use from its first unit; where two objects overlap it is
// usually close to the final minimum (decide mode: usually already a certain
// collision). Warps take the later object, lanes the earlier one. Returns
// the thread's minimum.
__device__ __forceinline__ float seed_pairs(const Smem& sm, int f, int n, float m, int lane, int warp, int nwarps) {
#pragma unroll 1
  for (int b = f + warp; b < n; b += nwarps) {
    const int b0 = sm.off[b], nb = sm.off[b + 1] - b0;
    if (nb == 0) continue;
    const float4 wb0 = sm.W[b0], wb1 = sm.W[b0 + (nb > 1)];
#pragma unroll 1
    for (int a = lane; a < b; a += 32) {
      const int a0 = sm.off[a], na = sm.off[a + 1] - a0;
      if (na == 0) continue;
      const float4 wa0 = sm.W[a0], wa1 = sm.W[a0 + (na > 1)];
      // with one sphere on a side its "second" is the first again: a repeat, not a wrong pair
      m = fminf(m, sphere_distance(wa0.x, wa0.y, wa0.z, wa0.w, wb0));
      m = fminf(m, sphere_distance(wa0.x, wa0.y, wa0.z, wa0.w, wb1));
      m = fminf(m, sphere_distance(wa1.x, wa1.y, wa1.z, wa1.w, wb0));
      m = fminf(m, sphere_distance(wa1.x, wa1.y, wa1.z, wa1.w, wb1));
    }
  }
  return m;
}

// Warps pull units until none are left; returns the warp's result (MIN: its
// running minimum; DECIDE: the minimum of the exact distances it computed).
// A unit's B segment is swept one B object ob at a time, each A slot taking
// part only where its object oa comes before ob and the two bounding balls
// can reach the threshold: |c_a - c_b| - R_a - R_b (below every sphere pair's
// distance between the two objects) under thr + kBroadMargin. A B object no
// slot of the warp reaches is skipped.
template <int APL, bool DECIDE>
__device__ __forceinline__ float pair_units(const Smem& sm, CtaShared& sh, int f, int n, int S, int seg_len, float m,
                                            float rmax, float eps, int lane, unsigned long long& my_pairs) {
  constexpr int BA = 32 * APL;
  const int B_lo = sm.off[f];
  const int A_end = sm.off[n - 1];
  const int total_units = sh.total_units;
  const int nb = sh.nb;
  for (;;) {
    int u = 0;
    if (lane == 0) u = atomicAdd(&sh.unit_next, 1);
    u = __shfl_sync(0xFFFFFFFFu, u, 0);
    if (u >= total_units) break;
    {  // CTA-wide state, broadcast so m stays warp-uniform
      int key = 0;
      if (lane == 0) key = DECIDE ? *(volatile int*)&sh.hit : *(volatile int*)&sh.best_key;
      key = __shfl_sync(0xFFFFFFFFu, key, 0);
      if (DECIDE) {
        if (key) break;
      } else {
        m = fminf(m, key_float(key));
      }
    }
    const int bk = upper_index(sm.blk_pref, nb + 1, u);
    const int seg = u - sm.blk_pref[bk];
    const int i0 = bk * BA, i1 = min(i0 + BA, A_end);
    const int lo = sm.blk_lo[bk];
    const int j0 = lo + seg * seg_len;
    const int j1 = min(j0 + seg_len, S);
    ABlock<APL> A;
    int oa[APL];  // object of each A slot (-1: padding)
#pragma unroll
    for (int s = 0; s < APL; ++s) {
      const int i = i0 + s * 32 + lane;
      const bool valid = i < i1;
      const float4 w = valid ? sm.W[i] : make_float4(0.f, 0.f, 0.f, 0.f);
      A.ax[s] = -2.f * w.x; A.ay[s] = -2.f * w.y; A.az[s] = -2.f * w.z;
      A.a2[s] = w.x * w.x + w.y * w.y + w.z * w.z;
      A.r[s] = w.w;
      oa[s] = valid ? (int)sm.oid[i] : -1;
      A.bst[s] = valid ? max(B_lo, sm.off[oa[s] + 1]) : INT_MAX;
    }
    bool alive = refresh<APL, DECIDE>(A, m, rmax, eps);
    if (!alive) continue;
    for (int j = max(j0, lo); j < j1;) {
      const int ob = sm.oid[j];
      const int je = min(j1, sm.off[ob + 1]);
      const float4 pb = sm.opose[ob];
      const float rb = sm.osc[ob].x;
      const float lim = (DECIDE ? kBand : m) + kBroadMargin + rb;
      bool any = false, cut = false;
#pragma unroll
      for (int s = 0; s < APL; ++s) {
        if (!A.act[s]) continue;
        bool near = false;
        if (oa[s] < ob) {
          // |c_a - c_b| < thr + margin + R_a + R_b, squared (false if the right side is <= 0)
          const float4 pa = sm.opose[oa[s]];
          const float dx = pa.x - pb.x, dy = pa.y - pb.y, dz = pa.z - pb.z;
          const float t = lim + sm.osc[oa[s]].x;
          near = t > 0.f && dx * dx + dy * dy + dz * dz < t * t;
        }
        if (near) {
          my_pairs += (unsigned long long)(je - j);
          any = true;
        } else {
          A.al[s] = kRetired;  // left out of this B object only
          cut = true;
        }
      }
      bool fresh = false;  // every slot's threshold already re-derived
      if (__any_sync(0xFFFFFFFFu, any)) {
        const float m0 = m;
        sweep<APL, false, DECIDE>(A, sm.W, sm.beta, j, je, S, m, rmax, eps, &sh.best_key, &sh.hit, alive);
        if (!alive) break;  // DECIDE: a certain collision; MIN: every slot retired
        fresh = !DECIDE && m != m0;  // MIN re-derives the thresholds when m drops
      }
      if (!fresh && __any_sync(0xFFFFFFFFu, cut)) alive = refresh<APL, DECIDE>(A, m, rmax, eps);
      j = je;
    }
    if (DECIDE && !alive) break;
  }
  return m;
}

// Bulk asynchronous copy of the local sphere block into shared memory: one
// thread arms the mbarrier with the byte count and issues the copy; every
// thread waits for the phase with a cycle budget (false: it ran out).
__device__ __forceinline__ void bulk_stage_issue(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
  const uint32_t b = static_cast<uint32_t>(__cvta_generic_to_shared(bar));
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
  for (uint32_t off = 0; off < bytes; off += 32768) {
    const uint32_t n = bytes - off < 32768 ? bytes - off : 32768;
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d + off),
                 "l"(static_cast<const char*>(src) + off), "r"(n), "r"(b)
                 : "memory");
  }
}

__device__ __forceinline__ bool bulk_stage_wait(unsigned long long* bar, uint32_t parity) {
  const uint32_t b = static_cast<uint32_t>(__cvta_generic_to_shared(bar));
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(b), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > 4000000000LL) return false;  // about 2 s
  }
}

struct KArgs {
  sc_scene_batch b;
  CollideLaunch a;
  int seg_len;
  int stage_bulk;  // the local sphere block arrives by one bulk copy
};

// MINB = 2 caps a 512-thread instantiation at 64 registers (four 256-thread
// CTAs per SM where shared memory allows); MINB = 1 leaves the pair sweep its
// registers where shared memory holds one or two CTAs per SM anyway.
template <int APL, int MAXT, int MINB, bool DECIDE>
__global__ void __launch_bounds__(MAXT, MINB) collide_kernel(KArgs K) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ CtaShared sh;
  const sc_scene_batch& b = K.b;
  const CollideLaunch& a = K.a;
  const Layout L = make_layout(b.max_sph, b.max_obj, APL);
  const Smem sm = smem_view(smem, L);
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
  unsigned long long my_pairs = 0, my_box = 0, my_tri = 0;

  // the next candidate is claimed while this one is reduced: thread 0 stores
  // it in sh.item just before the candidate's last barrier
  if (tid == 0) {
    sh.item = (int)atomicAdd(a.counter, 1u);
    if (K.stage_bulk) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(
                       static_cast<uint32_t>(__cvta_generic_to_shared(&sh.bar)))
                   : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  __syncthreads();
  uint32_t bulk_phase = 0;
  for (;;) {
    const int item = sh.item;
    if (item >= a.n_items) break;
    int next = 0;
    if (tid == 0) next = (int)atomicAdd(a.counter, 1u);
    const int c = a.active ? __ldg(&a.active[item]) : item;
    const int t = template_of(b, c);
    int o0 = 0, nt = 0, s0 = 0, S = 0, nobb = 0, bx0 = 0, ntri = 0;
    const float* tri = nullptr;
    int64_t pbase = 0;
    if (t >= 0 && b.n_tri > 0) {
      const int q0 = __ldg(&b.tmpl_tri_off[t]);
      ntri = __ldg(&b.tmpl_tri_off[t + 1]) - q0;
      tri = b.tri + 12 * (int64_t)q0;
    }
    if (t >= 0) {
      o0 = __ldg(&b.tmpl_obj_off[t]);
      nt = __ldg(&b.tmpl_obj_off[t + 1]) - o0;
      s0 = __ldg(&b.obj_sph_off[o0]);
      S = __ldg(&b.obj_sph_off[o0 + nt]) - s0;
      bx0 = __ldg(&b.tmpl_obb_off[t]);
      nobb = __ldg(&b.tmpl_obb_off[t + 1]) - bx0;
      pbase = __ldg(&b.tmpl_pose_off[t]) + (int64_t)(c - __ldg(&b.cand_tmpl_off[t])) * nt;
    }
    const int err = t < 0 ? kDevBadTemplate
                    : (S > b.max_sph || S + kPad > L.cap) ? kDevTooManySpheres
                    : (nt > b.max_obj || nt > kMaxObj || nt < 1) ? kDevTooManyObjects
                    : (nobb > kMaxObbPerTemplate) ? kDevTooManyBoxes
                    : (ntri < 0 || ntri > kMaxTriPerTemplate) ? kDevTooManyTriangles : kDevOk;
    if (err != kDevOk) {
      if (tid == 0) {
        latch_error(a.status, err);
        a.collide[item] = 0;
        a.min_dist[item] = __int_as_float(0x7FC00000);
        a.band[item] = 1;
      }
      __syncthreads();  // every thread has read sh.item
      if (tid == 0) sh.item = next;
      __syncthreads();
      continue;
    }
    const int f = a.first_new;
    // this thread's generic accesses of W (the previous candidate) are
    // ordered before the bulk copy that overwrites it (issued after a barrier)
    if (K.stage_bulk) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    stage_objects(b, reinterpret_cast<const float4*>(a.poses), pbase, o0, s0, nt, sm, tid, nthr);
    if (tid == 0) {
      sh.best_key = float_key(kFarSentinel);
      sh.r2max_key = 0;
      sh.rmax_key = 0;
      sh.hit = 0;
      sh.bad_box = 0;
    }
    __syncthreads();
    if (K.stage_bulk) {
      if (tid == 0) bulk_stage_issue(sm.W, reinterpret_cast<const float4*>(b.sph_local) + s0, 16u * (uint32_t)S, &sh.bar);
      const bool landed = bulk_stage_wait(&sh.bar, bulk_phase);
      if (!__syncthreads_and(landed)) {  // the copy did not arrive: no verdict, stop this CTA
        if (tid == 0) {
          latch_error(a.status, kDevTimeout);
          a.collide[item] = 0;
          a.min_dist[item] = __int_as_float(0x7FC00000);
          a.band[item] = 1;
        }
        bulk_stage_wait(&sh.bar, bulk_phase);  // do not leave the copy in flight into freed shared memory
        break;
      }
      bulk_phase ^= 1u;
    }
    stage_spheres(b, s0, nt, S, sm, sh, tid, nthr, lane, K.stage_bulk != 0);
    stage_boxes(b, t, c, bx0, nobb, sm, tid, nthr, a.status, &sh.bad_box);
    __syncthreads();
    if (*(volatile int*)&sh.bad_box) {  // a malformed part box: no verdict, marked like the checks above
      __syncthreads();  // every thread has read the flag
      if (tid == 0) {
        a.collide[item] = 0;
        a.min_dist[item] = __int_as_float(0x7FC00000);
        a.band[item] = 1;
        sh.item = next;
      }
      __syncthreads();
      continue;
    }
    const float rmax = __int_as_float(sh.rmax_key);
    const float eps = 1e-5f * (__int_as_float(sh.r2max_key) + 0.01f);
    float m = kFarSentinel;
    bool pairs = f < nt;
    if (pairs && (nobb > 0 || ntri > 0)) {
      if (DECIDE) {
        if (nobb > 0) m = box_units<0>(sm, sh, f, nt, nobb, m, lane, warp, nwarps, my_box);
        if (ntri > 0 && !__any_sync(0xFFFFFFFFu, *(volatile int*)&sh.hit != 0))
          m = tri_units<0>(sm, sh, tri, f, nt, ntri, m, lane, warp, nwarps, my_tri);
      } else {
        if (nobb > 0) m = box_units<1>(sm, sh, f, nt, nobb, m, lane, warp, nwarps, my_box);
        if (ntri > 0) m = tri_units<1>(sm, sh, tri, f, nt, ntri, m, lane, warp, nwarps, my_tri);
        const float wm = warp_min(m);
        if (lane == 0 && wm < kFarSentinel) atomicMin(&sh.best_key, float_key(wm));
        __syncthreads();
        // a unit left for pass 2 has L >= kBroadMargin: it can only matter
        // while the minimum so far is positive
        if (key_float(*(volatile int*)&sh.best_key) > 0.f) {
          if (nobb > 0) m = box_units<2>(sm, sh, f, nt, nobb, m, lane, warp, nwarps, my_box);
          if (ntri > 0) m = tri_units<2>(sm, sh, tri, f, nt, ntri, m, lane, warp, nwarps, my_tri);
        }
      }
      m = warp_min(m);
      if (!DECIDE && lane == 0 && m < kFarSentinel) atomicMin(&sh.best_key, float_key(m));
      if (DECIDE && lane == 0 && m < -kBand) *(volatile int*)&sh.hit = 1;
      __syncthreads();
      // A computed sphere-pair distance is never below -(r_i + r_j) >= -2 rmax
      // (rounding is monotone), so a box distance under that already is the
      // minimum; a certain collision already is the decision.
      pairs = DECIDE ? !*(volatile int*)&sh.hit : key_float(*(volatile int*)&sh.best_key) >= -2.f * rmax;
    }
    if (pairs) {
      m = seed_pairs(sm, f, nt, m, lane, warp, nwarps);
      m = warp_min(m);
      if (lane == 0) {
        if (!DECIDE && m < kFarSentinel) atomicMin(&sh.best_key, float_key(m));
        if (DECIDE && m < -kBand) *(volatile int*)&sh.hit = 1;
      }
      if (warp == 0) build_units(f, nt, S, 32 * APL, K.seg_len, sm, sh, lane);
      __syncthreads();
      m = pair_units<APL, DECIDE>(sm, sh, f, nt, S, K.seg_len, m, rmax, eps, lane, my_pairs);
    }
    m = warp_min(m);
    if (lane == 0) sh.warp_min[warp] = m;
    __syncthreads();
    if (tid == 0) {
      float mm = DECIDE ? kFarSentinel : key_float(sh.best_key);
      for (int w = 0; w < nwarps; ++w) mm = fminf(mm, sh.warp_min[w]);
      const float out = mm >= 0.5f * kFarSentinel ? FLT_MAX : mm;
      a.min_dist[item] = out;
      a.collide[item] = out < 0.f;
      a.band[item] = fabsf(out) <= kBand;
      sh.item = next;
    }
    __syncthreads();
  }
  // per-CTA work statistics
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    my_pairs += __shfl_xor_sync(0xFFFFFFFFu, my_pairs, o);
    my_box += __shfl_xor_sync(0xFFFFFFFFu, my_box, o);
    my_tri += __shfl_xor_sync(0xFFFFFFFFu, my_tri, o);
  }
  if (lane == 0 && a.stats) {
    atomicAdd(&a.stats[0], my_pairs);
    atomicAdd(&a.stats[1], my_box);
    atomicAdd(&a.stats[7], my_tri);
  }
}

template <int APL, int MAXT, int MINB, bool DECIDE>
cudaError_t launch_t(const KArgs& K, const sc_collide_config& cfg, size_t smem, int num_sms, cudaStream_t s) {
  auto kern = collide_kernel<APL, MAXT, MINB, DECIDE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, cfg.threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int grid = num_sms * (cfg.ctas_per_sm < per_sm ? cfg.ctas_per_sm : per_sm);
  if (grid > K.a.n_items) grid = K.a.n_items;
  kern<<<grid, cfg.threads, smem, s>>>(K);
  return cudaGetLastError();
}

template <bool DECIDE>
cudaError_t launch_mode(const KArgs& K, const sc_collide_config& cfg, size_t smem, int num_sms, cudaStream_t s) {
  switch (cfg.a_per_lane) {
    case 1: return launch_t<1, 1024, 1, DECIDE>(K, cfg, smem, num_sms, s);
    case 2: return launch_t<2, 1024, 1, DECIDE>(K, cfg, smem, num_sms, s);
    default:
      return 3 * (smem + 1024) <= 228 * 1024 ? launch_t<4, 512, 2, DECIDE>(K, cfg, smem, num_sms, s)
                                              : launch_t<4, 512, 1, DECIDE>(K, cfg, smem, num_sms, s);
  }
}

}  // namespace

// A candidate of up to 256 spheres is one or two register blocks of four
// spheres per lane: small CTAs with one sphere per lane and short B segments
// spread its few pairs over more warps and keep eight candidates per SM in
// flight (tabletop batch, 8 x 16 spheres: 2.3 ms against 9.8 ms exact, 1.2
// against 2.9 ms decide, for 262,144 candidates).
sc_collide_config default_collide_config(const sc_scene_batch& b) {
  return b.max_sph <= 256 ? sc_collide_config{128, 1, 32, 8, 0, 0} : sc_collide_config{256, 4, 256, 4, 0, 0};
}

size_t collide_smem_bytes(const sc_scene_batch& b, const sc_collide_config& cfg) {
  return (size_t)make_layout(b.max_sph, b.max_obj, cfg.a_per_lane).total;
}

const char* check_collide_config(const sc_collide_config& cfg) {
  if (cfg.a_per_lane != 1 && cfg.a_per_lane != 2 && cfg.a_per_lane != 4) return "a_per_lane must be 1, 2 or 4";
  const int maxt = cfg.a_per_lane == 4 ? 512 : 1024;
  if (cfg.threads < 128 || cfg.threads > maxt || cfg.threads % 32)
    return "threads must be a multiple of 32 in 128..1024 (..512 when a_per_lane = 4)";
  if (cfg.seg_len < 8 || cfg.seg_len > 4096 || cfg.seg_len % 8) return "seg_len must be a multiple of 8 in 8..4096";
  if (cfg.ctas_per_sm < 1 || cfg.ctas_per_sm > 8) return "ctas_per_sm must be in 1..8";
  if (cfg.decide_only != 0 && cfg.decide_only != 1) return "decide_only must be 0 or 1";
  if (cfg.stage_bulk != 0 && cfg.stage_bulk != 1) return "stage_bulk must be 0 or 1";
  return nullptr;
}

cudaError_t launch_collide(const sc_scene_batch& b, const CollideLaunch& a, const sc_collide_config& cfg, int num_sms,
                           cudaStream_t s, const char** why) {
  *why = check_collide_config(cfg);
  if (*why) return cudaErrorInvalidValue;
  const size_t smem = collide_smem_bytes(b, cfg);
  if (smem > 227 * 1024) { *why = "batch needs more shared memory than one CTA has (max_sph too large)"; return cudaErrorInvalidValue; }
  cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  if (a.stats && (e = cudaMemsetAsync(a.stats, 0, 2 * sizeof(unsigned long long), s)) != cudaSuccess) return e;
  if (a.stats && (e = cudaMemsetAsync(a.stats + 7, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
  if (a.n_items <= 0) return cudaSuccess;
  KArgs K{b, a, cfg.seg_len, cfg.stage_bulk};
  return cfg.decide_only ? launch_mode<true>(K, cfg, smem, num_sms, s) : launch_mode<false>(K, cfg, smem, num_sms, s);
}

}  // namespace sc
