// Device core of the collision reduction (Sec. IV-B one transform per
// instance, Sec. IV-D batched collision checking; per-object sphere sets and
// oriented boxes stand in for cuRobo's meshes). Shared by the collision
// kernel and the fused generation step.
//
// One CTA handles one candidate at a time:
//  * stage_*: the candidate's objects [0, n) are moved to shared memory once,
//    spheres in the world frame relative to the position of object 0 (small
//    coordinates keep the FP32 prune test tight);
//  * build_units: the pair set {(i, j): obj(i) < obj(j), obj(j) >= f} is cut
//    into units (A block of 32*APL consecutive spheres, one per lane per
//    slot) x (B segment of up to seg_len spheres); warps pull units from a
//    CTA-local counter;
//  * sweep: per pair, with q_i = r_i + m (m = threshold), the pair can reach
//    a distance below m iff |a - b|^2 < (q_i + r_j)^2, i.e.
//        (|a|^2 - q_i^2) + (|b|^2 - r_j^2) - 2 a.b - 2 q_i r_j  <  0,
//    one add and four FMAs with per-sphere terms precomputed. A slack eps
//    (bounding the FP32 rounding of that sum) makes the test never miss; a
//    group of pairs with a hit recomputes sqrt(|a - b|^2) - r_i - r_j
//    exactly. Two modes:
//      MIN    m = running minimum; the result is the exact minimum over all
//             pairs. A sphere with r_i + m + max r_j < 0 can no longer lower
//             m and is retired; a unit whose A spheres all retired is skipped.
//      DECIDE m = +1e-5 fixed (the decision band); exact distances of hits
//             are folded into the result, and the first distance below
//             -1e-5 (a certain collision) stops the candidate.
#pragma once

#include <cfloat>
#include <climits>

#include "common.cuh"

namespace sc {
namespace core {

constexpr int kPad = 8;    // dummy spheres after the last one (group tail reads)
constexpr int kGroup = 4;  // B spheres per prune group
constexpr float kRetired = 1e30f;

__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }

struct Layout {
  int W, beta, oid, off, opose, osc, obb, blk_lo, blk_mend, blk_pref, total, nb_max, cap;
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
  L.blk_mend = align16(L.blk_lo + 4 * L.nb_max);
  L.blk_pref = align16(L.blk_mend + 4 * L.nb_max);
  L.total = align16(L.blk_pref + 4 * (L.nb_max + 1));
  return L;
}

struct Smem {
  float4* W;
  float* beta;
  uint8_t* oid;
  int* off;
  float4* opose;
  float2* osc;
  float* obbd;
  int* blk_lo;
  int* blk_mend;
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
  s.blk_mend = reinterpret_cast<int*>(base + L.blk_mend);
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
  float warp_min[32];
  float4 new_pose;         // generation: the sampled pose of the new object
  int new_ok, new_band;
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

// Poses, sin/cos of yaw and sphere offsets of objects [0, n). Plain loads:
// the generation step writes poses earlier in the same kernel.
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
// 0's position, plus |c|^2 - r^2; kPad far-away dummies after them.
__device__ __forceinline__ void stage_spheres(const sc_scene_batch& b, int s0, int n, int S, const Smem& sm,
                                              CtaShared& sh, int tid, int nthr, int lane) {
  const float4 ref = sm.opose[0];
  float r2max = 0.f, rmx = 0.f;
  for (int q = tid; q < S + kPad; q += nthr) {
    if (q < S) {
      const int k = upper_index(sm.off, n + 1, q);
      const float4 l = __ldg(reinterpret_cast<const float4*>(b.sph_local) + s0 + q);
      const float4 p = sm.opose[k];
      const float2 sc2 = sm.osc[k];
      const float x = (p.x - ref.x) + (sc2.y * l.x - sc2.x * l.y);
      const float y = (p.y - ref.y) + (sc2.x * l.x + sc2.y * l.y);
      const float z = (p.z - ref.z) + l.z;
      const float c2 = x * x + y * y + z * z;
      sm.W[q] = make_float4(x, y, z, l.w);
      sm.beta[q] = c2 - l.w * l.w;
      sm.oid[q] = (uint8_t)k;
      r2max = fmaxf(r2max, c2);
      rmx = fmaxf(rmx, l.w);
    } else {
      sm.W[q] = make_float4(1e6f, 1e6f, 1e6f, 0.f);
      sm.beta[q] = 3e12f;
      sm.oid[q] = 255;
    }
  }
  r2max = -warp_min(-r2max);
  rmx = -warp_min(-rmx);
  if (lane == 0) {
    atomicMax(&sh.r2max_key, __float_as_int(r2max));  // non-negative floats order as ints
    atomicMax(&sh.rmax_key, __float_as_int(rmx));
  }
}

// World boxes: columns of R, centre relative to object 0, half extents.
__device__ __forceinline__ void stage_boxes(const sc_scene_batch& b, int bx0, int nobb, const Smem& sm, int tid,
                                            int nthr) {
  const float4 ref = sm.opose[0];
  for (int k = tid; k < nobb; k += nthr) {
    const float* o = b.obb + 12 * (bx0 + k);
    float qx = __ldg(o + 4), qy = __ldg(o + 5), qz = __ldg(o + 6), qw = __ldg(o + 7);
    const float inv = rsqrtf(qx * qx + qy * qy + qz * qz + qw * qw);
    qx *= inv; qy *= inv; qz *= inv; qw *= inv;
    float* d = sm.obbd + 16 * k;
    // R (row-major) of the unit quaternion; stored by columns
    d[0] = 1.f - 2.f * (qy * qy + qz * qz); d[1] = 2.f * (qx * qy + qz * qw); d[2] = 2.f * (qx * qz - qy * qw);
    d[3] = 2.f * (qx * qy - qz * qw); d[4] = 1.f - 2.f * (qx * qx + qz * qz); d[5] = 2.f * (qy * qz + qx * qw);
    d[6] = 2.f * (qx * qz + qy * qw); d[7] = 2.f * (qy * qz - qx * qw); d[8] = 1.f - 2.f * (qx * qx + qy * qy);
    d[9] = __ldg(o + 0) - ref.x; d[10] = __ldg(o + 1) - ref.y; d[11] = __ldg(o + 2) - ref.z;
    d[12] = __ldg(o + 8); d[13] = __ldg(o + 9); d[14] = __ldg(o + 10); d[15] = 0.f;
  }
}

// Thread 0: work units for pairs (i, j), obj(i) < obj(j), obj(j) in [f, n).
__device__ __forceinline__ void build_units(int f, int n, int S, int BA, int seg_len, const Smem& sm, CtaShared& sh) {
  int total = 0, nb = 0;
  if (f < n) {
    const int B_lo = sm.off[f];
    const int A_end = sm.off[n - 1];
    if (A_end > 0) {
      nb = (A_end + BA - 1) / BA;
      for (int bk = 0; bk < nb; ++bk) {
        const int i0 = bk * BA, i1 = min(i0 + BA, A_end);
        const int lo = max(B_lo, sm.off[sm.oid[i0] + 1]);
        const int mend = max(lo, max(B_lo, sm.off[sm.oid[i1 - 1] + 1]));
        sm.blk_lo[bk] = lo;
        sm.blk_mend[bk] = mend;
        sm.blk_pref[bk] = total;
        if (S > lo) total += (S - lo + seg_len - 1) / seg_len;
      }
    }
  }
  sm.blk_pref[nb] = total;
  sh.total_units = total;
  sh.nb = nb;
  sh.unit_next = 0;
}

template <int APL>
struct ABlock {
  float ax[APL], ay[APL], az[APL];  // -2 * centre
  float a2[APL], r[APL];            // |centre|^2, radius
  float qq[APL], al[APL];           // -2 q_i, |a|^2 - q_i^2 - eps (kRetired when retired)
  int bst[APL];                     // first B index this sphere may pair with (INT_MAX: padding)
  bool act[APL];
};

// Threshold per A sphere: MIN uses the running minimum m, DECIDE the band.
template <int APL, bool DECIDE>
__device__ __forceinline__ bool refresh(ABlock<APL>& A, float m, float rmax, float eps) {
  bool any = false;
#pragma unroll
  for (int s = 0; s < APL; ++s) {
    const float q = A.r[s] + (DECIDE ? kBand : m);
    const bool act = (A.bst[s] != INT_MAX) && (DECIDE || q + rmax >= 0.f);
    A.act[s] = act;
    A.qq[s] = -2.f * q;
    A.al[s] = act ? (A.a2[s] - q * q - eps) : kRetired;
    any |= act;
  }
  return __any_sync(0xFFFFFFFFu, any);
}

// Exact distances of the A block against B spheres [j, j + kGroup) (only the
// pairs allowed for each A sphere, only real B spheres), folded into m.
template <int APL>
__device__ __forceinline__ float slow_group(const ABlock<APL>& A, const float4* W, int j, int S, float m) {
  float mloc = m;
#pragma unroll
  for (int g = 0; g < kGroup; ++g) {
    const int jj = j + g;
    if (jj >= S) break;
    const float4 B = W[jj];
#pragma unroll
    for (int s = 0; s < APL; ++s) {
      if (jj >= A.bst[s]) {
        const float dx = -0.5f * A.ax[s] - B.x, dy = -0.5f * A.ay[s] - B.y, dz = -0.5f * A.az[s] - B.z;
        const float d = sqrtf(dx * dx + dy * dy + dz * dz) - A.r[s] - B.w;
        mloc = fminf(mloc, d);
      }
    }
  }
  return warp_min(mloc);
}

// best_key (MIN): CTA-wide minimum to lower; hit (DECIDE, may be NULL): flag
// raised on a certain collision. Either way `alive` turns false when the
// caller should stop this unit.
template <int APL, bool MASKED, bool DECIDE>
__device__ __forceinline__ void sweep(ABlock<APL>& A, const float4* W, const float* beta, int jb, int je, int S,
                                      float& m, float rmax, float eps, int* best_key, int* hit, bool& alive) {
#pragma unroll 1
  for (int j = jb; j < je; j += kGroup) {
    float4 B[kGroup];
    float bt[kGroup];
#pragma unroll
    for (int g = 0; g < kGroup; ++g) {
      B[g] = W[j + g];
      bt[g] = beta[j + g];
    }
    float v[APL * kGroup];
#pragma unroll
    for (int s = 0; s < APL; ++s) {
#pragma unroll
      for (int g = 0; g < kGroup; ++g) {
        float x = A.al[s] + bt[g];
        x = fmaf(A.ax[s], B[g].x, x);
        x = fmaf(A.ay[s], B[g].y, x);
        x = fmaf(A.az[s], B[g].z, x);
        x = fmaf(A.qq[s], B[g].w, x);
        if (MASKED) x = (j + g >= A.bst[s]) ? x : 1.f;
        v[s * kGroup + g] = x;
      }
    }
    // tree minimum (no serial dependency chain through one predicate)
#pragma unroll
    for (int w = (APL * kGroup) / 2; w >= 1; w >>= 1) {
#pragma unroll
      for (int k = 0; k < w; ++k) v[k] = fminf(v[k], v[k + w]);
    }
    if (__any_sync(0xFFFFFFFFu, v[0] < 0.f)) {
      const float mn = slow_group<APL>(A, W, j, S, m);
      if (mn < m) {
        m = mn;
        if (DECIDE) {
          if (m < -kBand) {  // certain collision: stop this candidate
            if (hit && (threadIdx.x & 31) == 0) *(volatile int*)hit = 1;
            alive = false;
            return;
          }
        } else {
          if ((threadIdx.x & 31) == 0) atomicMin(best_key, float_key(m));
          alive = refresh<APL, false>(A, m, rmax, eps);
          if (!alive) return;
        }
      }
    }
  }
}

// Sphere vs world box for spheres [B_lo, S): exact box SDF minus r where the
// lower bound max(q) - r beats the threshold (m in MIN, the band in DECIDE).
template <bool DECIDE>
__device__ __forceinline__ float box_phase(const Smem& sm, int nobb, int B_lo, int S, float m, int tid, int nthr,
                                           unsigned long long& my_box) {
  for (int i = B_lo + tid; i < S; i += nthr) {
    const float4 w = sm.W[i];
    for (int k = 0; k < nobb; ++k) {
      const float* d = sm.obbd + 16 * k;
      const float vx = w.x - d[9], vy = w.y - d[10], vz = w.z - d[11];
      // box frame: p = R^T v, i.e. p_k = (column k of R) . v
      const float px = d[0] * vx + d[1] * vy + d[2] * vz;
      const float py = d[3] * vx + d[4] * vy + d[5] * vz;
      const float pz = d[6] * vx + d[7] * vy + d[8] * vz;
      const float qx = fabsf(px) - d[12], qy = fabsf(py) - d[13], qz = fabsf(pz) - d[14];
      const float qm = fmaxf(qx, fmaxf(qy, qz));
      if (qm - w.w < (DECIDE ? kBand : m)) {
        const float ox = fmaxf(qx, 0.f), oy = fmaxf(qy, 0.f), oz = fmaxf(qz, 0.f);
        const float dist = sqrtf(ox * ox + oy * oy + oz * oz) + fminf(qm, 0.f) - w.w;
        m = fminf(m, dist);
      }
    }
    my_box += (unsigned long long)nobb;
  }
  return m;
}

// Warps pull units until none are left; returns the warp's result (MIN: its
// running minimum; DECIDE: the minimum of the exact distances it computed).
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
    const int lo = sm.blk_lo[bk], mend = sm.blk_mend[bk];
    const int j0 = lo + seg * seg_len;
    const int j1 = min(j0 + seg_len, S);
    ABlock<APL> A;
#pragma unroll
    for (int s = 0; s < APL; ++s) {
      const int i = i0 + s * 32 + lane;
      const bool valid = i < i1;
      const float4 w = valid ? sm.W[i] : make_float4(0.f, 0.f, 0.f, 0.f);
      A.ax[s] = -2.f * w.x; A.ay[s] = -2.f * w.y; A.az[s] = -2.f * w.z;
      A.a2[s] = w.x * w.x + w.y * w.y + w.z * w.z;
      A.r[s] = w.w;
      A.bst[s] = valid ? max(B_lo, sm.off[sm.oid[i] + 1]) : INT_MAX;
    }
    bool alive = refresh<APL, DECIDE>(A, m, rmax, eps);
    if (!alive) continue;
#pragma unroll
    for (int s = 0; s < APL; ++s)
      if (A.act[s]) my_pairs += (unsigned long long)max(0, j1 - max(j0, A.bst[s]));
    const int jm = min(j1, mend);
    if (j0 < jm) sweep<APL, true, DECIDE>(A, sm.W, sm.beta, j0, jm, S, m, rmax, eps, &sh.best_key, &sh.hit, alive);
    if (alive && max(j0, mend) < j1)
      sweep<APL, false, DECIDE>(A, sm.W, sm.beta, max(j0, mend), j1, S, m, rmax, eps, &sh.best_key, &sh.hit, alive);
    if (DECIDE && !alive) break;
  }
  return m;
}

}  // namespace core
}  // namespace sc
