// Device core of the sphere-pair reduction (Sec. IV-D batched collision
// checking; per-object sphere sets stand in for cuRobo's meshes), shared by
// the collision kernel (collide.cu) and the fused generation step
// (generate.cu). Spheres sit in shared memory in the world frame relative to
// one reference point (small coordinates keep the FP32 prune test tight).
//
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

// Signed distance of two spheres (centre (ax, ay, az), radius ar; b): the
// exact value every prune hit is settled with.
__device__ __forceinline__ float sphere_distance(float ax, float ay, float az, float ar, const float4& b) {
  const float dx = ax - b.x, dy = ay - b.y, dz = az - b.z;
  return sqrtf(dx * dx + dy * dy + dz * dz) - ar - b.w;
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
      if (jj >= A.bst[s])  // -ax / 2 is the centre again (scaling by powers of two is exact)
        mloc = fminf(mloc, sphere_distance(-0.5f * A.ax[s], -0.5f * A.ay[s], -0.5f * A.az[s], A.r[s], B));
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

}  // namespace core
}  // namespace sc
