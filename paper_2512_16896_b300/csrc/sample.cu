// Pose sampling: free / on-top / next-to proposals with point-in-polygon
// rejection (Sec. III position sampling, Sec. IV-C batch sampling with the
// canonical polygon moved per instance, Sec. IV-F relations and
// ratio_on_support erosion).
//
// One warp per listed candidate. Objects are sampled in placement order (a
// child reads its parent's pose); within one object the rejection attempts
// run in parallel, one per lane, and a ballot picks the lowest accepted
// attempt, which is exactly the outcome of trying them one after another.
#include "common.cuh"
#include "kernels.h"

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

__global__ void __launch_bounds__(256) sample_kernel(sc_scene_batch b, sc_sample_params p, const int32_t* active,
                                                     int n_items, float4* poses, uint8_t* out_ok, uint8_t* out_band,
                                                     int* status) {
  const int lane = threadIdx.x & 31;
  const int warps_per_block = blockDim.x >> 5;
  for (int item = blockIdx.x * warps_per_block + (threadIdx.x >> 5); item < n_items;
       item += gridDim.x * warps_per_block) {
    const int c = active ? __ldg(&active[item]) : item;
    const int t = template_of(b, c);
    if (t < 0) {
      if (lane == 0) { latch_error(status, kDevBadTemplate); out_ok[item] = 0; out_band[item] = 1; }
      continue;
    }
    const int o0 = __ldg(&b.tmpl_obj_off[t]);
    const int nt = __ldg(&b.tmpl_obj_off[t + 1]) - o0;
    const int64_t pbase = __ldg(&b.tmpl_pose_off[t]) + (int64_t)(c - __ldg(&b.cand_tmpl_off[t])) * nt;
    PolyView P{reinterpret_cast<const float2*>(b.poly_verts) + __ldg(&b.tmpl_poly_off[t]),
               __ldg(&b.tmpl_poly_off[t + 1]) - __ldg(&b.tmpl_poly_off[t])};
    if (P.n < 3 || P.n > kMaxPolyVerts) {
      if (lane == 0) { latch_error(status, kDevBadPolygon); out_ok[item] = 0; out_band[item] = 1; }
      continue;
    }
    // bounding box of the support polygon (warp reduction over vertices)
    float xmin = 3e38f, xmax = -3e38f, ymin = 3e38f, ymax = -3e38f;
    for (int i = lane; i < P.n; i += 32) {
      float2 v = __ldg(&P.v[i]);
      xmin = fminf(xmin, v.x); xmax = fmaxf(xmax, v.x);
      ymin = fminf(ymin, v.y); ymax = fmaxf(ymax, v.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      xmin = fminf(xmin, __shfl_xor_sync(0xFFFFFFFFu, xmin, o));
      xmax = fmaxf(xmax, __shfl_xor_sync(0xFFFFFFFFu, xmax, o));
      ymin = fminf(ymin, __shfl_xor_sync(0xFFFFFFFFu, ymin, o));
      ymax = fmaxf(ymax, __shfl_xor_sync(0xFFFFFFFFu, ymax, o));
    }
    const float zs = __ldg(&b.tmpl_support_z[t]);
    bool all_ok = true, any_band = false;
    const int k_end = min(nt, p.first_obj + p.n_obj);
    for (int k = p.first_obj; k < k_end; ++k) {
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
      __syncwarp();  // earlier poses written by lane 0 are visible to the warp
      if (kind == SC_REL_ON_TOP) {
        if (lane == 0) {
          const float4 u = draw_uniform4(p.seed, (uint32_t)c, (uint32_t)k, (uint32_t)p.retry, 0u);
          const float4 pp = poses[pbase + ref];
          const float4 pH = __ldg(reinterpret_cast<const float4*>(b.obj_half) + (o0 + ref));
          const float xl = pH.x * (2.f * u.x - 1.f), yl = pH.y * (2.f * u.y - 1.f);
          float sy, cy;
          sincosf(pp.w, &sy, &cy);
          poses[pbase + k] = make_float4(pp.x + cy * xl - sy * yl, pp.y + sy * xl + cy * yl, pp.z + pH.z + H.z,
                                         kTwoPi * u.z);
        }
        continue;
      }
      const float e = RP.z * fminf(H.x, H.y);  // ratio_on_support erosion
      float4 anchor = make_float4(0.f, 0.f, 0.f, 0.f);
      float rho_sum = 0.f;
      if (kind == SC_REL_NEXT_TO) {
        anchor = poses[pbase + ref];
        rho_sum = __ldg(&b.obj_half[4 * (o0 + ref) + 3]) + H.w;
      }
      bool placed = false, band_obj = false;
      float4 pose = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int a0 = 0; a0 < p.max_attempts && !placed; a0 += 32) {
        const int a = a0 + lane;
        const bool valid = a < p.max_attempts;
        float x = 0.f, y = 0.f, yaw = 0.f;
        bool acc = false, bnd = false;
        if (valid) {
          const float4 u = draw_uniform4(p.seed, (uint32_t)c, (uint32_t)k, (uint32_t)p.retry, (uint32_t)a);
          if (kind == SC_REL_NEXT_TO) {
            float sp, cp;
            sincosf(kTwoPi * u.x, &sp, &cp);
            const float r = rho_sum + RP.x + (RP.y - RP.x) * u.y;
            x = anchor.x + r * cp;
            y = anchor.y + r * sp;
          } else {
            x = xmin + (xmax - xmin) * u.x;
            y = ymin + (ymax - ymin) * u.y;
          }
          yaw = kTwoPi * u.z;
          float dist;
          const bool inside = pip_with_distance(P, x, y, &dist);
          acc = inside && dist >= e;
          bnd = dist <= kBand || (inside && fabsf(dist - e) <= kBand);
        }
        const unsigned acc_mask = __ballot_sync(0xFFFFFFFFu, acc);
        const unsigned bnd_mask = __ballot_sync(0xFFFFFFFFu, bnd);
        int src;
        if (acc_mask) {
          src = __ffs(acc_mask) - 1;
          const unsigned upto = (src == 31) ? 0xFFFFFFFFu : ((2u << src) - 1u);
          band_obj = band_obj || (bnd_mask & upto);
          placed = true;
        } else {
          band_obj = band_obj || bnd_mask;
          src = min(31, p.max_attempts - 1 - a0);  // last attempt of this chunk
        }
        pose.x = __shfl_sync(0xFFFFFFFFu, x, src);
        pose.y = __shfl_sync(0xFFFFFFFFu, y, src);
        pose.w = __shfl_sync(0xFFFFFFFFu, yaw, src);
      }
      pose.z = zs + H.z;
      if (lane == 0) poses[pbase + k] = pose;
      all_ok = all_ok && placed;
      any_band = any_band || band_obj;
    }
    if (lane == 0) {
      out_ok[item] = all_ok;
      out_band[item] = any_band;
    }
  }
}

cudaError_t launch_sample(const sc_scene_batch& b, const sc_sample_params& p, const int32_t* active, int n_items,
                          float* poses, uint8_t* ok, uint8_t* band, int* status, int num_sms, cudaStream_t s) {
  const int threads = 256, warps = threads / 32;
  int blocks = (n_items + warps - 1) / warps;
  blocks = blocks < num_sms * 8 ? blocks : num_sms * 8;
  if (blocks < 1) return cudaSuccess;
  sample_kernel<<<blocks, threads, 0, s>>>(b, p, active, n_items, reinterpret_cast<float4*>(poses), ok, band, status);
  return cudaGetLastError();
}

}  // namespace sc
