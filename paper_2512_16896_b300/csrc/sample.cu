// Pose sampling kernel (sc_sample_poses): one warp per listed candidate,
// objects in placement order (a child reads its parent's pose), the rejection
// attempts of one object spread over the lanes (see sample_core.cuh).
#include "kernels.h"
#include "sample_core.cuh"

namespace sc {

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
    const Support sup = warp_support(b, t, lane);
    if (!sup.ok) {
      if (lane == 0) { latch_error(status, kDevBadPolygon); out_ok[item] = 0; out_band[item] = 1; }
      continue;
    }
    bool all_ok = true, any_band = false;
    const int k_end = min(nt, p.first_obj + p.n_obj);
    for (int k = p.first_obj; k < k_end; ++k) {
      __syncwarp();  // earlier poses written by lane 0 are visible to the warp
      const SampleResult r = warp_sample_object(b, sup, p.seed, p.max_attempts, p.retry, c, k, o0, poses, pbase,
                                                status, lane, t);
      if (lane == 0) poses[pbase + k] = r.pose;
      all_ok = all_ok && r.placed;
      any_band = any_band || r.band;
    }
    if (lane == 0) {
      out_ok[item] = all_ok;
      out_band[item] = any_band;
    }
  }
}

// Joint values of the articulated parts (sc_sample_parts): one thread per
// (listed candidate, part slot), q = qmin + (qmax - qmin) u0 with
// u = Philox(seed; c, 0xFFFF0000 + j, 0, 0), counters no pose draw uses.
__global__ void __launch_bounds__(256) sample_parts_kernel(sc_scene_batch b, uint64_t seed, const int32_t* active,
                                                           int n_items, float* part_q, int* status) {
  const int64_t total = (int64_t)n_items * b.max_parts;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int item = (int)(i / b.max_parts), j = (int)(i % b.max_parts);
    const int c = active ? __ldg(&active[item]) : item;
    const int t = template_of(b, c);
    if (t < 0) {
      if (j == 0) latch_error(status, kDevBadTemplate);
      continue;
    }
    const int p0 = __ldg(&b.tmpl_part_off[t]), np = __ldg(&b.tmpl_part_off[t + 1]) - p0;
    if (np > b.max_parts && j == 0) latch_error(status, kDevBadPart);
    if (j >= np) continue;
    const float qmin = __ldg(&b.part_param[12 * (int64_t)(p0 + j) + 3]);
    const float qmax = __ldg(&b.part_param[12 * (int64_t)(p0 + j) + 4]);
    const float4 u = draw_uniform4(seed, (uint32_t)c, 0xFFFF0000u + (uint32_t)j, 0u, 0u);
    part_q[(int64_t)c * b.max_parts + j] = qmin + (qmax - qmin) * u.x;
  }
}

cudaError_t launch_sample_parts(const sc_scene_batch& b, uint64_t seed, const int32_t* active, int n_items,
                                float* part_q, int* status, int num_sms, cudaStream_t s) {
  const int threads = 256;
  const int64_t total = (int64_t)n_items * b.max_parts;
  int64_t blocks = (total + threads - 1) / threads;
  blocks = blocks < num_sms * 8 ? blocks : num_sms * 8;
  if (blocks < 1) return cudaSuccess;
  sample_parts_kernel<<<(int)blocks, threads, 0, s>>>(b, seed, active, n_items, part_q, status);
  return cudaGetLastError();
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
