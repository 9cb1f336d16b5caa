// Generation loop (Sec. IV-A and Fig. 2: per object, sample poses, check
// collisions, retry a limited number of times; Sec. IV-D: re-check only the
// scenes that retry; Sec. V-A: 10 retries per object, failing scenes invalid).
//
// One launch per (object k, try r) processes a device-resident list of the
// candidates that still need object k. A persistent CTA takes a candidate,
// its warp 0 samples object k (sample_core.cuh), the CTA moves objects 0..k
// to shared memory and decides whether object k collides with objects
// 0..k-1 or the world (collide_core.cuh, decide mode: exits at the first
// certain collision). Thread 0 then appends the candidate to the list for
// object k+1 (or marks it valid after its last object), to the retry list for
// try r+1, or leaves it invalid after the last try. The launch sequence is a
// fixed function of (max objects, retries), so it is captured once into a
// CUDA graph and replayed.
#include <vector>

#include "collide_core.cuh"
#include "kernels.h"
#include "sample_core.cuh"

namespace sc {

namespace {

using namespace core;

struct GenStepArgs {
  sc_scene_batch b;
  uint64_t seed;
  int max_attempts, retry, max_retries, k, seg_len;
  const int32_t* list_in;
  const int* n_in;
  int32_t* list_retry;
  int* n_retry;
  int32_t* list_next;
  int* n_next;
  float4* poses;
  uint8_t* valid;
  uint8_t* band;
  int32_t* tries;
  unsigned int* counter;
  unsigned long long* stats;
  int* status;
};

template <int APL, int MAXT>
__global__ void __launch_bounds__(MAXT) gen_step_kernel(GenStepArgs g) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ CtaShared sh;
  const sc_scene_batch& b = g.b;
  const Layout L = make_layout(b.max_sph, b.max_obj, APL);
  const Smem sm = smem_view(smem, L);
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
  const int n_items = *(volatile const int*)g.n_in;
  const int k = g.k;
  unsigned long long my_pairs = 0, my_box = 0;

  for (;;) {
    if (tid == 0) sh.item = (int)atomicAdd(g.counter, 1u);
    __syncthreads();
    const int item = sh.item;
    if (item >= n_items) break;
    const int c = __ldg(&g.list_in[item]);
    const int t = template_of(b, c);
    int o0 = 0, nt = 0, s0 = 0, S = 0, nobb = 0, bx0 = 0;
    int64_t pbase = 0;
    if (t >= 0) {
      o0 = __ldg(&b.tmpl_obj_off[t]);
      nt = __ldg(&b.tmpl_obj_off[t + 1]) - o0;
      s0 = __ldg(&b.obj_sph_off[o0]);
      bx0 = __ldg(&b.tmpl_obb_off[t]);
      nobb = __ldg(&b.tmpl_obb_off[t + 1]) - bx0;
      pbase = __ldg(&b.tmpl_pose_off[t]) + (int64_t)(c - __ldg(&b.cand_tmpl_off[t])) * nt;
      if (k < nt) S = __ldg(&b.obj_sph_off[o0 + k + 1]) - s0;  // spheres of objects 0..k
    }
    const int err = t < 0 ? kDevBadTemplate
                    : (k >= nt || nt > b.max_obj || nt > kMaxObj) ? kDevTooManyObjects
                    : (S > b.max_sph || S + kPad > L.cap) ? kDevTooManySpheres
                    : (nobb > kMaxObbPerTemplate) ? kDevTooManyBoxes : kDevOk;
    if (err != kDevOk) {
      if (tid == 0) {
        latch_error(g.status, err);
        if (t >= 0) g.band[c] = 1;
      }
      __syncthreads();
      continue;
    }
    // ---- sample object k (warp 0)
    if (warp == 0) {
      const Support sup = warp_support(b, t, lane);
      SampleResult r;
      r.placed = false;
      r.band = true;
      r.pose = make_float4(0.f, 0.f, 0.f, 0.f);
      if (sup.ok) {
        r = warp_sample_object(b, sup, g.seed, g.max_attempts, g.retry, c, k, o0, g.poses, pbase, g.status, lane);
      } else if (lane == 0) {
        latch_error(g.status, kDevBadPolygon);
      }
      if (lane == 0) {
        g.poses[pbase + k] = r.pose;
        sh.new_ok = r.placed;
        sh.new_band = r.band;
      }
    }
    if (tid == 0) {
      sh.r2max_key = 0;
      sh.rmax_key = 0;
      sh.hit = 0;
    }
    __syncthreads();
    const bool ok = sh.new_ok;
    float m = kFarSentinel;
    if (ok) {
      // ---- decide: object k against objects 0..k-1 and the world
      stage_objects(b, g.poses, pbase, o0, s0, k + 1, sm, tid, nthr);
      __syncthreads();
      stage_spheres(b, s0, k + 1, S, sm, sh, tid, nthr, lane);
      stage_boxes(b, bx0, nobb, sm, tid, nthr);
      __syncthreads();
      if (tid == 0) build_units(k, k + 1, S, 32 * APL, g.seg_len, sm, sh);
      __syncthreads();
      const float rmax = __int_as_float(sh.rmax_key);
      const float eps = 1e-5f * (__int_as_float(sh.r2max_key) + 0.01f);
      if (nobb > 0) m = box_phase<true>(sm, nobb, sm.off[k], S, m, tid, nthr, my_box);
      m = warp_min(m);
      if (lane == 0 && m < -kBand) *(volatile int*)&sh.hit = 1;
      m = pair_units<APL, true>(sm, sh, k, k + 1, S, g.seg_len, m, rmax, eps, lane, my_pairs);
    }
    m = warp_min(m);
    if (lane == 0) sh.warp_min[warp] = m;
    __syncthreads();
    if (tid == 0) {
      float mm = kFarSentinel;
      for (int w = 0; w < nwarps; ++w) mm = fminf(mm, sh.warp_min[w]);
      const bool pass = ok && !(mm < 0.f);
      const bool bnd = sh.new_band || (ok && fabsf(mm) <= kBand);
      if (bnd) g.band[c] = 1;
      g.tries[c] += 1;
      if (pass) {
        if (k + 1 == nt) g.valid[c] = 1;
        else g.list_next[atomicAdd(g.n_next, 1)] = c;
      } else if (g.retry < g.max_retries) {
        g.list_retry[atomicAdd(g.n_retry, 1)] = c;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    my_pairs += __shfl_xor_sync(0xFFFFFFFFu, my_pairs, o);
    my_box += __shfl_xor_sync(0xFFFFFFFFu, my_box, o);
  }
  if (lane == 0 && g.stats) {
    atomicAdd(&g.stats[0], my_pairs);
    atomicAdd(&g.stats[1], my_box);
  }
}

// First list = the caller's order (or 0..n-1); outputs of the listed
// candidates cleared, their poses set to NaN until placed.
__global__ void gen_init_kernel(sc_scene_batch b, const int32_t* order, int n, int32_t* list0, int* counts,
                                int n_counts, unsigned int* counters, int n_counters, float4* poses, uint8_t* valid,
                                uint8_t* band, int32_t* tries, unsigned long long* stats, int* status) {
  const int stride = gridDim.x * blockDim.x;
  const float nan = __int_as_float(0x7FC00000);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int c = order ? order[i] : i;
    list0[i] = c;
    const int t = template_of(b, c);
    if (t < 0) {  // the step kernel skips it too
      latch_error(status, kDevBadTemplate);
      continue;
    }
    valid[c] = 0;
    band[c] = 0;
    tries[c] = 0;
    const int o0 = b.tmpl_obj_off[t], nt = b.tmpl_obj_off[t + 1] - o0;
    const int64_t pbase = b.tmpl_pose_off[t] + (int64_t)(c - b.cand_tmpl_off[t]) * nt;
    for (int k = 0; k < nt; ++k) poses[pbase + k] = make_float4(nan, nan, nan, nan);
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_counts; i += stride) counts[i] = (i == 0) ? n : 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_counters; i += stride) counters[i] = 0;
  if (blockIdx.x == 0 && threadIdx.x < 2 && stats) stats[threadIdx.x] = 0;
}

template <int APL, int MAXT>
cudaError_t prepare_step_kernel(size_t smem, const sc_collide_config& cfg, int num_sms, int* grid) {
  auto kern = gen_step_kernel<APL, MAXT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, cfg.threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  *grid = num_sms * (cfg.ctas_per_sm < per_sm ? cfg.ctas_per_sm : per_sm);
  return cudaSuccess;
}

template <int APL, int MAXT>
void launch_step(const GenStepArgs& g, int grid, int threads, size_t smem, cudaStream_t s) {
  gen_step_kernel<APL, MAXT><<<grid, threads, smem, s>>>(g);
}

}  // namespace

size_t generate_scratch_bytes(int n_cand, int max_obj, int max_retries) {
  const size_t lists = 4 * (size_t)n_cand * sizeof(int32_t);
  const size_t counts = (size_t)(max_obj + 1) + (size_t)max_obj * (max_retries + 1);
  return lists + 2 * counts * sizeof(int) + 256;
}

cudaError_t enqueue_generate(const sc_scene_batch& b, const GenerateLaunch& a, const sc_collide_config& cfg,
                             int num_sms, cudaStream_t s, const char** why) {
  *why = check_collide_config(cfg);
  if (*why) return cudaErrorInvalidValue;
  const size_t smem = make_layout(b.max_sph, b.max_obj, cfg.a_per_lane).total;
  if (smem > 227 * 1024) { *why = "batch needs more shared memory than one CTA has (max_sph too large)"; return cudaErrorInvalidValue; }
  const int n = a.n_items;
  const int K = b.max_obj, R = a.max_retries;
  // scratch carve-up: 4 lists of n ints, counts[K+1] (list sizes per object),
  // retry counts[K][R+1], work counters[K][R+1]
  char* base = static_cast<char*>(a.scratch);
  int32_t* L[2] = {reinterpret_cast<int32_t*>(base), reinterpret_cast<int32_t*>(base) + n};
  int32_t* Rl[2] = {reinterpret_cast<int32_t*>(base) + 2 * (size_t)n, reinterpret_cast<int32_t*>(base) + 3 * (size_t)n};
  int* counts = reinterpret_cast<int*>(base + 4 * (size_t)n * sizeof(int32_t));
  const int n_counts = (K + 1) + K * (R + 1);
  int* cnt_list = counts;
  int* cnt_retry = counts + (K + 1);
  unsigned int* counters = reinterpret_cast<unsigned int*>(counts + n_counts);
  const int n_counters = K * (R + 1);

  int grid = 0;
  cudaError_t e;
  switch (cfg.a_per_lane) {
    case 1: e = prepare_step_kernel<1, 1024>(smem, cfg, num_sms, &grid); break;
    case 2: e = prepare_step_kernel<2, 1024>(smem, cfg, num_sms, &grid); break;
    default: e = prepare_step_kernel<4, 512>(smem, cfg, num_sms, &grid); break;
  }
  if (e != cudaSuccess) return e;
  {
    int blocks = (n + 255) / 256;
    blocks = blocks < num_sms * 4 ? blocks : num_sms * 4;
    if (blocks < 1) blocks = 1;
    gen_init_kernel<<<blocks, 256, 0, s>>>(b, a.order, n, L[0], counts, n_counts, counters, n_counters,
                                           reinterpret_cast<float4*>(a.poses), a.valid, a.band, a.tries, a.stats,
                                           a.status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  GenStepArgs g;
  g.b = b;
  g.seed = a.seed;
  g.max_attempts = a.max_attempts;
  g.max_retries = R;
  g.seg_len = cfg.seg_len;
  g.poses = reinterpret_cast<float4*>(a.poses);
  g.valid = a.valid;
  g.band = a.band;
  g.tries = a.tries;
  g.stats = a.stats;
  g.status = a.status;
  for (int k = 0; k < K; ++k) {
    g.k = k;
    g.list_next = L[(k + 1) & 1];
    g.n_next = cnt_list + k + 1;
    for (int r = 0; r <= R; ++r) {
      g.retry = r;
      g.list_in = r == 0 ? L[k & 1] : Rl[(r - 1) & 1];
      g.n_in = r == 0 ? cnt_list + k : cnt_retry + k * (R + 1) + (r - 1);
      g.list_retry = Rl[r & 1];
      g.n_retry = cnt_retry + k * (R + 1) + r;
      g.counter = counters + k * (R + 1) + r;
      switch (cfg.a_per_lane) {
        case 1: launch_step<1, 1024>(g, grid, cfg.threads, smem, s); break;
        case 2: launch_step<2, 1024>(g, grid, cfg.threads, smem, s); break;
        default: launch_step<4, 512>(g, grid, cfg.threads, smem, s); break;
      }
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace sc
