// Collision kernel of sc_collide / sc_collide_ex: persistent CTAs take
// candidates from the caller's list through a global atomic counter (list the
// heaviest first) and reduce each candidate's minimum signed distance with
// the device core in collide_core.cuh (exact minimum, or decide-only mode).
#include "collide_core.cuh"
#include "kernels.h"

namespace sc {

namespace {

using namespace core;

struct KArgs {
  sc_scene_batch b;
  CollideLaunch a;
  int seg_len;
};

template <int APL, int MAXT, bool DECIDE>
__global__ void __launch_bounds__(MAXT) collide_kernel(KArgs K) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ CtaShared sh;
  const sc_scene_batch& b = K.b;
  const CollideLaunch& a = K.a;
  const Layout L = make_layout(b.max_sph, b.max_obj, APL);
  const Smem sm = smem_view(smem, L);
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
  unsigned long long my_pairs = 0, my_box = 0;

  for (;;) {
    if (tid == 0) sh.item = (int)atomicAdd(a.counter, 1u);
    __syncthreads();
    const int item = sh.item;
    if (item >= a.n_items) break;
    const int c = a.active ? __ldg(&a.active[item]) : item;
    const int t = template_of(b, c);
    int o0 = 0, nt = 0, s0 = 0, S = 0, nobb = 0, bx0 = 0;
    int64_t pbase = 0;
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
                    : (nobb > kMaxObbPerTemplate) ? kDevTooManyBoxes : kDevOk;
    if (err != kDevOk) {
      if (tid == 0) {
        latch_error(a.status, err);
        a.collide[item] = 0;
        a.min_dist[item] = __int_as_float(0x7FC00000);
        a.band[item] = 1;
      }
      __syncthreads();
      continue;
    }
    const int f = a.first_new;
    stage_objects(b, reinterpret_cast<const float4*>(a.poses), pbase, o0, s0, nt, sm, tid, nthr);
    if (tid == 0) {
      sh.best_key = float_key(kFarSentinel);
      sh.r2max_key = 0;
      sh.rmax_key = 0;
      sh.hit = 0;
    }
    __syncthreads();
    stage_spheres(b, s0, nt, S, sm, sh, tid, nthr, lane);
    stage_boxes(b, bx0, nobb, sm, tid, nthr);
    __syncthreads();
    if (tid == 0) build_units(f, nt, S, 32 * APL, K.seg_len, sm, sh);
    __syncthreads();
    const float rmax = __int_as_float(sh.rmax_key);
    const float eps = 1e-5f * (__int_as_float(sh.r2max_key) + 0.01f);
    float m = kFarSentinel;
    if (f < nt) {
      if (nobb > 0) m = box_phase<DECIDE>(sm, nobb, sm.off[f], S, m, tid, nthr, my_box);
      m = warp_min(m);
      if (!DECIDE && lane == 0 && m < kFarSentinel) atomicMin(&sh.best_key, float_key(m));
      if (DECIDE && lane == 0 && m < -kBand) *(volatile int*)&sh.hit = 1;
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
    }
    __syncthreads();
  }
  // per-CTA work statistics
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    my_pairs += __shfl_xor_sync(0xFFFFFFFFu, my_pairs, o);
    my_box += __shfl_xor_sync(0xFFFFFFFFu, my_box, o);
  }
  if (lane == 0 && a.stats) {
    atomicAdd(&a.stats[0], my_pairs);
    atomicAdd(&a.stats[1], my_box);
  }
}

template <int APL, int MAXT, bool DECIDE>
cudaError_t launch_t(const KArgs& K, const sc_collide_config& cfg, size_t smem, int num_sms, cudaStream_t s) {
  auto kern = collide_kernel<APL, MAXT, DECIDE>;
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
    case 1: return launch_t<1, 1024, DECIDE>(K, cfg, smem, num_sms, s);
    case 2: return launch_t<2, 1024, DECIDE>(K, cfg, smem, num_sms, s);
    default: return launch_t<4, 512, DECIDE>(K, cfg, smem, num_sms, s);
  }
}

}  // namespace

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
  if (a.n_items <= 0) return cudaSuccess;
  KArgs K{b, a, cfg.seg_len};
  return cfg.decide_only ? launch_mode<true>(K, cfg, smem, num_sms, s) : launch_mode<false>(K, cfg, smem, num_sms, s);
}

}  // namespace sc
