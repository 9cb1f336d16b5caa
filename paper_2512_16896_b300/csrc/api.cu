// C ABI of libsceniris_b300: context management, host-side argument
// validation and the entry points declared in include/sceniris.h.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "rmap.h"

struct sc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  // scratch (one allocation): [0] status word, [1] collide work counter, then stats
  void* scratch = nullptr;
  int* d_status = nullptr;
  unsigned int* d_counter = nullptr;
  unsigned long long* d_stats = nullptr;  // [9] (generation); [0..1] and [7] (collision)
  // grow-on-demand scratch of sc_generate (candidate lists and counters)
  void* gen_scratch = nullptr;
  size_t gen_scratch_bytes = 0;
  // side streams and events of sc_generate's rounds (reach stages overlap generation)
  cudaStream_t side[2] = {nullptr, nullptr};
  std::vector<cudaEvent_t> round_events;
  // sc_generate's launch sequence captured as a CUDA graph, and what it was captured for
  cudaStream_t capture_stream = nullptr;
  cudaGraph_t gen_graph = nullptr;
  cudaGraphExec_t gen_exec = nullptr;
  unsigned char gen_key[768] = {};
  size_t gen_key_len = 0;
  unsigned long long seed_host = 0;
  // stage timing (sc_ctx_set_timing)
  int timing = 0;
  std::vector<cudaEvent_t> tev;
  std::vector<int> tcls;
  sc::StageTimer timer;
  int gen_timer_used = 0;  // event pairs the captured graph records
  // cached scan of the last batch generated from: reach extent, most spheres of one object
  const void* scan_key[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  int reach_extent = -1;
  int max_sph_obj = -1;
  int ext_rel = 0;
};

struct sc_mlp {
  int device = 0;
  sc::MlpState* st = nullptr;
  float tau = 0.f;
  int32_t* index = nullptr;  // epoch permutation scratch
  int index_cap = 0;
  float* loss_dev = nullptr;
};

struct sc_rmap {
  int device = 0;
  sc::RmapGrid g{};
  uint2* counts = nullptr;
  int32_t tau = 1;
};

namespace {

thread_local std::string g_err;

sc_status fail(sc_status s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
sc_status fail(sc_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

sc_status cuda_fail(cudaError_t e, const char* where) {
  return fail(SC_ERR_CUDA, "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

sc_status check_batch(const sc_scene_batch* b) {
  if (!b) return fail(SC_ERR_INVALID, "batch is NULL");
  if (b->n_templates < 1 || b->n_objects < 1 || b->n_spheres < 1 || b->n_verts < 3 || b->n_obb < 0 || b->n_cand < 0)
    return fail(SC_ERR_INVALID, "batch sizes out of range (templates %d, objects %d, spheres %d, verts %d, obb %d, cand %d)",
                b->n_templates, b->n_objects, b->n_spheres, b->n_verts, b->n_obb, b->n_cand);
  if (b->max_obj < 1 || b->max_obj > sc::kMaxObj)
    return fail(SC_ERR_INVALID, "max_obj = %d outside 1..%d", b->max_obj, sc::kMaxObj);
  if (b->max_sph < 1 || b->max_sph > sc::kMaxSph)
    return fail(SC_ERR_INVALID, "max_sph = %d outside 1..%d", b->max_sph, sc::kMaxSph);
  const void* req[] = {b->tmpl_obj_off, b->obj_sph_off, b->sph_local, b->obj_half, b->obj_rel, b->obj_rel_param,
                       b->tmpl_poly_off, b->poly_verts, b->tmpl_support_z, b->tmpl_obb_off, b->cand_tmpl_off,
                       b->tmpl_pose_off};
  for (const void* p : req)
    if (!p) return fail(SC_ERR_INVALID, "a required batch array is NULL");
  if (b->n_obb > 0 && !b->obb) return fail(SC_ERR_INVALID, "obb is NULL but n_obb = %d", b->n_obb);
  if (!aligned(b->sph_local, 16) || !aligned(b->obj_half, 16) || !aligned(b->obj_rel_param, 16) ||
      !aligned(b->poly_verts, 8) || (b->obb && !aligned(b->obb, 16)) || (b->tmpl_base && !aligned(b->tmpl_base, 16)))
    return fail(SC_ERR_INVALID, "float4 / float2 batch arrays must be 16 / 8 byte aligned");
  if (!b->obj_anchor_off != !b->obj_anchor) return fail(SC_ERR_INVALID, "obj_anchor_off and obj_anchor go together");
  if ((b->obj_rel_dir && !aligned(b->obj_rel_dir, 4)) || (b->obj_anchor_off && !aligned(b->obj_anchor_off, 4)) ||
      (b->obj_anchor && !aligned(b->obj_anchor, 4)))
    return fail(SC_ERR_INVALID, "relation arrays must be 4-byte aligned");
  if (b->n_parts < 0 || b->max_parts < 0 || b->max_parts > sc::kMaxParts || (b->n_parts > 0) != (b->max_parts > 0))
    return fail(SC_ERR_INVALID, "n_parts = %d, max_parts = %d: both 0, or n_parts > 0 and max_parts in 1..%d",
                b->n_parts, b->max_parts, sc::kMaxParts);
  if (b->n_parts > 0) {
    if (!b->tmpl_part_off || !b->part_param || !b->part_q)
      return fail(SC_ERR_INVALID, "a batch with parts needs tmpl_part_off, part_param and part_q");
    if (!aligned(b->part_param, 16) || !aligned(b->tmpl_part_off, 4) || !aligned(b->part_q, 4) ||
        (b->obb_part && !aligned(b->obb_part, 4)))
      return fail(SC_ERR_INVALID, "part_param must be 16-byte aligned, the other part arrays 4-byte aligned");
  }
  if (b->n_tri < 0) return fail(SC_ERR_INVALID, "n_tri = %d < 0", b->n_tri);
  if (b->n_tri > 0 && (!b->tmpl_tri_off || !b->tri))
    return fail(SC_ERR_INVALID, "a batch with triangles needs tmpl_tri_off and tri");
  if (b->n_tri > 0 && (!aligned(b->tri, 16) || !aligned(b->tmpl_tri_off, 4)))
    return fail(SC_ERR_INVALID, "tri must be 16-byte aligned, tmpl_tri_off 4-byte aligned");
  return SC_OK;
}

sc_status check_ctx(sc_ctx* ctx) {
  if (!ctx) return fail(SC_ERR_INVALID, "ctx is NULL");
  return SC_OK;
}

}  // namespace

namespace sc {
void set_error_message(const std::string& msg) { g_err = msg; }
sc_status validate_batch(const sc_scene_batch* b) { return check_batch(b); }
}  // namespace sc

extern "C" {

int32_t sc_version(void) { return 100; }

const char* sc_last_error(void) { return g_err.c_str(); }

sc_status sc_ctx_create(int device, void* cuda_stream, sc_ctx** out) {
  g_err.clear();
  if (!out) return fail(SC_ERR_INVALID, "out is NULL");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= n) return fail(SC_ERR_INVALID, "device %d outside 0..%d", device, n - 1);
  DeviceGuard g(device);
  sc_ctx* c = new (std::nothrow) sc_ctx;
  if (!c) return fail(SC_ERR_OOM, "host allocation of the context failed");
  c->device = device;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaDeviceGetAttribute"); }
  e = cudaMalloc(&c->scratch, 256);
  if (e != cudaSuccess) { delete c; return fail(SC_ERR_OOM, "scratch allocation failed: %s", cudaGetErrorString(e)); }
  char* base = static_cast<char*>(c->scratch);
  c->d_status = reinterpret_cast<int*>(base);
  c->d_counter = reinterpret_cast<unsigned int*>(base + 16);
  c->d_stats = reinterpret_cast<unsigned long long*>(base + 32);
  e = cudaMemset(c->scratch, 0, 256);
  if (e != cudaSuccess) { cudaFree(c->scratch); delete c; return cuda_fail(e, "cudaMemset"); }
  *out = c;
  return SC_OK;
}

void sc_ctx_destroy(sc_ctx* ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  cudaFree(ctx->scratch);
  if (ctx->gen_exec) cudaGraphExecDestroy(ctx->gen_exec);
  if (ctx->gen_graph) cudaGraphDestroy(ctx->gen_graph);
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  for (cudaStream_t st : ctx->side)
    if (st) cudaStreamDestroy(st);
  for (cudaEvent_t e : ctx->round_events) cudaEventDestroy(e);
  for (cudaEvent_t e : ctx->tev) cudaEventDestroy(e);
  if (ctx->gen_scratch) cudaFree(ctx->gen_scratch);
  delete ctx;
}

sc_status sc_ctx_set_stream(sc_ctx* ctx, void* cuda_stream) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  return SC_OK;
}

int32_t sc_ctx_num_sms(const sc_ctx* ctx) { return ctx ? ctx->num_sms : 0; }

sc_status sc_ctx_synchronize(sc_ctx* ctx) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  int st = 0;
  e = cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  if (st != 0) {
    cudaMemset(ctx->d_status, 0, sizeof(int));
    if (st == sc::kDevTimeout) return fail(SC_ERR_TIMEOUT, "a bounded tensor-core wait gave up (device code 7)");
    return fail(SC_ERR_DEVICE, "a kernel latched device error code %d (1 bad template, 2 too many spheres, "
                "3 too many objects, 4 too many boxes, 5 bad polygon, 6 bad relation, 8 bad part, "
                "9 too many triangles)", st);
  }
  return SC_OK;
}

sc_status sc_sample_poses(sc_ctx* ctx, const sc_scene_batch* batch, const sc_sample_params* params,
                          const int32_t* active, int32_t n_active, float* poses, uint8_t* sample_ok, uint8_t* band) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  if (sc_status s = check_batch(batch)) return s;
  if (!params) return fail(SC_ERR_INVALID, "params is NULL");
  if (active && n_active < 0) return fail(SC_ERR_INVALID, "n_active < 0");
  if ((active ? n_active : batch->n_cand) == 0) return SC_OK;  // nothing to sample
  if (!poses || !sample_ok || !band) return fail(SC_ERR_INVALID, "an output pointer is NULL");
  if (!aligned(poses, 16)) return fail(SC_ERR_INVALID, "poses must be 16-byte aligned");
  if (params->max_attempts < 1 || params->max_attempts > 1024)
    return fail(SC_ERR_INVALID, "max_attempts = %d outside 1..1024", params->max_attempts);
  if (params->retry < 0 || params->first_obj < 0 || params->n_obj < 0)
    return fail(SC_ERR_INVALID, "retry, first_obj and n_obj must be >= 0");
  if (active && n_active < 0) return fail(SC_ERR_INVALID, "n_active < 0");
  const int n = active ? n_active : batch->n_cand;
  DeviceGuard g(ctx->device);
  cudaError_t e = sc::launch_sample(*batch, *params, active, n, poses, sample_ok, band, ctx->d_status, ctx->num_sms,
                                    ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "sample_kernel launch");
  return SC_OK;
}

sc_status sc_sample_parts(sc_ctx* ctx, const sc_scene_batch* batch, uint64_t seed, const int32_t* active,
                          int32_t n_active, float* part_q) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  if (sc_status s = check_batch(batch)) return s;
  if (batch->n_parts == 0) return fail(SC_ERR_INVALID, "the batch has no articulated parts");
  if (!part_q || !aligned(part_q, 4)) return fail(SC_ERR_INVALID, "part_q is NULL or not 4-byte aligned");
  if (active && n_active < 0) return fail(SC_ERR_INVALID, "n_active < 0");
  const int n = active ? n_active : batch->n_cand;
  if (n == 0) return SC_OK;
  DeviceGuard g(ctx->device);
  cudaError_t e = sc::launch_sample_parts(*batch, seed, active, n, part_q, ctx->d_status, ctx->num_sms, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "sample_parts_kernel launch");
  return SC_OK;
}

// The generation step culls spheres before its pair sweep, so its register
// blocks are small; one A sphere per lane also keeps its instruction
// footprint smallest (the step is bound by instruction fetch, not the FMA pipe).
static const sc_collide_config kDefaultGenerate = {256, 1, 256, 4, 1, 0};

sc_status sc_collide_ex(sc_ctx* ctx, const sc_scene_batch* batch, const float* poses, const int32_t* active,
                        int32_t n_active, int32_t first_new_obj, const sc_collide_config* config, uint8_t* collide,
                        float* min_dist, uint8_t* band) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  if (sc_status s = check_batch(batch)) return s;
  if (active && n_active < 0) return fail(SC_ERR_INVALID, "n_active < 0");
  if ((active ? n_active : batch->n_cand) == 0) return SC_OK;  // nothing to check
  if (!poses || !collide || !min_dist || !band) return fail(SC_ERR_INVALID, "an input or output pointer is NULL");
  if (!aligned(poses, 16)) return fail(SC_ERR_INVALID, "poses must be 16-byte aligned");
  if (first_new_obj < 0) return fail(SC_ERR_INVALID, "first_new_obj = %d < 0", first_new_obj);
  if (active && n_active < 0) return fail(SC_ERR_INVALID, "n_active < 0");
  sc_collide_config cfg = sc::default_collide_config(*batch);
  if (config) {  // zero fields keep the default
    if (config->threads) cfg.threads = config->threads;
    if (config->a_per_lane) cfg.a_per_lane = config->a_per_lane;
    if (config->seg_len) cfg.seg_len = config->seg_len;
    if (config->ctas_per_sm) cfg.ctas_per_sm = config->ctas_per_sm;
    cfg.decide_only = config->decide_only;
    cfg.stage_bulk = config->stage_bulk;
  }
  sc::CollideLaunch a;
  a.poses = poses;
  a.active = active;
  a.n_items = active ? n_active : batch->n_cand;
  a.first_new = first_new_obj;
  a.collide = collide;
  a.min_dist = min_dist;
  a.band = band;
  a.counter = ctx->d_counter;
  a.stats = ctx->d_stats;
  a.status = ctx->d_status;
  DeviceGuard g(ctx->device);
  const char* why = nullptr;
  cudaError_t e = sc::launch_collide(*batch, a, cfg, ctx->num_sms, ctx->stream, &why);
  if (why) return fail(SC_ERR_INVALID, "collide config: %s", why);
  if (e != cudaSuccess) return cuda_fail(e, "collide_kernel launch");
  return SC_OK;
}

sc_status sc_collide(sc_ctx* ctx, const sc_scene_batch* batch, const float* poses, const int32_t* active,
                     int32_t n_active, int32_t first_new_obj, uint8_t* collide, float* min_dist, uint8_t* band) {
  return sc_collide_ex(ctx, batch, poses, active, n_active, first_new_obj, nullptr, collide, min_dist, band);
}

sc_status sc_generate(sc_ctx* ctx, const sc_scene_batch* batch, const sc_gen_params* params, const int32_t* order,
                      int32_t n_order, const sc_collide_config* config, const sc_gen_reach* reach, float* poses,
                      uint8_t* valid, uint8_t* band, int32_t* tries, float* q_reach) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  if (sc_status s = check_batch(batch)) return s;
  if (!params) return fail(SC_ERR_INVALID, "params is NULL");
  if (params->max_attempts < 1 || params->max_attempts > 1024)
    return fail(SC_ERR_INVALID, "max_attempts = %d outside 1..1024", params->max_attempts);
  if (params->max_retries < 0 || params->max_retries > 1000)
    return fail(SC_ERR_INVALID, "max_retries = %d outside 0..1000", params->max_retries);
  if (order && n_order < 0) return fail(SC_ERR_INVALID, "n_order < 0");
  const int n = order ? n_order : batch->n_cand;
  if (n == 0) return SC_OK;
  if (!poses || !valid || !band || !tries) return fail(SC_ERR_INVALID, "an output pointer is NULL");
  if (!aligned(poses, 16)) return fail(SC_ERR_INVALID, "poses must be 16-byte aligned");
  const bool want_reach = reach && reach->arm;
  if (want_reach) {
    if (!reach->ik) return fail(SC_ERR_INVALID, "reach->ik is NULL");
    if (reach->gate && reach->map) return fail(SC_ERR_INVALID, "reach->gate and reach->map are both set");
    if (!batch->tmpl_base) return fail(SC_ERR_INVALID, "a reachability stage needs batch->tmpl_base");
    const sc_ik_params& P = *reach->ik;
    if (P.seeds < 1 || P.seeds > 32 || P.iters < 0 || !(P.tol_pos > 0.f) || !(P.tol_rot > 0.f) ||
        !(P.tol_rot < 1.5707963f) || !(P.lambda >= 0.f))
      return fail(SC_ERR_INVALID, "bad IK parameters (seeds 1..32, iters >= 0, tolerances > 0, tol_rot < pi/2)");
    if (params->max_retries > 65535) return fail(SC_ERR_INVALID, "max_retries > 65535 with a reachability stage");
    if (batch->max_obj > 65535) return fail(SC_ERR_INVALID, "max_obj > 65535 with a reachability stage");
  }
  sc_collide_config cfg = kDefaultGenerate;
  if (config) {
    if (config->threads) cfg.threads = config->threads;
    if (config->a_per_lane) cfg.a_per_lane = config->a_per_lane;
    if (config->seg_len) cfg.seg_len = config->seg_len;
    if (config->ctas_per_sm) cfg.ctas_per_sm = config->ctas_per_sm;
  }
  DeviceGuard g(ctx->device);
  const size_t need = sc::generate_scratch_bytes(*batch, n, params->max_retries);
  if (need > ctx->gen_scratch_bytes) {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (ctx->gen_scratch) cudaFree(ctx->gen_scratch);
    ctx->gen_scratch = nullptr;
    ctx->gen_scratch_bytes = 0;
    e = cudaMalloc(&ctx->gen_scratch, need);
    if (e != cudaSuccess) return fail(SC_ERR_OOM, "generation scratch (%zu bytes): %s", need, cudaGetErrorString(e));
    ctx->gen_scratch_bytes = need;
  }
  sc::GenerateLaunch a;
  a.order = order;
  a.n_items = n;
  // the seed lives in device scratch (an aligned slot after the lists), written before each run
  unsigned long long* seed_dev = reinterpret_cast<unsigned long long*>(
      static_cast<char*>(ctx->gen_scratch) + sc::generate_seed_offset(*batch, n, params->max_retries));
  a.seed_dev = seed_dev;
  a.max_attempts = params->max_attempts;
  a.max_retries = params->max_retries;
  a.poses = poses;
  a.valid = valid;
  a.band = band;
  a.tries = tries;
  a.scratch = ctx->gen_scratch;
  a.stats = ctx->d_stats;
  a.status = ctx->d_status;
  a.arm = want_reach ? reach->arm : nullptr;
  a.ik = want_reach ? reach->ik : nullptr;
  a.gate = (want_reach && reach->gate) ? reach->gate->st : nullptr;
  a.tau = (want_reach && reach->gate) ? reach->gate->tau : 0.f;
  a.map_counts = (want_reach && reach->map) ? reach->map->counts : nullptr;
  a.map_grid = (want_reach && reach->map) ? reach->map->g : sc::RmapGrid{};
  a.map_tau = (want_reach && reach->map) ? reach->map->tau : 0;
  a.q_reach = want_reach ? q_reach : nullptr;
  a.reach_objects = 0;
  a.max_sph_obj = 0;
  a.ext_rel = 0;
  a.timer = nullptr;
  a.side[0] = a.side[1] = nullptr;
  a.events = nullptr;
  a.n_events = 0;
  if (ctx->timing) {
    ctx->timer.used = 0;
    a.timer = &ctx->timer;
  }
  {
    const void* key[5] = {batch->tmpl_obj_off, batch->obj_rel, batch->obj_sph_off,
                          reinterpret_cast<const void*>((intptr_t)batch->n_templates),
                          reinterpret_cast<const void*>((intptr_t)batch->n_objects)};
    if (ctx->reach_extent < 0 || std::memcmp(key, ctx->scan_key, sizeof(key))) {
      int out[3] = {0, 0, 0};
      int* scan_scratch = reinterpret_cast<int*>(static_cast<char*>(ctx->scratch) + 96);  // past the stats
      cudaError_t e = sc::batch_scan(*batch, scan_scratch, out, ctx->stream);
      if (e != cudaSuccess) return cuda_fail(e, "batch scan");
      std::memcpy(ctx->scan_key, key, sizeof(key));
      ctx->reach_extent = out[0];
      ctx->max_sph_obj = out[1];
      ctx->ext_rel = out[2];
    }
    a.reach_objects = want_reach ? ctx->reach_extent : 0;
    a.max_sph_obj = ctx->max_sph_obj;
    // instances: 2 with parts (boxes moved, INSIDE supports) or triangles,
    // 1 with the full relation set, 0 with free / on-top / next-to only
    a.ext_rel = (batch->n_parts > 0 || batch->n_tri > 0) ? 2 : ctx->ext_rel ? 1 : 0;
  }
  if (a.reach_objects > 0) {  // side streams and events of the rounds
    const size_t need_ev = 2 * (size_t)sc::generate_rounds(a.reach_objects, params->max_retries) + 1;
    for (int j = 0; j < 2; ++j) {
      if (!ctx->side[j]) {
        cudaError_t e = cudaStreamCreateWithFlags(&ctx->side[j], cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreateWithFlags");
      }
    }
    while (ctx->round_events.size() < need_ev) {
      cudaEvent_t ev = nullptr;
      cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreateWithFlags");
      ctx->round_events.push_back(ev);
    }
    a.side[0] = ctx->side[0];
    a.side[1] = ctx->side[1];
    a.events = ctx->round_events.data();
    a.n_events = (int)ctx->round_events.size();
  }
  ctx->seed_host = params->seed;
  cudaError_t e = cudaMemcpyAsync(seed_dev, &ctx->seed_host, 8, cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "seed upload");
  const char* why = nullptr;
  if (!params->use_graph) {
    ctx->timer.flags = cudaEventRecordDefault;
    e = sc::enqueue_generate(*batch, a, cfg, ctx->num_sms, ctx->stream, &why);
    if (why) return fail(SC_ERR_INVALID, "generate config: %s", why);
    if (e != cudaSuccess) return cuda_fail(e, "generate launch");
    return SC_OK;
  }
  // graph replay: capture once per (batch, list, outputs, tries, launch shape)
  struct Key {
    sc_scene_batch batch;
    const int32_t* order;
    int32_t n, max_attempts, max_retries;
    sc_collide_config cfg;
    float* poses;
    uint8_t* valid;
    uint8_t* band;
    int32_t* tries;
    void* scratch;
    sc_arm arm;
    sc_ik_params ik;
    const void* gate;
    float tau;
    const void* map;
    int32_t map_tau;
    float* q_reach;
    int reach_objects;
    int max_sph_obj;
    int timing;
  } key;
  static_assert(sizeof(Key) <= sizeof(ctx->gen_key), "graph key too large");
  std::memset(&key, 0, sizeof(key));
  key.batch = *batch;
  key.order = order;
  key.n = n;
  key.max_attempts = params->max_attempts;
  key.max_retries = params->max_retries;
  key.cfg = cfg;
  key.poses = poses;
  key.valid = valid;
  key.band = band;
  key.tries = tries;
  key.scratch = ctx->gen_scratch;
  if (want_reach) {
    key.arm = *reach->arm;
    key.ik = *reach->ik;
  }
  key.gate = a.gate;
  key.tau = a.tau;
  key.map = a.map_counts;
  key.map_tau = a.map_tau;
  key.q_reach = a.q_reach;
  key.reach_objects = a.reach_objects;
  key.max_sph_obj = a.max_sph_obj;
  key.timing = ctx->timing;
  const bool hit = ctx->gen_exec && ctx->gen_key_len == sizeof(key) && !std::memcmp(ctx->gen_key, &key, sizeof(key));
  if (!hit) {
    if (ctx->gen_exec) { cudaGraphExecDestroy(ctx->gen_exec); ctx->gen_exec = nullptr; }
    if (ctx->gen_graph) { cudaGraphDestroy(ctx->gen_graph); ctx->gen_graph = nullptr; }
    ctx->gen_key_len = 0;
    if (!ctx->capture_stream) {
      e = cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreateWithFlags");
    }
    e = cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    ctx->timer.flags = cudaEventRecordExternal;
    cudaError_t e_enq = sc::enqueue_generate(*batch, a, cfg, ctx->num_sms, ctx->capture_stream, &why);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(ctx->capture_stream, &graph);
    if (why) { if (graph) cudaGraphDestroy(graph); return fail(SC_ERR_INVALID, "generate config: %s", why); }
    if (e_enq != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cuda_fail(e_enq, "generate capture"); }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&ctx->gen_exec, graph, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return cuda_fail(e, "cudaGraphInstantiate"); }
    ctx->gen_graph = graph;
    std::memcpy(ctx->gen_key, &key, sizeof(key));
    ctx->gen_key_len = sizeof(key);
    ctx->gen_timer_used = ctx->timer.used;
  }
  if (ctx->timing) ctx->timer.used = ctx->gen_timer_used;  // the replay records the captured events again
  e = cudaGraphLaunch(ctx->gen_exec, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  return SC_OK;
}

sc_status sc_ik_reach(sc_ctx* ctx, const sc_arm* arm, const sc_ik_params* params, const float* targets,
                      const uint32_t* target_ids, int32_t n, uint8_t* reachable, float* q_out, float* err,
                      uint8_t* band) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  if (!arm || !params) return fail(SC_ERR_INVALID, "arm or params is NULL");
  if (n < 0) return fail(SC_ERR_INVALID, "n < 0");
  if (n == 0) return SC_OK;
  if (!targets || !reachable || !q_out || !err) return fail(SC_ERR_INVALID, "an input or output pointer is NULL");
  if (params->seeds < 1 || params->seeds > 32) return fail(SC_ERR_INVALID, "seeds = %d outside 1..32", params->seeds);
  if (params->iters < 0) return fail(SC_ERR_INVALID, "iters < 0");
  if (!(params->tol_pos > 0.f) || !(params->tol_rot > 0.f) || !(params->tol_rot < 1.5707963f) || !(params->lambda >= 0.f))
    return fail(SC_ERR_INVALID, "tolerances must be positive, tol_rot < pi/2, lambda >= 0");
  DeviceGuard g(ctx->device);
  cudaError_t e = sc::launch_ik(*arm, *params, targets, target_ids, n, reachable, q_out, err, nullptr, band,
                                ctx->d_counter, ctx->d_stats + 4, ctx->num_sms, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "ik_kernel launch");
  return SC_OK;
}

sc_status sc_ik_dls_step(sc_ctx* ctx, const sc_arm* arm, float lambda, const float* targets, const float* q_in,
                         int32_t n, float* q_out, float* tool) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  if (!arm) return fail(SC_ERR_INVALID, "arm is NULL");
  if (n < 0) return fail(SC_ERR_INVALID, "n < 0");
  if (n == 0) return SC_OK;
  if (!targets || !q_in || !q_out) return fail(SC_ERR_INVALID, "an input or output pointer is NULL");
  DeviceGuard g(ctx->device);
  cudaError_t e = sc::launch_ik_step(*arm, lambda, targets, q_in, n, q_out, tool, ctx->num_sms, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "ik_step_kernel launch");
  return SC_OK;
}

// ------------------------------------------------------------- surrogate


int32_t sc_mlp_param_count(void) { return sc::mlp_param_count(); }

sc_status sc_mlp_create(sc_ctx* ctx, uint64_t seed, sc_mlp** out) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  if (!out) return fail(SC_ERR_INVALID, "out is NULL");
  *out = nullptr;
  DeviceGuard g(ctx->device);
  sc_mlp* m = new (std::nothrow) sc_mlp;
  if (!m) return fail(SC_ERR_OOM, "host allocation failed");
  m->device = ctx->device;
  cudaError_t e = sc::mlp_alloc(&m->st);
  if (e == cudaSuccess) e = cudaMalloc(&m->loss_dev, 256);
  if (e != cudaSuccess) { sc_mlp_destroy(m); return fail(SC_ERR_OOM, "surrogate allocation: %s", cudaGetErrorString(e)); }
  e = sc::mlp_init(m->st, seed, ctx->stream);
  if (e != cudaSuccess) { sc_mlp_destroy(m); return cuda_fail(e, "surrogate init"); }
  *out = m;
  return SC_OK;
}

void sc_mlp_destroy(sc_mlp* m) {
  if (!m) return;
  DeviceGuard g(m->device);
  cudaDeviceSynchronize();
  sc::mlp_free(m->st);
  if (m->index) cudaFree(m->index);
  if (m->loss_dev) cudaFree(m->loss_dev);
  delete m;
}

sc_status sc_mlp_get(sc_ctx* ctx, const sc_mlp* m, float* params, float* mu, float* sigma, float* tau) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  if (!m) return fail(SC_ERR_INVALID, "mlp is NULL");
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  const int n = sc::mlp_param_count();
  if (!e && params) e = cudaMemcpy(params, sc::mlp_params_ptr(m->st), n * 4, cudaMemcpyDeviceToHost);
  float inv[9];
  if (!e && mu) e = cudaMemcpy(mu, sc::mlp_mu_ptr(m->st), 36, cudaMemcpyDeviceToHost);
  if (!e && sigma) {
    e = cudaMemcpy(inv, sc::mlp_inv_sigma_ptr(m->st), 36, cudaMemcpyDeviceToHost);
    for (int i = 0; i < 9; ++i) sigma[i] = 1.f / inv[i];
  }
  if (e) return cuda_fail(e, "surrogate read-back");
  if (tau) *tau = m->tau;
  return SC_OK;
}

sc_status sc_mlp_set(sc_ctx* ctx, sc_mlp* m, const float* params, const float* mu, const float* sigma, float tau) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  if (!m) return fail(SC_ERR_INVALID, "mlp is NULL");
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  const int n = sc::mlp_param_count();
  if (!e && params) e = cudaMemcpy(sc::mlp_params_ptr(m->st), params, n * 4, cudaMemcpyHostToDevice);
  if (!e && mu) e = cudaMemcpy(sc::mlp_mu_ptr(m->st), mu, 36, cudaMemcpyHostToDevice);
  if (!e && sigma) {
    float inv[9];
    for (int i = 0; i < 9; ++i) {
      if (!(sigma[i] > 0.f)) return fail(SC_ERR_INVALID, "sigma[%d] must be > 0", i);
      inv[i] = 1.f / sigma[i];
    }
    e = cudaMemcpy(sc::mlp_inv_sigma_ptr(m->st), inv, 36, cudaMemcpyHostToDevice);
  }
  if (!e) e = sc::mlp_refresh_copies(m->st, ctx->stream);
  if (e) return cuda_fail(e, "surrogate upload");
  m->tau = tau;
  return SC_OK;
}

sc_status sc_surrogate_infer(sc_ctx* ctx, const sc_mlp* m, const float* targets, int32_t n, float* logits) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  if (!m) return fail(SC_ERR_INVALID, "mlp is NULL");
  if (n < 0) return fail(SC_ERR_INVALID, "n < 0");
  if (n == 0) return SC_OK;
  if (!targets || !logits) return fail(SC_ERR_INVALID, "targets or logits is NULL");
  DeviceGuard g(ctx->device);
  cudaError_t e = sc::mlp_infer(m->st, targets, n, logits, ctx->d_status, ctx->num_sms, ctx->stream);
  if (e) return cuda_fail(e, "surrogate inference");
  return SC_OK;
}

sc_status sc_surrogate_grads(sc_ctx* ctx, sc_mlp* m, const float* targets, const uint8_t* labels, int32_t n,
                             float* grads, float* loss) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  if (!m) return fail(SC_ERR_INVALID, "mlp is NULL");
  if (n < 1 || n > (1 << 20)) return fail(SC_ERR_INVALID, "n = %d outside 1..2^20", n);
  if (!targets || !labels) return fail(SC_ERR_INVALID, "targets or labels is NULL");
  DeviceGuard g(ctx->device);
  cudaError_t e = sc::mlp_reserve(m->st, n);
  if (e) return fail(SC_ERR_OOM, "surrogate training buffers: %s", cudaGetErrorString(e));
  e = sc::mlp_gradients(m->st, targets, labels, nullptr, n, m->loss_dev, ctx->d_status, ctx->num_sms, ctx->stream);
  if (!e && grads)
    e = cudaMemcpyAsync(grads, sc::mlp_grads_ptr(m->st), sc::mlp_param_count() * 4, cudaMemcpyDeviceToDevice,
                        ctx->stream);
  if (!e && loss) {
    e = cudaMemcpyAsync(loss, m->loss_dev, 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (!e) e = cudaStreamSynchronize(ctx->stream);
  }
  if (e) return cuda_fail(e, "surrogate gradients");
  return SC_OK;
}

static sc_status check_train(const sc_train_params* p) {
  if (!p) return fail(SC_ERR_INVALID, "train params is NULL");
  if (p->epochs < 0 || p->batch < 16 || p->batch > 65536)
    return fail(SC_ERR_INVALID, "epochs >= 0 and batch in 16..65536 required");
  if (!(p->lr > 0.f) || !(p->beta1 >= 0.f && p->beta1 < 1.f) || !(p->beta2 >= 0.f && p->beta2 < 1.f) || !(p->eps > 0.f))
    return fail(SC_ERR_INVALID, "lr > 0, betas in [0, 1), eps > 0 required");
  return SC_OK;
}

sc_status sc_mlp_train_step(sc_ctx* ctx, sc_mlp* m, const float* targets, const uint8_t* labels, int32_t n,
                            const sc_train_params* p, float* loss) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  if (!m) return fail(SC_ERR_INVALID, "mlp is NULL");
  if (sc_status s = check_train(p)) return s;
  if (n < 1 || n > (1 << 20)) return fail(SC_ERR_INVALID, "n = %d outside 1..2^20", n);
  if (!targets || !labels) return fail(SC_ERR_INVALID, "targets or labels is NULL");
  DeviceGuard g(ctx->device);
  cudaError_t e = sc::mlp_reserve(m->st, n);
  if (e) return fail(SC_ERR_OOM, "surrogate training buffers: %s", cudaGetErrorString(e));
  e = sc::mlp_train_step(m->st, targets, labels, nullptr, n, m->loss_dev, ctx->d_status, ctx->num_sms, p->lr,
                         p->beta1, p->beta2, p->eps, ctx->stream);
  if (!e && loss) {
    e = cudaMemcpyAsync(loss, m->loss_dev, 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (!e) e = cudaStreamSynchronize(ctx->stream);
  }
  if (e) return cuda_fail(e, "training step");
  return SC_OK;
}

sc_status sc_mlp_adam_step(sc_ctx* ctx, sc_mlp* m, const float* grads, const sc_train_params* p) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  if (!m) return fail(SC_ERR_INVALID, "mlp is NULL");
  if (sc_status s = check_train(p)) return s;
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaSuccess;
  if (grads)
    e = cudaMemcpyAsync(sc::mlp_grads_ptr(m->st), grads, sc::mlp_param_count() * 4, cudaMemcpyDeviceToDevice,
                        ctx->stream);
  if (!e) e = sc::mlp_adam(m->st, p->lr, p->beta1, p->beta2, p->eps, ctx->stream);
  if (e) return cuda_fail(e, "adam step");
  return SC_OK;
}

sc_status sc_surrogate_train(sc_ctx* ctx, sc_mlp* m, const float* targets, const uint8_t* labels, int32_t n,
                             const sc_train_params* p, float* loss_per_epoch) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  if (!m) return fail(SC_ERR_INVALID, "mlp is NULL");
  if (sc_status s = check_train(p)) return s;
  if (n < p->batch) return fail(SC_ERR_INVALID, "n = %d smaller than one batch (%d)", n, p->batch);
  if (!targets || !labels) return fail(SC_ERR_INVALID, "targets or labels is NULL");
  DeviceGuard g(ctx->device);
  cudaError_t e = sc::mlp_reserve(m->st, p->batch);
  if (!e && m->index_cap < n) {
    if (m->index) cudaFree(m->index);
    m->index = nullptr;
    m->index_cap = 0;
    e = cudaMalloc(&m->index, (size_t)n * 4);
    if (!e) m->index_cap = n;
  }
  if (e) return fail(SC_ERR_OOM, "training buffers: %s", cudaGetErrorString(e));
  if (sc::mlp_step(m->st) == 0) {  // a fresh network takes its input standardisation from the training set
    e = sc::mlp_set_norm_from(m->st, targets, n, ctx->stream);
    if (e) return cuda_fail(e, "feature standardisation");
  }
  const int nb = n / p->batch;  // whole batches per epoch (the remainder changes with the shuffle)
  for (int ep = 0; ep < p->epochs; ++ep) {
    e = sc::mlp_epoch_index(n, p->seed, (int)(sc::mlp_step(m->st) / nb), m->index, ctx->stream);
    if (e) return cuda_fail(e, "epoch shuffle");
    float loss_acc = 0.f;
    for (int bi = 0; bi < nb; ++bi) {
      e = sc::mlp_train_step(m->st, targets, labels, m->index + (size_t)bi * p->batch, p->batch, m->loss_dev,
                             ctx->d_status, ctx->num_sms, p->lr, p->beta1, p->beta2, p->eps, ctx->stream);
      if (e) return cuda_fail(e, "training step");
      if (loss_per_epoch && bi == nb - 1) {  // the epoch's last batch reports its mean BCE
        float l = 0.f;
        e = cudaMemcpyAsync(&l, m->loss_dev, 4, cudaMemcpyDeviceToHost, ctx->stream);
        if (!e) e = cudaStreamSynchronize(ctx->stream);
        if (e) return cuda_fail(e, "loss read-back");
        loss_acc = l;
      }
    }
    if (loss_per_epoch) loss_per_epoch[ep] = loss_acc;
  }
  return SC_OK;
}

sc_status sc_surrogate_tune_threshold(sc_ctx* ctx, sc_mlp* m, const float* targets, const uint8_t* labels, int32_t n,
                                      float min_recall, float* tau_out, float* recall_out, float* pass_rate_out) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  if (!m) return fail(SC_ERR_INVALID, "mlp is NULL");
  if (n < 1 || !targets || !labels) return fail(SC_ERR_INVALID, "need n >= 1 targets and labels");
  if (!(min_recall > 0.f && min_recall <= 1.f)) return fail(SC_ERR_INVALID, "min_recall must be in (0, 1]");
  DeviceGuard g(ctx->device);
  float* logits = nullptr;
  cudaError_t e = cudaMalloc(&logits, (size_t)n * 4);
  if (e) return fail(SC_ERR_OOM, "logit buffer: %s", cudaGetErrorString(e));
  e = sc::mlp_infer(m->st, targets, n, logits, ctx->d_status, ctx->num_sms, ctx->stream);
  std::vector<float> z(n);
  std::vector<uint8_t> y(n);
  if (!e) e = cudaMemcpyAsync(z.data(), logits, (size_t)n * 4, cudaMemcpyDeviceToHost, ctx->stream);
  if (!e) e = cudaMemcpyAsync(y.data(), labels, (size_t)n, cudaMemcpyDeviceToHost, ctx->stream);
  if (!e) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(logits);
  if (e) return cuda_fail(e, "threshold tuning");
  // largest tau with recall >= min_recall: keep the top ceil(min_recall * P) positive logits
  std::vector<float> pos;
  for (int i = 0; i < n; ++i)
    if (y[i]) pos.push_back(z[i]);
  if (pos.empty()) return fail(SC_ERR_INVALID, "no positive labels");
  std::sort(pos.begin(), pos.end(), std::greater<float>());
  const size_t need = (size_t)std::ceil((double)min_recall * pos.size());
  const float tau = pos[std::min(pos.size(), std::max<size_t>(need, 1)) - 1];
  size_t tp = 0, pass = 0;
  for (int i = 0; i < n; ++i)
    if (z[i] >= tau) { ++pass; tp += y[i] ? 1 : 0; }
  m->tau = tau;
  if (tau_out) *tau_out = tau;
  if (recall_out) *recall_out = (float)tp / pos.size();
  if (pass_rate_out) *pass_rate_out = (float)pass / n;
  return SC_OK;
}

// ---- 4D reachability map

sc_status sc_rmap_create(sc_ctx* ctx, const sc_rmap_params* p, sc_rmap** out) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  if (!p || !out) return fail(SC_ERR_INVALID, "params or out is NULL");
  *out = nullptr;
  if (p->nz < 1 || p->nc < 1 || p->nxy < 1) return fail(SC_ERR_INVALID, "bin counts must be >= 1");
  const double cells = (double)p->nz * p->nc * (double)p->nxy * p->nxy;
  if (cells > (double)(1 << 27)) return fail(SC_ERR_INVALID, "nz * nc * nxy^2 = %.0f cells > 2^27", cells);
  if (!(std::isfinite(p->z_lo) && std::isfinite(p->z_hi) && p->z_hi > p->z_lo))
    return fail(SC_ERR_INVALID, "need finite z_lo < z_hi");
  if (!(std::isfinite(p->r_max) && p->r_max > 0.f)) return fail(SC_ERR_INVALID, "need a finite r_max > 0");
  sc::RmapGrid g;
  g.nz = p->nz;
  g.nc = p->nc;
  g.nxy = p->nxy;
  g.z_lo = p->z_lo;
  const float span = p->z_hi - p->z_lo;  // FP32 operations, as the key definition states
  g.sz = (float)p->nz / span;
  g.sc = (float)p->nc / 2.f;
  g.r_max = p->r_max;
  g.sxy = (float)p->nxy / (2.f * p->r_max);
  g.cells = (size_t)cells;
  if (!(std::isfinite(g.sz) && std::isfinite(g.sxy))) return fail(SC_ERR_INVALID, "grid scale is not finite");
  DeviceGuard gd(ctx->device);
  sc_rmap* m = new (std::nothrow) sc_rmap;
  if (!m) return fail(SC_ERR_OOM, "host allocation failed");
  m->device = ctx->device;
  m->g = g;
  cudaError_t e = cudaMalloc(&m->counts, g.cells * sizeof(uint2));
  if (e) { delete m; return fail(SC_ERR_OOM, "map counts (%zu cells): %s", g.cells, cudaGetErrorString(e)); }
  e = cudaMemsetAsync(m->counts, 0, g.cells * sizeof(uint2), ctx->stream);
  if (e) { sc_rmap_destroy(m); return cuda_fail(e, "map clear"); }
  *out = m;
  return SC_OK;
}

void sc_rmap_destroy(sc_rmap* m) {
  if (!m) return;
  DeviceGuard g(m->device);
  cudaDeviceSynchronize();
  if (m->counts) cudaFree(m->counts);
  delete m;
}

int64_t sc_rmap_cells(const sc_rmap* m) { return m ? (int64_t)m->g.cells : 0; }

sc_status sc_rmap_build(sc_ctx* ctx, sc_rmap* m, const float* targets, const uint8_t* labels, int32_t n) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  if (!m) return fail(SC_ERR_INVALID, "map is NULL");
  if (n < 0) return fail(SC_ERR_INVALID, "n < 0");
  if (n == 0) return SC_OK;
  if (!targets || !labels) return fail(SC_ERR_INVALID, "targets or labels is NULL");
  DeviceGuard g(ctx->device);
  cudaError_t e = sc::rmap_build(m->g, m->counts, targets, labels, n, ctx->num_sms, ctx->stream);
  if (e) return cuda_fail(e, "rmap_build_kernel launch");
  return SC_OK;
}

sc_status sc_rmap_query(sc_ctx* ctx, const sc_rmap* m, const float* targets, int32_t n, uint16_t* score) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  if (!m) return fail(SC_ERR_INVALID, "map is NULL");
  if (n < 0) return fail(SC_ERR_INVALID, "n < 0");
  if (n == 0) return SC_OK;
  if (!targets || !score) return fail(SC_ERR_INVALID, "targets or score is NULL");
  DeviceGuard g(ctx->device);
  cudaError_t e = sc::rmap_query(m->g, m->counts, targets, n, score, ctx->num_sms, ctx->stream);
  if (e) return cuda_fail(e, "rmap_query_kernel launch");
  return SC_OK;
}

sc_status sc_rmap_tune_threshold(sc_ctx* ctx, sc_rmap* m, const float* targets, const uint8_t* labels, int32_t n,
                                 float min_recall, int32_t* tau_out, float* recall_out, float* pass_rate_out) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  if (!m) return fail(SC_ERR_INVALID, "map is NULL");
  if (n < 1 || !targets || !labels) return fail(SC_ERR_INVALID, "need n >= 1 targets and labels");
  if (!(min_recall > 0.f && min_recall <= 1.f)) return fail(SC_ERR_INVALID, "min_recall must be in (0, 1]");
  DeviceGuard g(ctx->device);
  uint16_t* dscore = nullptr;
  cudaError_t e = cudaMalloc(&dscore, (size_t)n * 2);
  if (e) return fail(SC_ERR_OOM, "score buffer: %s", cudaGetErrorString(e));
  e = sc::rmap_query(m->g, m->counts, targets, n, dscore, ctx->num_sms, ctx->stream);
  std::vector<uint16_t> z(n);
  std::vector<uint8_t> y(n);
  if (!e) e = cudaMemcpyAsync(z.data(), dscore, (size_t)n * 2, cudaMemcpyDeviceToHost, ctx->stream);
  if (!e) e = cudaMemcpyAsync(y.data(), labels, (size_t)n, cudaMemcpyDeviceToHost, ctx->stream);
  if (!e) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(dscore);
  if (e) return cuda_fail(e, "map threshold tuning");
  // largest tau with recall >= min_recall: the ceil(min_recall * P)-th largest positive score
  std::vector<int32_t> pos;
  for (int i = 0; i < n; ++i)
    if (y[i]) pos.push_back(z[i]);
  if (pos.empty()) return fail(SC_ERR_INVALID, "no positive labels");
  std::sort(pos.begin(), pos.end(), std::greater<int32_t>());
  const size_t need = (size_t)std::ceil((double)min_recall * pos.size());
  const int32_t tau = pos[std::min(pos.size(), std::max<size_t>(need, 1)) - 1];
  size_t tp = 0, pass = 0;
  for (int i = 0; i < n; ++i)
    if (z[i] >= tau) { ++pass; tp += y[i] ? 1 : 0; }
  m->tau = tau;
  if (tau_out) *tau_out = tau;
  if (recall_out) *recall_out = (float)tp / pos.size();
  if (pass_rate_out) *pass_rate_out = (float)pass / n;
  return SC_OK;
}

sc_status sc_rmap_set_threshold(sc_rmap* m, int32_t tau) {
  g_err.clear();
  if (!m) return fail(SC_ERR_INVALID, "map is NULL");
  if (tau < 0 || tau > 65536) return fail(SC_ERR_INVALID, "tau = %d outside 0..65536", tau);
  m->tau = tau;
  return SC_OK;
}

sc_status sc_rmap_get_counts(sc_ctx* ctx, const sc_rmap* m, uint32_t* counts) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  if (!m || !counts) return fail(SC_ERR_INVALID, "map or counts is NULL");
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (!e) e = cudaMemcpy(counts, m->counts, m->g.cells * sizeof(uint2), cudaMemcpyDeviceToHost);
  if (e) return cuda_fail(e, "map read-back");
  return SC_OK;
}

// File: "SCMLP001", int64 step, int32 n_params, float params[n], m[n], v[n], mu[9], sigma[9], tau.
sc_status sc_mlp_save(sc_ctx* ctx, const sc_mlp* m, const char* path) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  if (!m || !path) return fail(SC_ERR_INVALID, "mlp or path is NULL");
  DeviceGuard g(ctx->device);
  const int n = sc::mlp_param_count();
  std::vector<float> buf(3 * (size_t)n + 18);
  float inv[9];
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (!e) e = cudaMemcpy(buf.data(), sc::mlp_params_ptr(m->st), n * 4, cudaMemcpyDeviceToHost);
  if (!e) e = cudaMemcpy(buf.data() + n, sc::mlp_m_ptr(m->st), n * 4, cudaMemcpyDeviceToHost);
  if (!e) e = cudaMemcpy(buf.data() + 2 * n, sc::mlp_v_ptr(m->st), n * 4, cudaMemcpyDeviceToHost);
  if (!e) e = cudaMemcpy(buf.data() + 3 * n, sc::mlp_mu_ptr(m->st), 36, cudaMemcpyDeviceToHost);
  if (!e) e = cudaMemcpy(inv, sc::mlp_inv_sigma_ptr(m->st), 36, cudaMemcpyDeviceToHost);
  if (e) return cuda_fail(e, "surrogate read-back");
  for (int i = 0; i < 9; ++i) buf[3 * (size_t)n + 9 + i] = 1.f / inv[i];
  FILE* f = fopen(path, "wb");
  if (!f) return fail(SC_ERR_INVALID, "cannot open %s for writing", path);
  const int64_t step = sc::mlp_step(m->st);
  const int32_t np = n;
  bool ok = fwrite("SCMLP001", 1, 8, f) == 8 && fwrite(&step, 8, 1, f) == 1 && fwrite(&np, 4, 1, f) == 1 &&
            fwrite(buf.data(), 4, buf.size(), f) == buf.size() && fwrite(&m->tau, 4, 1, f) == 1;
  ok = (fclose(f) == 0) && ok;
  if (!ok) return fail(SC_ERR_INVALID, "write to %s failed", path);
  return SC_OK;
}

sc_status sc_mlp_load(sc_ctx* ctx, const char* path, sc_mlp** out) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  if (!path || !out) return fail(SC_ERR_INVALID, "path or out is NULL");
  FILE* f = fopen(path, "rb");
  if (!f) return fail(SC_ERR_INVALID, "cannot open %s", path);
  char magic[8];
  int64_t step = 0;
  int32_t np = 0;
  const int n = sc::mlp_param_count();
  std::vector<float> buf(3 * (size_t)n + 18);
  float tau = 0.f;
  bool ok = fread(magic, 1, 8, f) == 8 && !std::memcmp(magic, "SCMLP001", 8) && fread(&step, 8, 1, f) == 1 &&
            fread(&np, 4, 1, f) == 1 && np == n && fread(buf.data(), 4, buf.size(), f) == buf.size() &&
            fread(&tau, 4, 1, f) == 1;
  fclose(f);
  if (!ok) return fail(SC_ERR_INVALID, "%s is not a surrogate file of this version", path);
  sc_mlp* m = nullptr;
  if (sc_status s = sc_mlp_create(ctx, 0, &m)) return s;
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (!e) e = cudaMemcpy(sc::mlp_m_ptr(m->st), buf.data() + n, n * 4, cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(sc::mlp_v_ptr(m->st), buf.data() + 2 * n, n * 4, cudaMemcpyHostToDevice);
  if (e) { sc_mlp_destroy(m); return cuda_fail(e, "surrogate upload"); }
  if (sc_status s = sc_mlp_set(ctx, m, buf.data(), buf.data() + 3 * n, buf.data() + 3 * n + 9, tau)) {
    sc_mlp_destroy(m);
    return s;
  }
  sc::mlp_set_step(m->st, step);
  *out = m;
  return SC_OK;
}

sc_status sc_ctx_set_timing(sc_ctx* ctx, int32_t on) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  DeviceGuard g(ctx->device);
  if (on && ctx->tev.empty()) {
    const int cap = 8192;
    ctx->tev.resize(2 * cap);
    ctx->tcls.resize(cap);
    for (auto& e : ctx->tev) {
      cudaError_t err = cudaEventCreate(&e);
      if (err != cudaSuccess) {
        for (auto& x : ctx->tev)
          if (x) cudaEventDestroy(x);
        ctx->tev.clear();
        ctx->tcls.clear();
        return cuda_fail(err, "cudaEventCreate");
      }
    }
    ctx->timer.ev = ctx->tev.data();
    ctx->timer.cls = ctx->tcls.data();
    ctx->timer.cap = cap;
  }
  ctx->timing = on ? 1 : 0;
  return SC_OK;
}

sc_status sc_generate_stats(sc_ctx* ctx, sc_gen_stats* out) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  if (!out) return fail(SC_ERR_INVALID, "out is NULL");
  DeviceGuard g(ctx->device);
  unsigned long long h[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  cudaError_t e = cudaMemcpyAsync(h, ctx->d_stats, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream);
  if (!e) e = cudaStreamSynchronize(ctx->stream);
  if (e) return cuda_fail(e, "stats read");
  std::memset(out, 0, sizeof(*out));
  out->sphere_pairs = (int64_t)h[0];
  out->sphere_box_pairs = (int64_t)h[1];
  out->ik_solves = (int64_t)h[2];
  out->gate_rejections = (int64_t)h[3];
  out->ik_seed_iterations = (int64_t)h[4];
  out->cull_tests = (int64_t)h[5];
  out->exhaustive_pairs = (int64_t)h[6];
  out->sphere_tri_pairs = (int64_t)h[7];
  out->reach_bound_rejections = (int64_t)h[8];
  if (ctx->timing) {
    for (int i = 0; i < ctx->timer.used; ++i) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, ctx->tev[2 * i], ctx->tev[2 * i + 1]);
      if (e) return cuda_fail(e, "cudaEventElapsedTime");
      const int c = ctx->tcls[i];
      if (c >= 0 && c < 3) {
        out->ms_stage[c] += ms;
        out->launches_stage[c] += 1;
      }
    }
  }
  return SC_OK;
}

sc_status sc_generate_trace(sc_ctx* ctx, int32_t cap, int32_t* n, int32_t* stage, float* start_ms, float* end_ms) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  if (!n || cap < 0 || (cap > 0 && (!stage || !start_ms || !end_ms)))
    return fail(SC_ERR_INVALID, "NULL output or negative cap");
  DeviceGuard g(ctx->device);
  *n = ctx->timing ? ctx->timer.used : 0;
  if (*n == 0) return SC_OK;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e) return cuda_fail(e, "synchronize");
  const int m = *n < cap ? *n : cap;
  for (int i = 0; i < m; ++i) {
    float a = 0.f, b = 0.f;
    e = cudaEventElapsedTime(&a, ctx->tev[0], ctx->tev[2 * i]);
    if (!e) e = cudaEventElapsedTime(&b, ctx->tev[0], ctx->tev[2 * i + 1]);
    if (e) return cuda_fail(e, "cudaEventElapsedTime");
    stage[i] = ctx->tcls[i];
    start_ms[i] = a;
    end_ms[i] = b;
  }
  return SC_OK;
}

sc_status sc_collide_last_work(sc_ctx* ctx, int64_t* sphere_pairs, int64_t* sphere_box_pairs) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  DeviceGuard g(ctx->device);
  unsigned long long h[2] = {0, 0};
  cudaError_t e = cudaMemcpyAsync(h, ctx->d_stats, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "stats read");
  if (sphere_pairs) *sphere_pairs = (int64_t)h[0];
  if (sphere_box_pairs) *sphere_box_pairs = (int64_t)h[1];
  return SC_OK;
}

sc_status sc_ik_last_work(sc_ctx* ctx, int64_t* seed_iterations) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  if (!seed_iterations) return fail(SC_ERR_INVALID, "seed_iterations is NULL");
  DeviceGuard g(ctx->device);
  unsigned long long h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, ctx->d_stats + 4, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "stats read");
  *seed_iterations = (int64_t)h;
  return SC_OK;
}

sc_status sc_collide_last_tri_work(sc_ctx* ctx, int64_t* sphere_tri_pairs) {
  g_err.clear();
  if (sc_status s = check_ctx(ctx)) return s;
  DeviceGuard g(ctx->device);
  unsigned long long h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, ctx->d_stats + 7, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "stats read");
  if (sphere_tri_pairs) *sphere_tri_pairs = (int64_t)h;
  return SC_OK;
}

sc_status sc_order_by_work(int32_t n_templates, const int32_t* tmpl_obj_off, const int32_t* obj_sph_off,
                           const int32_t* cand_tmpl_off, int32_t* out_order) {
  g_err.clear();
  if (n_templates < 1 || !tmpl_obj_off || !obj_sph_off || !cand_tmpl_off || !out_order)
    return fail(SC_ERR_INVALID, "bad arguments to sc_order_by_work");
  std::vector<double> work(n_templates);
  for (int t = 0; t < n_templates; ++t) {
    double s = 0, s2 = 0;
    for (int o = tmpl_obj_off[t]; o < tmpl_obj_off[t + 1]; ++o) {
      double n = obj_sph_off[o + 1] - obj_sph_off[o];
      s += n;
      s2 += n * n;
    }
    work[t] = 0.5 * (s * s - s2);  // pairs of spheres in different objects
  }
  std::vector<int> tm(n_templates);
  std::iota(tm.begin(), tm.end(), 0);
  std::stable_sort(tm.begin(), tm.end(), [&](int x, int y) { return work[x] > work[y]; });
  int k = 0;
  for (int t : tm)
    for (int c = cand_tmpl_off[t]; c < cand_tmpl_off[t + 1]; ++c) out_order[k++] = c;
  return SC_OK;
}

}  // extern "C"
