// sc_collide_noalloc: the collision check for callers that cannot allocate
// device memory.
//
// sc_collide needs an sc_ctx, and creating one calls cudaMalloc for the
// kernel's scratch (its work counter and statistics). Some callers cannot do
// that: code whose device memory is owned by a framework's own pool and that
// may not allocate outside it, per-frame or real-time loops where a
// cudaMalloc would synchronise the device and stall, and code that keeps no
// library context at all. This entry point runs the same persistent kernel
// with its scratch in a fixed array compiled into the library instead.
//
// The array below is file-scope device memory: every GPU that loads the
// library holds it until the process exits. Host code must not pass its name
// to a kernel (in host code the name is only a host-side stand-in); the
// device address is looked up once per device with cudaGetSymbolAddress.
#include <mutex>
#include <string>

#include "common.cuh"
#include "kernels.h"

namespace {

// Scratch of one call: [0, 4) work counter (u32, zeroed by the launcher before
// each launch); work statistics as u64 words from byte 16: sphere pairs at
// [16, 24), sphere-box pairs at [24, 32) and point-triangle distances at
// [72, 80) (word 7), zeroed likewise; the rest is unused. Status is not
// latched here: candidates the kernel's own checks reject come back with
// min_dist = NaN and band = 1.
constexpr size_t kScratchBytes = 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};

// errors are reported through sc_last_error(), like every other call
sc_status fail(sc_status s, const std::string& msg) {
  sc::set_error_message(msg);
  return s;
}

}  // namespace

extern "C" {

// Declared in include/sceniris.h.
sc_status sc_collide_noalloc(void* cuda_stream, const sc_scene_batch* batch, const float* poses,
                             const int32_t* active, int32_t n_active, int32_t first_new_obj, uint8_t* collide,
                             float* min_dist, uint8_t* band) {
  sc::set_error_message("");
  if (sc_status s = sc::validate_batch(batch)) return s;
  if (active && n_active < 0) return fail(SC_ERR_INVALID, "sc_collide_noalloc: n_active < 0");
  const int64_t n_items = active ? n_active : batch->n_cand;
  if (n_items > SC_NOALLOC_MAX_ITEMS)
    return fail(SC_ERR_INVALID, "sc_collide_noalloc: " + std::to_string(n_items) +
                                    " candidates exceed the per-call limit of " +
                                    std::to_string(SC_NOALLOC_MAX_ITEMS) +
                                    " (the 32-bit work counter runs past the end by up to the grid size)");
  if (n_items == 0) return SC_OK;
  if (!poses || !collide || !min_dist || !band)
    return fail(SC_ERR_INVALID, "sc_collide_noalloc: an input or output pointer is NULL");
  if (first_new_obj < 0) return fail(SC_ERR_INVALID, "sc_collide_noalloc: first_new_obj < 0");
  if (reinterpret_cast<uintptr_t>(poses) & 15) return fail(SC_ERR_INVALID, "sc_collide_noalloc: poses must be 16-byte aligned");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(SC_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(SC_ERR_UNSUPPORTED, "sc_collide_noalloc: device index too large");
  void* scratch = nullptr;
  int num_sms = 0;
  {
    // once per device, with that device current: find the array's device address
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return fail(SC_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      int sms = 0;
      e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return fail(SC_ERR_CUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
      g_num_sms[dev] = sms;
      g_scratch_addr[dev] = p;
    }
    scratch = g_scratch_addr[dev];
    num_sms = g_num_sms[dev];
  }
  sc::CollideLaunch a;
  a.poses = poses;
  a.active = active;
  a.n_items = (int)n_items;
  a.first_new = first_new_obj;
  a.collide = collide;
  a.min_dist = min_dist;
  a.band = band;
  a.counter = reinterpret_cast<unsigned int*>(static_cast<char*>(scratch));
  a.stats = reinterpret_cast<unsigned long long*>(static_cast<char*>(scratch) + 16);
  a.status = nullptr;
  const sc_collide_config cfg = sc::default_collide_config(*batch);
  const char* why = nullptr;
  e = sc::launch_collide(*batch, a, cfg, num_sms, static_cast<cudaStream_t>(cuda_stream), &why);
  if (why) return fail(SC_ERR_INVALID, std::string("sc_collide_noalloc: ") + why);
  if (e != cudaSuccess) return fail(SC_ERR_CUDA, std::string("collide launch: ") + cudaGetErrorString(e));
  return SC_OK;
}

}  // extern "C"
