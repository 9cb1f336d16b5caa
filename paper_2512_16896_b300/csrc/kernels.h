// Host-side launch wrappers of the CUDA kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "rmap.h"
#include "sceniris.h"

namespace sc {

cudaError_t launch_sample_parts(const sc_scene_batch& b, uint64_t seed, const int32_t* active, int n_items,
                               float* part_q, int* status, int num_sms, cudaStream_t s);
cudaError_t launch_sample(const sc_scene_batch& b, const sc_sample_params& p, const int32_t* active, int n_items,
                          float* poses, uint8_t* ok, uint8_t* band, int* status, int num_sms, cudaStream_t s);

struct CollideLaunch {
  const float* poses;
  const int32_t* active;
  int n_items;
  int first_new;
  uint8_t* collide;
  float* min_dist;
  uint8_t* band;
  unsigned int* counter;          // scratch: work counter, zeroed by the launcher
  unsigned long long* stats;      // scratch: [0] sphere pairs, [1] sphere-box pairs
  int* status;
};

// Validates the config against the batch (returns cudaErrorInvalidValue with
// *why set when it cannot run) and enqueues the persistent kernel.
cudaError_t launch_collide(const sc_scene_batch& b, const CollideLaunch& a, const sc_collide_config& cfg, int num_sms,
                           cudaStream_t s, const char** why);

// Error message / batch validation of the C ABI (defined in api.cu) for entry
// points that live in other files.
void set_error_message(const std::string& msg);
sc_status validate_batch(const sc_scene_batch* b);

struct MlpState;

// Optional stage timing: event pairs recorded around launches, by class
// (0 = generation step, 1 = grasp targets + gate, 2 = exact IK).
struct StageTimer {
  cudaEvent_t* ev = nullptr;  // pool of 2 * cap events
  int* cls = nullptr;         // class of each pair
  int cap = 0;
  int used = 0;
  // Inside a stream capture the records must be external event nodes (a plain
  // record would only be an internal dependency); outside, plain records.
  unsigned int flags = cudaEventRecordDefault;
  void begin(int c, cudaStream_t s) {
    if (!ev || used >= cap) return;
    cls[used] = c;
    cudaEventRecordWithFlags(ev[2 * used], s, flags);
  }
  void end(cudaStream_t s) {
    if (!ev || used >= cap) return;
    cudaEventRecordWithFlags(ev[2 * used + 1], s, flags);
    ++used;
  }
};

struct GenerateLaunch {
  const int32_t* order;  // candidates to generate (NULL: 0..n_items-1)
  int n_items;
  const unsigned long long* seed_dev;  // device scalar holding the Philox seed
  int max_attempts, max_retries;
  float* poses;
  uint8_t* valid;
  uint8_t* band;
  int32_t* tries;
  void* scratch;  // generate_scratch_bytes(batch, n_items, max_retries)
  unsigned long long* stats;  // [0] sphere pairs [1] sphere-box pairs [2] IK solves [3] gate rejections
                              // [4] IK seed-iterations [5] cull tests [6] exhaustive pairs
  int* status;
  // reachability (arm == NULL: none)
  const sc_arm* arm;
  const sc_ik_params* ik;
  const MlpState* gate;  // NULL: exact IK on every candidate
  float tau;
  const uint2* map_counts;  // 4D reachability map gate instead of the surrogate (NULL: none)
  RmapGrid map_grid;
  int map_tau;
  int reach_objects;     // object indices < reach_objects may carry the reach flag
  int max_sph_obj;       // most spheres of one object in the batch (batch_scan)
  int ext_rel;           // generation instance: 0 basic relations, 1 DIRECTIONAL / MIDDLE / LOCAL /
                         // FACE_TO in use (batch_scan), 2 also parts or world triangles
  float* q_reach;        // [P][7] IK solution of every reach-checked placed object (may be NULL)
  StageTimer* timer;     // NULL: no timing
  // rounds of the objects with reachability: two side streams for the reach
  // stages and 2 * generate_rounds(reach_objects, max_retries) + 1 events
  cudaStream_t side[2];
  cudaEvent_t* events;
  int n_events;
};

// Upper bound on the rounds the objects with reachability take (a try of a
// reach-flagged object spans two rounds).
int generate_rounds(int reach_objects, int max_retries);

size_t generate_scratch_bytes(const sc_scene_batch& b, int n_items, int max_retries);
// Byte offset of the 8-byte seed scalar inside that scratch (256-aligned).
size_t generate_seed_offset(const sc_scene_batch& b, int n_items, int max_retries);
// out_host3[0]: 1 + largest object index with the reach flag; [1]: most
// spheres of one object; [2]: 1 if some object uses a relation beyond FREE /
// ON_TOP / NEXT_TO (uses 3 device ints; synchronises the stream).
cudaError_t batch_scan(const sc_scene_batch& b, int* scratch_int3, int* out_host3, cudaStream_t s);
// Enqueues the whole generation (init + one launch per object and try).
cudaError_t enqueue_generate(const sc_scene_batch& b, const GenerateLaunch& a, const sc_collide_config& cfg,
                             int num_sms, cudaStream_t s, const char** why);

// claim: a device work counter, zeroed by the launcher on the stream.
cudaError_t launch_ik(const sc_arm& arm, const sc_ik_params& P, const float* targets, const uint32_t* target_ids,
                      int n, uint8_t* reach, float* q_out, float* err, int32_t* iters_out, uint8_t* band,
                      unsigned int* claim, unsigned long long* seed_iters, int num_sms, cudaStream_t s);
// Blocks of 128 threads of the IK kernels that fit on the device at once.
int ik_resident_blocks(int num_sms);
cudaError_t launch_ik_step(const sc_arm& arm, float lambda, const float* targets, const float* q_in, int n,
                           float* q_out, float* tool, int num_sms, cudaStream_t s);

// ---- surrogate MLP (mlp.cu)
struct MlpState;
int mlp_param_count();

// Weights of the surrogate as the tensor-core forward pass reads them.
struct MlpTcWeights {
  const float* params;     // FP32 masters (biases)
  const void* W1c;         // bf16 [256][16] canonical layout (see canon_offset)
  const void* W2c;         // bf16 [256][256] canonical layout
  const void* W3c;
  const void* W2k;         // the same K-sliced: 16 x [256][16] canonical (8 KB each)
  const void* W3k;
  const void* W4;          // bf16 [256]
  const float* mu;         // [9]
  const float* inv_sigma;  // [9]
  int off_b1, off_b2, off_b3, off_b4;
};
// The tensor-core view of a surrogate's weights.
MlpTcWeights mlp_tc_weights(const MlpState* S);
// Logits of n rows of targets (or min(n, *n_dev) when n_dev is set) on
// tcgen05; a wait that gives up latches kDevTimeout into *status.
cudaError_t mlp_forward_tc(const MlpTcWeights& w, const float* targets, int n, const int* n_dev, float* logits,
                           int* status, int num_sms, cudaStream_t s);
cudaError_t mlp_alloc(MlpState** out);
void mlp_free(MlpState* S);
cudaError_t mlp_init(MlpState* S, uint64_t seed, cudaStream_t s);
cudaError_t mlp_refresh_copies(MlpState* S, cudaStream_t s);
cudaError_t mlp_set_norm_from(MlpState* S, const float* targets, int n, cudaStream_t s);
cudaError_t mlp_infer(const MlpState* S, const float* targets, int n, float* logits, int* status,
                      int num_sms, cudaStream_t s);
cudaError_t mlp_infer_counted(const MlpState* S, const float* targets, const int* n_dev, int n_cap, float* logits,
                              int* status, int num_sms, cudaStream_t s);
cudaError_t mlp_reserve(MlpState* S, int Bcap);
cudaError_t mlp_gradients(MlpState* S, const float* targets, const uint8_t* labels, const int32_t* index, int B,
                          float* loss_dev, int* status, int num_sms, cudaStream_t s);
// One training step's contractions on tcgen05 (mlp_train_tc.cu): the
// forward pass with its caches, the backward pass through the activations
// and the weight gradients dW1..dW3 (bias and last-layer gradients are
// summed by the caller). Feature-major arrays have row stride ld.
namespace mlpp {
struct AdamArgs;
}
struct TrainTcLaunch {
  MlpTcWeights w;
  const void* W2tc;  // bf16 canonical [in][out] copies (B operands of dH = dA W)
  const void* W3tc;
  const float* targets;
  const uint8_t* labels;
  const int32_t* index;  // batch row -> target / label (NULL: identity)
  int n;
  float* logits;         // [n]
  uint8_t* x16T;         // chunk-tiled (64-row chunks, canonical K-major over the rows): 16 features
  uint8_t* hT[2];        // chunk-tiled, 256 features: h1, h2
  uint8_t* daT[3];       // chunk-tiled, 256 features: dL/da1..3
  float* dz;             // [n]
  float* loss_sum;       // the mean BCE (written by the step)
  float* tile_sums;      // mlp_train_tc_tile_sum_bytes(n): per-tile sums of dz h3, dz and the BCE
  float* dW1;            // [256][9]
  float* dW2;            // [256][256]
  float* dW3;
  float* db[3];          // [256] bias gradients
  float* dW4;            // [256]
  float* db4;            // [1]
  int* status;
  const mlpp::AdamArgs* adam;  // non-NULL: Adam on every parameter as its gradient is written
};
size_t mlp_train_tc_tile_sum_bytes(int Bcap);
cudaError_t mlp_train_tc_step(const TrainTcLaunch& L, int num_sms, cudaStream_t s);
cudaError_t mlp_adam(MlpState* S, float lr, float b1, float b2, float eps, cudaStream_t s);
// One training step: the gradients of rows index[0..B) (as mlp_gradients)
// with the Adam update (as mlp_adam) applied by the weight-gradient kernel
// to each gradient it writes.
cudaError_t mlp_train_step(MlpState* S, const float* targets, const uint8_t* labels, const int32_t* index, int B,
                           float* loss_dev, int* status, int num_sms, float lr, float b1, float b2, float eps,
                           cudaStream_t s);
cudaError_t mlp_epoch_index(int n, uint64_t seed, int epoch, int32_t* index, cudaStream_t s);
float* mlp_params_ptr(MlpState* S);
float* mlp_grads_ptr(MlpState* S);
float* mlp_mu_ptr(MlpState* S);
float* mlp_inv_sigma_ptr(MlpState* S);
float* mlp_m_ptr(MlpState* S);
float* mlp_v_ptr(MlpState* S);
int64_t mlp_step(const MlpState* S);
void mlp_set_step(MlpState* S, int64_t t);

// NULL if the launch shape is valid, else why not.
const char* check_collide_config(const sc_collide_config& cfg);

// Dynamic shared memory one collide CTA needs for this batch and config.
size_t collide_smem_bytes(const sc_scene_batch& b, const sc_collide_config& cfg);

// Default launch shape of the collision kernel for a batch (decide_only = 0).
sc_collide_config default_collide_config(const sc_scene_batch& b);

}  // namespace sc
