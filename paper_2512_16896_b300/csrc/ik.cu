// Reachability by damped-least-squares IK (Sec. IV-E: reject a sampled pose
// the robot cannot reach; the paper queries an RM4D map, this build solves
// IK exactly). 7-DoF serial arm in standard DH form:
//   T_i = Rz(q_i) Tz(d_i) Tx(a_i) Rx(alpha_i),  tool frame = frame 7.
// One warp per target, one seed per lane, all seeds in lock step:
//   check every seed (|p* - p| <= tol_pos and angle(R^T R*) <= tol_rot); the
//   first check where any seed succeeds ends the target with the lowest such
//   seed; otherwise step every seed by
//     dq = J^T (J J^T + lambda^2 I)^-1 e,  e = [p* - p; 1/2 sum_k r_k x r*_k],
//   and clamp q to the joint limits. After `iters` steps and a last check the
//   target is unreachable and returns the seed with the smallest position
//   error. FK, the geometric Jacobian, the 6x6 system and its Cholesky factor
//   live in registers.
#include "ik_core.cuh"
#include "kernels.h"

namespace sc {

namespace {

using namespace ikc;

// Targets cost from one check to iters steps, so warps claim them one at a
// time (first target static, the claim for the next issued before solving
// the current one) from a grid sized to the resident blocks.
// kRight: the signed forward kinematics of arms whose middle twists are
// +-pi/2 (ArmK::right).
template <bool kRight>
__global__ void __launch_bounds__(128) ik_kernel(IkArgs K) {
  const int lane = threadIdx.x & 31;
  const int warps = blockDim.x >> 5;
  const int warps_total = gridDim.x * warps;
  unsigned long long seed_iters = 0;
  int i = blockIdx.x * warps + (threadIdx.x >> 5);
  while (i < K.n) {
    int next = 0;
    if (lane == 0) next = warps_total + (int)atomicAdd(K.claim, 1u);
    const Target T = load_target(K.targets + 12 * (size_t)i);
    const uint32_t tid = K.target_ids ? __ldg(&K.target_ids[i]) : (uint32_t)i;
    float q[7], pe2, s, c;
    const Solve r = warp_solve<kRight>(K, T, tid, 0u, lane, q, pe2, s, c);
    seed_iters += (unsigned long long)r.checks * (unsigned long long)K.seeds;
    if (lane == r.winner) {
      K.reach[i] = r.found;
#pragma unroll
      for (int j = 0; j < 7; ++j) K.q_out[7 * (size_t)i + j] = q[j];
      K.err[2 * (size_t)i] = sqrtf(pe2);
      K.err[2 * (size_t)i + 1] = atan2f(s, c);
      if (K.iters_out) K.iters_out[i] = r.it;
      if (K.band) K.band[i] = r.band;
    }
    i = __shfl_sync(0xFFFFFFFFu, next, 0);
  }
  if (lane == 0 && seed_iters && K.seed_iters) atomicAdd(K.seed_iters, seed_iters);
}

// One DLS step for each (target, configuration) pair: the building block the
// tests compare against the FP64 step.
template <bool kRight>
__global__ void ik_step_kernel(ArmK arm, float lambda2, const float* targets, const float* q_in, int n, float* q_out,
                               float* tool) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const Target T = load_target(targets + 12 * (size_t)i);
    float q[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) q[j] = q_in[7 * (size_t)i + j];
    float z[7][3], p[7][3], Rh[9], t[3];
    fk<kRight>(arm, q, z, p, Rh, t);
    if (tool) {
      float R[9];
      tool_rotation(arm, Rh, R);
#pragma unroll
      for (int j = 0; j < 9; ++j) tool[12 * (size_t)i + j] = R[j];
#pragma unroll
      for (int j = 0; j < 3; ++j) tool[12 * (size_t)i + 9 + j] = t[j];
    }
    const Target H = target_frame(arm, T);
    float v[3], c;
    rot_error(H, Rh, v, &c);
    dls_step(arm, lambda2, H, q, z, p, Rh, t, v);
#pragma unroll
    for (int j = 0; j < 7; ++j) q_out[7 * (size_t)i + j] = q[j];
  }
}

}  // namespace

int ik_resident_blocks(int num_sms) {
  static int per_sm = 0;
  if (per_sm == 0) {
    int a = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, ik_kernel<false>, 128, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ik_kernel<true>, 128, 0) != cudaSuccess)
      a = b = 4;
    per_sm = a < b ? a : b;
  }
  return num_sms * (per_sm > 0 ? per_sm : 1);
}

cudaError_t launch_ik(const sc_arm& arm, const sc_ik_params& P, const float* targets, const uint32_t* target_ids,
                      int n, uint8_t* reach, float* q_out, float* err, int32_t* iters_out, uint8_t* band,
                      unsigned int* claim, unsigned long long* seed_iters, int num_sms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(claim, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess && seed_iters) e = cudaMemsetAsync(seed_iters, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  IkArgs K;
  fill_params(K, arm, P);
  K.targets = targets;
  K.target_ids = target_ids;
  K.n = n;
  K.reach = reach;
  K.q_out = q_out;
  K.err = err;
  K.iters_out = iters_out;
  K.band = band;
  K.seed_iters = seed_iters;
  K.claim = claim;
  const int threads = 128, warps = threads / 32;
  int blocks = (n + warps - 1) / warps;
  const int cap = ik_resident_blocks(num_sms);
  if (blocks > cap) blocks = cap;
  if (K.arm.right)
    ik_kernel<true><<<blocks, threads, 0, s>>>(K);
  else
    ik_kernel<false><<<blocks, threads, 0, s>>>(K);
  return cudaGetLastError();
}

cudaError_t launch_ik_step(const sc_arm& arm, float lambda, const float* targets, const float* q_in, int n,
                           float* q_out, float* tool, int num_sms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int blocks = (n + 127) / 128;
  if (blocks > num_sms * 8) blocks = num_sms * 8;
  const ArmK k = make_arm(arm);
  if (k.right)
    ik_step_kernel<true><<<blocks, 128, 0, s>>>(k, lambda * lambda, targets, q_in, n, q_out, tool);
  else
    ik_step_kernel<false><<<blocks, 128, 0, s>>>(k, lambda * lambda, targets, q_in, n, q_out, tool);
  return cudaGetLastError();
}

}  // namespace sc
