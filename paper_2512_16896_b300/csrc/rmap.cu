// Build and query kernels of the 4D reachability map (the key is in rmap.h):
// one thread per target, counts added with integer atomics, a query one
// 8-byte gather of its cell.
#include "common.cuh"
#include "rmap.h"

namespace sc {

namespace {

__device__ __forceinline__ void load_target(const float* src, float t[12]) {
#pragma unroll
  for (int j = 0; j < 12; ++j) t[j] = __ldg(src + j);
}

__global__ void __launch_bounds__(256) rmap_build_kernel(RmapGrid g, uint2* counts, const float* targets,
                                                         const uint8_t* labels, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float t[12];
    load_target(targets + 12 * (size_t)i, t);
    const int cell = rmap_cell(g, t);
    if (cell < 0) continue;
    atomicAdd(&counts[cell].y, 1u);
    if (__ldg(labels + i)) atomicAdd(&counts[cell].x, 1u);
  }
}

__global__ void __launch_bounds__(256) rmap_query_kernel(RmapGrid g, const uint2* counts, const float* targets, int n,
                                                         uint16_t* score) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float t[12];
    load_target(targets + 12 * (size_t)i, t);
    score[i] = (uint16_t)rmap_score(counts, rmap_cell(g, t));
  }
}

int grid_for(int n, int num_sms) {
  const int blocks = (n + 255) / 256;
  const int cap = 8 * num_sms;
  return blocks < cap ? blocks : cap;
}

}  // namespace

cudaError_t rmap_build(const RmapGrid& g, uint2* counts, const float* targets, const uint8_t* labels, int n,
                       int num_sms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  rmap_build_kernel<<<grid_for(n, num_sms), 256, 0, s>>>(g, counts, targets, labels, n);
  return cudaGetLastError();
}

cudaError_t rmap_query(const RmapGrid& g, const uint2* counts, const float* targets, int n, uint16_t* score,
                       int num_sms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  rmap_query_kernel<<<grid_for(n, num_sms), 256, 0, s>>>(g, counts, targets, n, score);
  return cudaGetLastError();
}

}  // namespace sc
