// Plain surrogate inference: logits of n rows of grasp targets with the
// tensor-core forward pass of mlp_tc_core.cuh (Sec. IV-E learned gate).
#include "mlp_tc_core.cuh"

namespace sc {

namespace {

// Rows from a target array [n][12] (R row-major, p), logits to an array.
struct PlainIO {
  static constexpr int kColGroups = 4;
  const float* targets;
  int n;
  const int* n_dev;  // optional device row count (n is then its cap)
  float* logits;
  __device__ int rows() const { return n_dev ? min(n, *(volatile const int*)n_dev) : n; }
  __device__ void features(int row, float f[9]) const {
    const float* t = targets + 12 * (size_t)row;
    f[0] = __ldg(t + 9); f[1] = __ldg(t + 10); f[2] = __ldg(t + 11);
    f[3] = __ldg(t + 0); f[4] = __ldg(t + 3); f[5] = __ldg(t + 6);
    f[6] = __ldg(t + 1); f[7] = __ldg(t + 4); f[8] = __ldg(t + 7);
  }
  __device__ void emit(int row, bool valid, float logit) const {
    if (valid) logits[row] = logit;
  }
};

}  // namespace

cudaError_t mlp_forward_tc(const MlpTcWeights& w, const float* targets, int n, const int* n_dev, float* logits,
                           int* status, int num_sms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  PlainIO io{targets, n, n_dev, logits};
  return launch_mlp_tc(w, io, n, status, num_sms, s);
}

}  // namespace sc
