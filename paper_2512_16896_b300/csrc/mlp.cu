// Reachability surrogate: an MLP 9 -> 256 -> 256 -> 256 -> 1 with SiLU,
// BF16 weights and activations, FP32 accumulation, trained with
// binary-cross-entropy on logits and Adam (the learned gate in front of the
// exact IK check of Sec. IV-E). Features of a target (R row-major, p):
// x = (p, R[:,0], R[:,1]), standardised by the stored mean / std.
//
// This file keeps the network's state (FP32 masters, Adam moments, the bf16
// weight copies in the tensor cores' canonical layout, the input
// standardisation, the training buffers) and the small kernels around
// training: the standalone Adam step, the weight copies, initialisation,
// the epoch shuffle. The contractions of inference and training run on
// tcgen05 (mlp_tc_core.cuh, mlp_tc.cu, mlp_train_tc.cu); a training step
// applies Adam inside its weight-gradient kernel (mlp_adam.cuh).
// Rounding points (matching the FP64 reference): standardised input, every
// SiLU output, W copies, and every dL/da are rounded to bf16; biases,
// pre-activations, accumulations, gradients and Adam state are FP32.
#include <cstring>

#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "mlp_adam.cuh"

namespace sc {

namespace {

using mlpp::H;
using mlpp::KIN;
using mlpp::OFF_W1;
using mlpp::OFF_B1;
using mlpp::OFF_W2;
using mlpp::OFF_B2;
using mlpp::OFF_W3;
using mlpp::OFF_B3;
using mlpp::OFF_W4;
using mlpp::OFF_B4;
using mlpp::N_PARAMS;

// Features of one target (12 floats).
__device__ __forceinline__ void features(const float* t, float x[9]) {
  x[0] = t[9]; x[1] = t[10]; x[2] = t[11];
  x[3] = t[0]; x[4] = t[3]; x[5] = t[6];  // R[:,0]
  x[6] = t[1]; x[7] = t[4]; x[8] = t[7];  // R[:,1]
}

// Adam on the FP32 masters (step t, 1-based); each updated weight also
// rewrites its bf16 copies in the canonical layouts (as mlp_copies_kernel).
__global__ void mlp_adam_kernel(mlpp::AdamArgs a, const float* grads, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    mlpp::adam_update(a, i, grads[i]);
}

// bf16 copies of the weights in the tensor cores' canonical K-major layout:
// W1c, W2c, W3c ([out][in], B operands of the forward pass; W2k, W3k the
// same K-sliced for the inference kernel's stream) and W2tc, W3tc
// ([in][out], B operands of the backward pass dH = dA W); W4 plain.
__global__ void mlp_copies_kernel(const float* params, __nv_bfloat16* W4, __nv_bfloat16* W1c, __nv_bfloat16* W2c,
                                  __nv_bfloat16* W3c, __nv_bfloat16* W2k, __nv_bfloat16* W3k, __nv_bfloat16* W2tc,
                                  __nv_bfloat16* W3tc) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < H * H; i += gridDim.x * blockDim.x) {
    const int n = i / H, k = i % H;
    const __nv_bfloat16 w2 = __float2bfloat16_rn(params[OFF_W2 + i]);
    const __nv_bfloat16 w3 = __float2bfloat16_rn(params[OFF_W3 + i]);
    W2c[canon_offset(n, k, H) / 2] = w2;
    W3c[canon_offset(n, k, H) / 2] = w3;
    W2k[mlpp::kslice_offset(n, k) / 2] = w2;
    W3k[mlpp::kslice_offset(n, k) / 2] = w3;
    W2tc[canon_offset(k, n, H) / 2] = w2;
    W3tc[canon_offset(k, n, H) / 2] = w3;
    if (i < H * KIN) {
      const int n1 = i / KIN, k1 = i % KIN;
      W1c[canon_offset(n1, k1, KIN) / 2] = __float2bfloat16_rn(k1 < 9 ? params[OFF_W1 + n1 * 9 + k1] : 0.f);
    }
    if (i < H) W4[i] = __float2bfloat16_rn(params[OFF_W4 + i]);
  }
}

// Per-feature sums and sums of squares (double) of the training targets.
__global__ void feature_moments_kernel(const float* targets, int n, double* acc /*[18]*/) {
  double s[9] = {0}, s2[9] = {0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float tt[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) tt[j] = targets[12 * (size_t)i + j];
    float x[9];
    features(tt, x);
#pragma unroll
    for (int j = 0; j < 9; ++j) { s[j] += x[j]; s2[j] += (double)x[j] * x[j]; }
  }
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    for (int off = 16; off > 0; off >>= 1) {
      s[j] += __shfl_xor_sync(0xFFFFFFFFu, s[j], off);
      s2[j] += __shfl_xor_sync(0xFFFFFFFFu, s2[j], off);
    }
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int j = 0; j < 9; ++j) { atomicAdd(&acc[j], s[j]); atomicAdd(&acc[9 + j], s2[j]); }
  }
}

__global__ void feature_norm_kernel(const double* acc, int n, float* mu, float* inv_sigma) {
  const int j = threadIdx.x;
  if (j < 9) {
    const double m = acc[j] / n;
    const double var = acc[9 + j] / n - m * m;
    const double sd = var > 1e-12 ? sqrt(var) : 1.0;  // a constant feature keeps unit scale
    mu[j] = (float)m;
    inv_sigma[j] = (float)(1.0 / sd);
  }
}

// Batch rows of an epoch: an affine permutation i -> (a i + c) mod n with
// gcd(a, n) = 1, a and c drawn from Philox (epoch-wise shuffling).
__global__ void epoch_index_kernel(int n, uint64_t a, uint64_t c, int32_t* index) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    index[i] = (int32_t)((a * (uint64_t)i + c) % (uint64_t)n);
}

// U(-1/sqrt(fan_in), 1/sqrt(fan_in)) initial weights and biases from Philox.
__global__ void mlp_init_kernel(float* params, uint64_t seed) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N_PARAMS; i += gridDim.x * blockDim.x) {
    const int fan_in = i < OFF_W2 ? 9 : i < OFF_W4 ? H : H;
    const float kk = rsqrtf((float)fan_in);
    const float4 u = draw_uniform4(seed, (uint32_t)i, 0x4D4C50u, 0u, 0u);
    params[i] = kk * (2.f * u.x - 1.f);
  }
}

}  // namespace

// ------------------------------------------------------------------ host side

int mlp_param_count() { return N_PARAMS; }

struct MlpState {
  float* params = nullptr;  // device, FP32 masters
  float* m = nullptr;
  float* v = nullptr;
  float* grads = nullptr;
  __nv_bfloat16* W4 = nullptr;
  __nv_bfloat16 *W1c = nullptr, *W2c = nullptr, *W3c = nullptr;  // canonical [out][in] (forward)
  __nv_bfloat16 *W2k = nullptr, *W3k = nullptr;                   // the same, K-sliced (inference stream)
  __nv_bfloat16 *W2tc = nullptr, *W3tc = nullptr;                 // canonical [in][out] (backward)
  float* mu = nullptr;
  float* inv_sigma = nullptr;
  double* moments = nullptr;
  int64_t step = 0;
  // training scratch for a batch of Bcap rows
  int Bcap = 0;
  void* train_buf = nullptr;
};

cudaError_t mlp_alloc(MlpState** out) {
  MlpState* S = new (std::nothrow) MlpState;
  if (!S) return cudaErrorMemoryAllocation;
  const size_t nf = N_PARAMS;
  cudaError_t e;
  if ((e = cudaMalloc(&S->params, nf * 4)) || (e = cudaMalloc(&S->m, nf * 4)) || (e = cudaMalloc(&S->v, nf * 4)) ||
      (e = cudaMalloc(&S->grads, nf * 4)) || (e = cudaMalloc(&S->W4, H * 2)) ||
      (e = cudaMalloc(&S->W1c, H * KIN * 2)) || (e = cudaMalloc(&S->W2c, H * H * 2)) ||
      (e = cudaMalloc(&S->W3c, H * H * 2)) || (e = cudaMalloc(&S->W2k, H * H * 2)) ||
      (e = cudaMalloc(&S->W3k, H * H * 2)) || (e = cudaMalloc(&S->W2tc, H * H * 2)) ||
      (e = cudaMalloc(&S->W3tc, H * H * 2)) || (e = cudaMalloc(&S->mu, 64)) ||
      (e = cudaMalloc(&S->inv_sigma, 64)) || (e = cudaMalloc(&S->moments, 18 * 8))) {
    mlp_free(S);
    return e;
  }
  *out = S;
  return cudaSuccess;
}

void mlp_free(MlpState* S) {
  if (!S) return;
  void* ptrs[] = {S->params, S->m,   S->v,    S->grads, S->W4, S->W1c,        S->W2c,      S->W3c,
                  S->W2k,    S->W3k, S->W2tc, S->W3tc,  S->mu, S->inv_sigma, S->moments, S->train_buf};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete S;
}

cudaError_t mlp_refresh_copies(MlpState* S, cudaStream_t s) {
  mlp_copies_kernel<<<128, 256, 0, s>>>(S->params, S->W4, S->W1c, S->W2c, S->W3c, S->W2k, S->W3k, S->W2tc, S->W3tc);
  return cudaGetLastError();
}

cudaError_t mlp_init(MlpState* S, uint64_t seed, cudaStream_t s) {
  mlp_init_kernel<<<128, 256, 0, s>>>(S->params, seed);
  cudaError_t e;
  if ((e = cudaMemsetAsync(S->m, 0, N_PARAMS * 4, s)) || (e = cudaMemsetAsync(S->v, 0, N_PARAMS * 4, s))) return e;
  const float zeros[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, ones[9] = {1, 1, 1, 1, 1, 1, 1, 1, 1};
  if ((e = cudaMemcpyAsync(S->mu, zeros, 36, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(S->inv_sigma, ones, 36, cudaMemcpyHostToDevice, s)))
    return e;
  S->step = 0;
  return mlp_refresh_copies(S, s);
}

cudaError_t mlp_set_norm_from(MlpState* S, const float* targets, int n, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(S->moments, 0, 18 * 8, s);
  if (e) return e;
  feature_moments_kernel<<<256, 256, 0, s>>>(targets, n, S->moments);
  feature_norm_kernel<<<1, 32, 0, s>>>(S->moments, n, S->mu, S->inv_sigma);
  return cudaGetLastError();
}

static MlpTcWeights tc_view(const MlpState& S) {
  MlpTcWeights w;
  w.params = S.params;
  w.W1c = S.W1c;
  w.W2c = S.W2c;
  w.W3c = S.W3c;
  w.W2k = S.W2k;
  w.W3k = S.W3k;
  w.W4 = S.W4;
  w.mu = S.mu;
  w.inv_sigma = S.inv_sigma;
  w.off_b1 = OFF_B1;
  w.off_b2 = OFF_B2;
  w.off_b3 = OFF_B3;
  w.off_b4 = OFF_B4;
  return w;
}

MlpTcWeights mlp_tc_weights(const MlpState* S) { return tc_view(*S); }

cudaError_t mlp_infer(const MlpState* S, const float* targets, int n, float* logits, int* status, int num_sms,
                      cudaStream_t s) {
  return mlp_forward_tc(tc_view(*S), targets, n, nullptr, logits, status, num_sms, s);
}

cudaError_t mlp_infer_counted(const MlpState* S, const float* targets, const int* n_dev, int n_cap, float* logits,
                              int* status, int num_sms, cudaStream_t s) {
  return mlp_forward_tc(tc_view(*S), targets, n_cap, n_dev, logits, status, num_sms, s);
}

// Batch buffers of Bcap rows: the standardised input and h1, h2 (feature-
// major) for the weight gradients, the dL/da (feature-major), dz, logits,
// the loss word and the per-tile sums of dz h3 and dz. (SiLU'(z) stays in
// the tensor memory of the fused forward-backward kernel.)
struct TrainViews {
  uint8_t* x16T;    // chunk-tiled [Bt / 64][16 x 64] bf16
  uint8_t* hT[2];   // chunk-tiled [Bt / 64][256 x 64] bf16: h1, h2
  uint8_t* daT[3];  // chunk-tiled [Bt / 64][256 x 64] bf16
  float* dz;        // [Bcap]
  float* logits;    // [Bcap]
  float* loss_sum;
  float* part;      // mlp_train_tc_tile_sum_bytes(Bcap): per-tile sums
};

static size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// rows of the chunk-tiled caches: whole 128-row tiles
static size_t tiled_rows(int Bcap) { return ((size_t)Bcap + 127) / 128 * 128; }

static size_t train_bytes(int Bcap) {
  const size_t Bp = (size_t)Bcap, Bt = tiled_rows(Bcap);
  return align256(Bt * KIN * 2) + 2 * align256(Bt * H * 2) + 3 * align256(Bt * H * 2) + 2 * align256(Bp * 4) + 256 +
         align256(mlp_train_tc_tile_sum_bytes(Bcap));
}

static TrainViews carve(MlpState* S, int Bcap) {
  char* p = static_cast<char*>(S->train_buf);
  auto take = [&](size_t bytes) { char* r = p; p += align256(bytes); return r; };
  const size_t Bt = tiled_rows(Bcap);
  TrainViews v;
  v.x16T = reinterpret_cast<uint8_t*>(take(Bt * KIN * 2));
  for (int l = 0; l < 2; ++l) v.hT[l] = reinterpret_cast<uint8_t*>(take(Bt * H * 2));
  for (int l = 0; l < 3; ++l) v.daT[l] = reinterpret_cast<uint8_t*>(take(Bt * H * 2));
  v.dz = reinterpret_cast<float*>(take((size_t)Bcap * 4));
  v.logits = reinterpret_cast<float*>(take((size_t)Bcap * 4));
  v.loss_sum = reinterpret_cast<float*>(take(256));
  v.part = reinterpret_cast<float*>(take(mlp_train_tc_tile_sum_bytes(Bcap)));
  return v;
}

cudaError_t mlp_reserve(MlpState* S, int Bcap) {
  Bcap = (Bcap + 15) & ~15;
  if (Bcap <= S->Bcap) return cudaSuccess;
  if (S->train_buf) cudaFree(S->train_buf);
  S->train_buf = nullptr;
  S->Bcap = 0;
  cudaError_t e = cudaMalloc(&S->train_buf, train_bytes(Bcap));
  if (e) return e;
  S->Bcap = Bcap;
  return cudaSuccess;
}

// Gradients of the mean BCE over rows index[0..B) into S->grads (packed):
// the tcgen05 forward, backward and weight-gradient contractions and the
// bias and last-layer sums (mlp_train_tc.cu). Rows past B are never read
// (the weight-gradient staging masks them).
static cudaError_t gradients(MlpState* S, const float* targets, const uint8_t* labels, const int32_t* index, int B,
                             float* loss_dev, int* status, int num_sms, const mlpp::AdamArgs* adam, cudaStream_t s) {
  if (B > S->Bcap) return cudaErrorInvalidValue;
  TrainViews v = carve(S, S->Bcap);
  float* loss = loss_dev ? loss_dev : v.loss_sum;
  TrainTcLaunch L;
  L.w = tc_view(*S);
  L.W2tc = S->W2tc;
  L.W3tc = S->W3tc;
  L.targets = targets;
  L.labels = labels;
  L.index = index;
  L.n = B;
  L.logits = v.logits;
  L.x16T = v.x16T;
  for (int l = 0; l < 2; ++l) L.hT[l] = v.hT[l];
  for (int l = 0; l < 3; ++l) L.daT[l] = v.daT[l];
  L.dz = v.dz;
  L.loss_sum = loss;
  L.tile_sums = v.part;
  L.dW1 = S->grads + OFF_W1;
  L.dW2 = S->grads + OFF_W2;
  L.dW3 = S->grads + OFF_W3;
  L.db[0] = S->grads + OFF_B1;
  L.db[1] = S->grads + OFF_B2;
  L.db[2] = S->grads + OFF_B3;
  L.dW4 = S->grads + OFF_W4;
  L.db4 = S->grads + OFF_B4;
  L.status = status;
  L.adam = adam;
  return mlp_train_tc_step(L, num_sms, s);
}

// The Adam arguments of the next step (advances the step count).
static mlpp::AdamArgs next_adam(MlpState* S, float lr, float b1, float b2, float eps) {
  S->step += 1;
  const double t = (double)S->step;
  mlpp::AdamArgs a;
  a.params = S->params;
  a.m = S->m;
  a.v = S->v;
  a.lr = lr;
  a.b1 = b1;
  a.b2 = b2;
  a.eps = eps;
  a.ibc1 = (float)(1.0 / (1.0 - pow((double)b1, t)));
  a.ibc2 = (float)(1.0 / (1.0 - pow((double)b2, t)));
  a.W4 = S->W4;
  a.W1c = S->W1c;
  a.W2c = S->W2c;
  a.W3c = S->W3c;
  a.W2k = S->W2k;
  a.W3k = S->W3k;
  a.W2tc = S->W2tc;
  a.W3tc = S->W3tc;
  return a;
}

cudaError_t mlp_gradients(MlpState* S, const float* targets, const uint8_t* labels, const int32_t* index, int B,
                          float* loss_dev, int* status, int num_sms, cudaStream_t s) {
  return gradients(S, targets, labels, index, B, loss_dev, status, num_sms, nullptr, s);
}

cudaError_t mlp_train_step(MlpState* S, const float* targets, const uint8_t* labels, const int32_t* index, int B,
                           float* loss_dev, int* status, int num_sms, float lr, float b1, float b2, float eps,
                           cudaStream_t s) {
  if (B > S->Bcap) return cudaErrorInvalidValue;
  const mlpp::AdamArgs a = next_adam(S, lr, b1, b2, eps);
  return gradients(S, targets, labels, index, B, loss_dev, status, num_sms, &a, s);
}

cudaError_t mlp_adam(MlpState* S, float lr, float b1, float b2, float eps, cudaStream_t s) {
  const mlpp::AdamArgs a = next_adam(S, lr, b1, b2, eps);
  mlp_adam_kernel<<<(N_PARAMS + 255) / 256, 256, 0, s>>>(a, S->grads, N_PARAMS);
  return cudaGetLastError();
}

// Epoch shuffle: i -> (a i + c) mod n, a odd and coprime with n, both taken
// from a 64-bit mix of (seed, epoch).
cudaError_t mlp_epoch_index(int n, uint64_t seed, int epoch, int32_t* index, cudaStream_t s) {
  uint64_t x = seed * 0x9E3779B97F4A7C15ull + (uint64_t)(epoch + 1) * 0xBF58476D1CE4E5B9ull;
  x ^= x >> 31;
  x *= 0x94D049BB133111EBull;
  x ^= x >> 29;
  auto gcd = [](uint64_t p, uint64_t q) {
    while (q) { const uint64_t r = p % q; p = q; q = r; }
    return p;
  };
  uint64_t a = (x % (uint64_t)n) | 1u;
  while (gcd(a, (uint64_t)n) != 1) a = ((a + 2) % (uint64_t)n) | 1u;
  const uint64_t c = (x >> 23) % (uint64_t)n;
  epoch_index_kernel<<<256, 256, 0, s>>>(n, a, c, index);
  return cudaGetLastError();
}

float* mlp_params_ptr(MlpState* S) { return S->params; }
float* mlp_grads_ptr(MlpState* S) { return S->grads; }
float* mlp_mu_ptr(MlpState* S) { return S->mu; }
float* mlp_inv_sigma_ptr(MlpState* S) { return S->inv_sigma; }
float* mlp_m_ptr(MlpState* S) { return S->m; }
float* mlp_v_ptr(MlpState* S) { return S->v; }
int64_t mlp_step(const MlpState* S) { return S->step; }
void mlp_set_step(MlpState* S, int64_t t) { S->step = t; }

}  // namespace sc
