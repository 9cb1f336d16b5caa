// Collision check: per-candidate SE(3) transform of the object sphere sets and
// the minimum signed distance over sphere-sphere pairs of different objects
// and sphere-box pairs against the static world (Sec. IV-B one transform per
// instance, Sec. IV-D batched collision checking; spheres and oriented boxes
// stand in for cuRobo's meshes).
//
// Design (sm_103a, FP32 pipe bound):
//  * Persistent CTAs take candidates from the caller's list through a global
//    atomic counter (list the heaviest first).
//  * A CTA moves its candidate's spheres into shared memory once, expressed
//    relative to the pose of object 0 so that coordinates stay small.
//  * The sphere-pair set {(i, j): obj(i) < obj(j), obj(j) >= first_new} is cut
//    into units of (A block of 32*APL consecutive spheres held in registers,
//    one per lane per slot) x (segment of up to seg_len B spheres broadcast
//    from shared memory). Warps pull units from a CTA-local counter.
//  * Inner loop, per pair: with t = r_i + r_j + m (m = running minimum), the
//    pair can lower m iff |a - b|^2 < t^2. Expanding,
//        |a|^2 - q_i^2  +  |b|^2 - r_j^2  -  2 a.b  -  2 q_i r_j  <  0,   q_i = r_i + m,
//    which is one add and four FMAs with the per-sphere terms precomputed. A
//    slack eps (bounding the FP32 rounding of this sum) makes the test never
//    miss an improvement; hits recompute the exact distance
//    sqrt(|a - b|^2) - r_i - r_j and lower m. The reduction is therefore the
//    exact minimum of the per-pair distances.
//  * An A sphere whose r_i + m + max r_j < 0 cannot lower m any more and is
//    retired; a unit whose A spheres are all retired is skipped.
#include <cfloat>
#include <climits>

#include "common.cuh"
#include "kernels.h"

namespace sc {

namespace {

constexpr int kPad = 8;       // dummy spheres after the last one (group tail reads)
constexpr int kGroup = 4;     // B spheres per prune group
constexpr float kRetired = 1e30f;

__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }

struct Layout {
  int W, beta, oid, off, opose, osc, obb, blk_lo, blk_mend, blk_pref, total, nb_max, cap;
};

__host__ __device__ inline Layout make_layout(int max_sph, int max_obj, int apl) {
  Layout L;
  L.cap = ((max_sph + kPad + 7) / 8) * 8;
  L.nb_max = L.cap / (32 * apl) + 2;
  L.W = 0;
  L.beta = align16(L.W + 16 * L.cap);
  L.oid = align16(L.beta + 4 * L.cap);
  L.off = align16(L.oid + L.cap);
  L.opose = align16(L.off + 4 * (max_obj + 1));
  L.osc = align16(L.opose + 16 * max_obj);
  L.obb = align16(L.osc + 8 * max_obj);
  L.blk_lo = align16(L.obb + 4 * 16 * kMaxObbPerTemplate);
  L.blk_mend = align16(L.blk_lo + 4 * L.nb_max);
  L.blk_pref = align16(L.blk_mend + 4 * L.nb_max);
  L.total = align16(L.blk_pref + 4 * (L.nb_max + 1));
  return L;
}

struct KArgs {
  sc_scene_batch b;
  CollideLaunch a;
  int seg_len;
};

// largest k in [0, n) with arr[k] <= v, for non-decreasing arr with arr[0] <= v
__device__ __forceinline__ int upper_index(const int* arr, int n, int v) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (arr[mid] <= v) lo = mid; else hi = mid;
  }
  return lo;
}

template <int APL>
struct ABlock {
  float ax[APL], ay[APL], az[APL];  // -2 * centre
  float a2[APL], r[APL];            // |centre|^2, radius
  float qq[APL], al[APL];           // -2 q_i, |a|^2 - q_i^2 - eps (kRetired when retired)
  int bst[APL];                     // first B index this sphere may pair with (INT_MAX: padding)
  bool act[APL];
};

template <int APL>
__device__ __forceinline__ bool refresh(ABlock<APL>& A, float m, float rmax, float eps) {
  bool any = false;
#pragma unroll
  for (int s = 0; s < APL; ++s) {
    const float q = A.r[s] + m;
    const bool act = (A.bst[s] != INT_MAX) && (q + rmax >= 0.f);
    A.act[s] = act;
    A.qq[s] = -2.f * q;
    A.al[s] = act ? (A.a2[s] - q * q - eps) : kRetired;
    any |= act;
  }
  return __any_sync(0xFFFFFFFFu, any);
}

// Exact distances of the A block against B spheres [j, j + kGroup) (only the
// pairs allowed for each A sphere, only real B spheres), folded into m.
template <int APL>
__device__ __forceinline__ float slow_group(const ABlock<APL>& A, const float4* W, int j, int S, float m) {
  float mloc = m;
#pragma unroll
  for (int g = 0; g < kGroup; ++g) {
    const int jj = j + g;
    if (jj >= S) break;
    const float4 B = W[jj];
#pragma unroll
    for (int s = 0; s < APL; ++s) {
      if (jj >= A.bst[s]) {
        const float dx = -0.5f * A.ax[s] - B.x, dy = -0.5f * A.ay[s] - B.y, dz = -0.5f * A.az[s] - B.z;
        const float d = sqrtf(dx * dx + dy * dy + dz * dz) - A.r[s] - B.w;
        mloc = fminf(mloc, d);
      }
    }
  }
  return warp_min(mloc);
}

template <int APL, bool MASKED>
__device__ __forceinline__ void sweep(ABlock<APL>& A, const float4* W, const float* beta, int jb, int je, int S,
                                      float& m, float rmax, float eps, int* best_key, bool& alive) {
  for (int j = jb; j < je; j += kGroup) {
    float4 B[kGroup];
    float bt[kGroup];
#pragma unroll
    for (int g = 0; g < kGroup; ++g) {
      B[g] = W[j + g];
      bt[g] = beta[j + g];
    }
    bool hit = false;
#pragma unroll
    for (int s = 0; s < APL; ++s) {
#pragma unroll
      for (int g = 0; g < kGroup; ++g) {
        float v = A.al[s] + bt[g];
        v = fmaf(A.ax[s], B[g].x, v);
        v = fmaf(A.ay[s], B[g].y, v);
        v = fmaf(A.az[s], B[g].z, v);
        v = fmaf(A.qq[s], B[g].w, v);
        if (MASKED) hit |= (v < 0.f) && (j + g >= A.bst[s]);
        else hit |= v < 0.f;
      }
    }
    if (__any_sync(0xFFFFFFFFu, hit)) {
      const float mn = slow_group<APL>(A, W, j, S, m);
      if (mn < m) {
        m = mn;
        if ((threadIdx.x & 31) == 0) atomicMin(best_key, float_key(m));
        alive = refresh<APL>(A, m, rmax, eps);
        if (!alive) return;
      }
    }
  }
}

template <int APL, int MAXT>
__global__ void __launch_bounds__(MAXT) collide_kernel(KArgs K) {
  extern __shared__ __align__(16) unsigned char smem[];
  const sc_scene_batch& b = K.b;
  const CollideLaunch& a = K.a;
  const Layout L = make_layout(b.max_sph, b.max_obj, APL);
  float4* W = reinterpret_cast<float4*>(smem + L.W);
  float* beta = reinterpret_cast<float*>(smem + L.beta);
  uint8_t* oid = smem + L.oid;
  int* off = reinterpret_cast<int*>(smem + L.off);
  float4* opose = reinterpret_cast<float4*>(smem + L.opose);
  float2* osc = reinterpret_cast<float2*>(smem + L.osc);
  float* obbd = reinterpret_cast<float*>(smem + L.obb);
  int* blk_lo = reinterpret_cast<int*>(smem + L.blk_lo);
  int* blk_mend = reinterpret_cast<int*>(smem + L.blk_mend);
  int* blk_pref = reinterpret_cast<int*>(smem + L.blk_pref);
  __shared__ int s_item, s_unit_next, s_total_units, s_best_key, s_r2max_key, s_rmax_key, s_nb;
  __shared__ float s_warp_min[32];

  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
  constexpr int BA = 32 * APL;
  unsigned long long my_pairs = 0, my_box = 0;

  for (;;) {
    if (tid == 0) {
      s_item = (int)atomicAdd(a.counter, 1u);
    }
    __syncthreads();
    const int item = s_item;
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
    int err = t < 0 ? kDevBadTemplate
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
    // ---- stage objects
    for (int k = tid; k < nt; k += nthr) {
      const float4 p = __ldg(reinterpret_cast<const float4*>(a.poses) + pbase + k);
      float sn, cs;
      sincosf(p.w, &sn, &cs);
      opose[k] = p;
      osc[k] = make_float2(sn, cs);
      off[k] = __ldg(&b.obj_sph_off[o0 + k]) - s0;
    }
    if (tid == 0) {
      off[nt] = S;
      s_best_key = float_key(kFarSentinel);
      s_unit_next = 0;
      s_r2max_key = 0;
      s_rmax_key = 0;
    }
    __syncthreads();
    const float4 ref = opose[0];
    // ---- stage spheres (world frame relative to ref)
    float r2max = 0.f, rmx = 0.f;
    for (int q = tid; q < S + kPad; q += nthr) {
      if (q < S) {
        const int k = upper_index(off, nt + 1, q);
        const float4 l = __ldg(reinterpret_cast<const float4*>(b.sph_local) + s0 + q);
        const float4 p = opose[k];
        const float2 sc2 = osc[k];
        const float x = (p.x - ref.x) + (sc2.y * l.x - sc2.x * l.y);
        const float y = (p.y - ref.y) + (sc2.x * l.x + sc2.y * l.y);
        const float z = (p.z - ref.z) + l.z;
        const float c2 = x * x + y * y + z * z;
        W[q] = make_float4(x, y, z, l.w);
        beta[q] = c2 - l.w * l.w;
        oid[q] = (uint8_t)k;
        r2max = fmaxf(r2max, c2);
        rmx = fmaxf(rmx, l.w);
      } else {
        W[q] = make_float4(1e6f, 1e6f, 1e6f, 0.f);
        beta[q] = 3e12f;
        oid[q] = 255;
      }
    }
    // ---- stage world boxes: columns of R, centre relative to ref, half extents
    for (int k = tid; k < nobb; k += nthr) {
      const float* o = b.obb + 12 * (bx0 + k);
      float qx = __ldg(o + 4), qy = __ldg(o + 5), qz = __ldg(o + 6), qw = __ldg(o + 7);
      const float inv = rsqrtf(qx * qx + qy * qy + qz * qz + qw * qw);
      qx *= inv; qy *= inv; qz *= inv; qw *= inv;
      float* d = obbd + 16 * k;
      // R (row-major) of the unit quaternion; store its columns
      d[0] = 1.f - 2.f * (qy * qy + qz * qz); d[1] = 2.f * (qx * qy + qz * qw); d[2] = 2.f * (qx * qz - qy * qw);
      d[3] = 2.f * (qx * qy - qz * qw); d[4] = 1.f - 2.f * (qx * qx + qz * qz); d[5] = 2.f * (qy * qz + qx * qw);
      d[6] = 2.f * (qx * qz + qy * qw); d[7] = 2.f * (qy * qz - qx * qw); d[8] = 1.f - 2.f * (qx * qx + qy * qy);
      d[9] = __ldg(o + 0) - ref.x; d[10] = __ldg(o + 1) - ref.y; d[11] = __ldg(o + 2) - ref.z;
      d[12] = __ldg(o + 8); d[13] = __ldg(o + 9); d[14] = __ldg(o + 10); d[15] = 0.f;
    }
    r2max = warp_min(-r2max);  // max via min of negatives
    rmx = warp_min(-rmx);
    if (lane == 0) {
      atomicMax(&s_r2max_key, __float_as_int(-r2max));  // non-negative floats order as ints
      atomicMax(&s_rmax_key, __float_as_int(-rmx));
    }
    __syncthreads();
    // ---- work units (A blocks x B segments)
    const bool any_new = f < nt;
    const int B_lo = any_new ? off[f] : S;
    const int A_end = off[nt - 1];
    if (tid == 0) {
      int total = 0, nb = 0;
      if (any_new && A_end > 0) {
        nb = (A_end + BA - 1) / BA;
        for (int bk = 0; bk < nb; ++bk) {
          const int i0 = bk * BA, i1 = min(i0 + BA, A_end);
          const int lo = max(B_lo, off[oid[i0] + 1]);
          const int mend = max(lo, max(B_lo, off[oid[i1 - 1] + 1]));
          blk_lo[bk] = lo;
          blk_mend[bk] = mend;
          blk_pref[bk] = total;
          if (S > lo) total += (S - lo + K.seg_len - 1) / K.seg_len;
        }
      }
      blk_pref[nb] = total;
      s_total_units = total;
      s_nb = nb;
    }
    __syncthreads();
    const float r2m = __int_as_float(s_r2max_key);
    const float rmax = __int_as_float(s_rmax_key);
    const float eps = 1e-5f * (r2m + 0.01f);
    float m = kFarSentinel;
    // ---- sphere vs world box
    if (any_new && nobb > 0) {
      for (int i = B_lo + tid; i < S; i += nthr) {
        const float4 w = W[i];
        for (int k = 0; k < nobb; ++k) {
          const float* d = obbd + 16 * k;
          const float vx = w.x - d[9], vy = w.y - d[10], vz = w.z - d[11];
          // box frame: p = R^T v, i.e. p_k = (column k of R) . v
          const float px = d[0] * vx + d[1] * vy + d[2] * vz;
          const float py = d[3] * vx + d[4] * vy + d[5] * vz;
          const float pz = d[6] * vx + d[7] * vy + d[8] * vz;
          const float qx = fabsf(px) - d[12], qy = fabsf(py) - d[13], qz = fabsf(pz) - d[14];
          const float qm = fmaxf(qx, fmaxf(qy, qz));
          if (qm - w.w < m) {  // lower bound of the box distance
            const float ox = fmaxf(qx, 0.f), oy = fmaxf(qy, 0.f), oz = fmaxf(qz, 0.f);
            const float dist = sqrtf(ox * ox + oy * oy + oz * oz) + fminf(qm, 0.f) - w.w;
            m = fminf(m, dist);
          }
        }
        my_box += (unsigned long long)nobb;
      }
    }
    m = warp_min(m);
    if (lane == 0 && m < kFarSentinel) atomicMin(&s_best_key, float_key(m));
    // ---- sphere vs sphere
    const int total_units = s_total_units;
    const int nb = s_nb;
    for (;;) {
      int u = 0;
      if (lane == 0) u = atomicAdd(&s_unit_next, 1);
      u = __shfl_sync(0xFFFFFFFFu, u, 0);
      if (u >= total_units) break;
      const int bk = upper_index(blk_pref, nb + 1, u);
      const int seg = u - blk_pref[bk];
      const int i0 = bk * BA, i1 = min(i0 + BA, A_end);
      const int lo = blk_lo[bk], mend = blk_mend[bk];
      const int j0 = lo + seg * K.seg_len;
      const int j1 = min(j0 + K.seg_len, S);
      {  // CTA-wide best so far, broadcast so m stays warp-uniform
        int key = lane == 0 ? *(volatile int*)&s_best_key : 0;
        key = __shfl_sync(0xFFFFFFFFu, key, 0);
        m = fminf(m, key_float(key));
      }
      ABlock<APL> A;
#pragma unroll
      for (int s = 0; s < APL; ++s) {
        const int i = i0 + s * 32 + lane;
        const bool valid = i < i1;
        const float4 w = valid ? W[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        A.ax[s] = -2.f * w.x; A.ay[s] = -2.f * w.y; A.az[s] = -2.f * w.z;
        A.a2[s] = w.x * w.x + w.y * w.y + w.z * w.z;
        A.r[s] = w.w;
        A.bst[s] = valid ? max(B_lo, off[oid[i] + 1]) : INT_MAX;
      }
      bool alive = refresh<APL>(A, m, rmax, eps);
      if (!alive) continue;
#pragma unroll
      for (int s = 0; s < APL; ++s)
        if (A.act[s]) my_pairs += (unsigned long long)max(0, j1 - max(j0, A.bst[s]));
      const int jm = min(j1, mend);
      if (j0 < jm) sweep<APL, true>(A, W, beta, j0, jm, S, m, rmax, eps, &s_best_key, alive);
      if (alive && max(j0, mend) < j1) sweep<APL, false>(A, W, beta, max(j0, mend), j1, S, m, rmax, eps, &s_best_key, alive);
    }
    m = warp_min(m);
    if (lane == 0) s_warp_min[warp] = m;
    __syncthreads();
    if (tid == 0) {
      float mm = key_float(s_best_key);
      for (int w = 0; w < nwarps; ++w) mm = fminf(mm, s_warp_min[w]);
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

template <int APL, int MAXT>
cudaError_t launch_t(const KArgs& K, const sc_collide_config& cfg, size_t smem, int num_sms, cudaStream_t s) {
  auto kern = collide_kernel<APL, MAXT>;
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

}  // namespace

size_t collide_smem_bytes(const sc_scene_batch& b, const sc_collide_config& cfg) {
  return (size_t)make_layout(b.max_sph, b.max_obj, cfg.a_per_lane).total;
}

cudaError_t launch_collide(const sc_scene_batch& b, const CollideLaunch& a, const sc_collide_config& cfg, int num_sms,
                           cudaStream_t s, const char** why) {
  *why = nullptr;
  if (cfg.a_per_lane != 1 && cfg.a_per_lane != 2 && cfg.a_per_lane != 4) { *why = "a_per_lane must be 1, 2 or 4"; return cudaErrorInvalidValue; }
  const int maxt = cfg.a_per_lane == 4 ? 512 : 1024;
  if (cfg.threads < 128 || cfg.threads > maxt || cfg.threads % 32) { *why = "threads must be a multiple of 32 in 128..1024 (..512 when a_per_lane = 4)"; return cudaErrorInvalidValue; }
  if (cfg.seg_len < 8 || cfg.seg_len > 4096 || cfg.seg_len % 8) { *why = "seg_len must be a multiple of 8 in 8..4096"; return cudaErrorInvalidValue; }
  if (cfg.ctas_per_sm < 1 || cfg.ctas_per_sm > 8) { *why = "ctas_per_sm must be in 1..8"; return cudaErrorInvalidValue; }
  const size_t smem = collide_smem_bytes(b, cfg);
  if (smem > 227 * 1024) { *why = "batch needs more shared memory than one CTA has (max_sph too large)"; return cudaErrorInvalidValue; }
  cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  if (a.stats && (e = cudaMemsetAsync(a.stats, 0, 2 * sizeof(unsigned long long), s)) != cudaSuccess) return e;
  if (a.n_items <= 0) return cudaSuccess;
  KArgs K{b, a, cfg.seg_len};
  switch (cfg.a_per_lane) {
    case 1: return launch_t<1, 1024>(K, cfg, smem, num_sms, s);
    case 2: return launch_t<2, 1024>(K, cfg, smem, num_sms, s);
    default: return launch_t<4, 512>(K, cfg, smem, num_sms, s);
  }
}

}  // namespace sc
