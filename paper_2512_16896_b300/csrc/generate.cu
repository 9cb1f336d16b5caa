// Generation loop (Sec. IV-A and Fig. 2: per object, sample poses, check
// collisions, retry a limited number of times; Sec. IV-D: re-check only the
// scenes that retry; Sec. V-A: 10 retries per object, failing scenes invalid).
//
// One launch per (object k, try r) processes a device-resident list of the
// candidates that still need object k. Each warp of the persistent grid takes
// one candidate at a time (most tries are small: one object against the few
// placed before it, so a warp, not a CTA, is the unit of work): it samples
// object k (sample_core.cuh), stages object k's spheres in its own slice of
// shared memory and streams the spheres of objects 0..k-1 through registers
// (the A side of the prune test in collide_core.cuh, decide mode: it stops at
// the first certain collision). Lane 0 then appends the candidate to the list
// for object k+1 (or marks it valid after its last object), to the retry list
// for try r+1, or leaves it invalid after the last try.
#include <cstring>
#include <vector>

#include "collide_core.cuh"
#include "ik_core.cuh"
#include "kernels.h"
#include "sample_core.cuh"

namespace sc {

namespace {

using namespace core;

struct GenStepArgs {
  sc_scene_batch b;
  const unsigned long long* seed;  // device scalar, so a replayed graph takes a new seed
  int max_attempts, retry, max_retries, k, seg_len;
  const int32_t* list_in;
  const int* n_in;
  int32_t* list_retry;
  int* n_retry;
  int32_t* list_next;
  int* n_next;
  int32_t* list_reach;  // collision-free tries of reach-flagged objects (NULL: no reach stage)
  int* n_reach;
  float4* poses;
  uint8_t* valid;
  uint8_t* band;
  int32_t* tries;
  unsigned int* counter;
  unsigned long long* stats;
  int* status;
};

// Shared memory of one warp: objects 0..k (sphere offsets, poses, sin/cos of
// yaw) and the new object's spheres in the world frame (relative to object
// 0's position) with |c|^2 - r^2.
struct WarpLayout {
  int off, pose, sc, kobj, kpref, B, beta, bytes;
};

__host__ __device__ inline WarpLayout make_warp_layout(int max_obj) {
  WarpLayout W;
  W.off = 0;
  W.pose = align16(4 * (max_obj + 1));
  W.sc = align16(W.pose + 16 * max_obj);
  W.kobj = align16(W.sc + 8 * max_obj);
  W.kpref = align16(W.kobj + 4 * max_obj);
  W.B = align16(W.kpref + 4 * (max_obj + 1));
  W.beta = align16(W.B + 16 * (kMaxSphPerObj + kPad));
  W.bytes = align16(W.beta + 4 * (kMaxSphPerObj + kPad));
  return W;
}

// One warp per candidate: sample object k, then decide whether any sphere of
// object k is closer than the band to a sphere of objects 0..k-1 (A side,
// moved into registers 32*APL at a time) or to a world box.
// Broad phase (exact): every sphere of an object lies in the ball of radius
// |H| (its box's half-diagonal) around the object's frame origin, so two
// objects whose origins are farther apart than |H_j| + |H_k| + margin have no
// sphere pair within the band; only the other objects' spheres are streamed.
template <int APL>
__global__ void __launch_bounds__(256, 3) gen_warp_kernel(GenStepArgs g) {
  extern __shared__ __align__(16) unsigned char smem[];
  const sc_scene_batch& b = g.b;
  const WarpLayout WL = make_warp_layout(b.max_obj);
  const int lane = threadIdx.x & 31;
  unsigned char* base = smem + (size_t)(threadIdx.x >> 5) * WL.bytes;
  int* off = reinterpret_cast<int*>(base + WL.off);
  float4* opose = reinterpret_cast<float4*>(base + WL.pose);
  float2* osc = reinterpret_cast<float2*>(base + WL.sc);
  int* kobj = reinterpret_cast<int*>(base + WL.kobj);
  int* kpref = reinterpret_cast<int*>(base + WL.kpref);
  float4* Bs = reinterpret_cast<float4*>(base + WL.B);
  float* Bb = reinterpret_cast<float*>(base + WL.beta);
  const int n_items = *(volatile const int*)g.n_in;
  const int k = g.k;
  const uint64_t seed = *g.seed;
  unsigned long long my_pairs = 0, my_box = 0;

  for (;;) {
    int item = 0;
    if (lane == 0) item = (int)atomicAdd(g.counter, 1u);
    item = __shfl_sync(0xFFFFFFFFu, item, 0);
    if (item >= n_items) break;
    const int c = __ldg(&g.list_in[item]);
    const int t = template_of(b, c);
    int o0 = 0, nt = 0, s0 = 0, Sprev = 0, Sk = 0, nobb = 0, bx0 = 0;
    int64_t pbase = 0;
    if (t >= 0) {
      o0 = __ldg(&b.tmpl_obj_off[t]);
      nt = __ldg(&b.tmpl_obj_off[t + 1]) - o0;
      s0 = __ldg(&b.obj_sph_off[o0]);
      bx0 = __ldg(&b.tmpl_obb_off[t]);
      nobb = __ldg(&b.tmpl_obb_off[t + 1]) - bx0;
      pbase = __ldg(&b.tmpl_pose_off[t]) + (int64_t)(c - __ldg(&b.cand_tmpl_off[t])) * nt;
      if (k < nt) {
        Sprev = __ldg(&b.obj_sph_off[o0 + k]) - s0;
        Sk = __ldg(&b.obj_sph_off[o0 + k + 1]) - s0 - Sprev;
      }
    }
    const int err = t < 0 ? kDevBadTemplate
                    : (k >= nt || nt > b.max_obj || nt > kMaxObj) ? kDevTooManyObjects
                    : (Sk > kMaxSphPerObj || Sprev + Sk > b.max_sph) ? kDevTooManySpheres
                    : (nobb > kMaxObbPerTemplate) ? kDevTooManyBoxes : kDevOk;
    if (err != kDevOk) {
      if (lane == 0) {
        latch_error(g.status, err);
        if (t >= 0) g.band[c] = 1;
      }
      continue;
    }
    // ---- sample object k
    const Support sup = warp_support(b, t, lane);
    SampleResult r;
    r.placed = false;
    r.band = true;
    r.pose = make_float4(0.f, 0.f, 0.f, 0.f);
    if (sup.ok) {
      r = warp_sample_object(b, sup, seed, g.max_attempts, g.retry, c, k, o0, g.poses, pbase, g.status, lane);
    } else if (lane == 0) {
      latch_error(g.status, kDevBadPolygon);
    }
    if (lane == 0) g.poses[pbase + k] = r.pose;
    bool pass = false, bnd = r.band;
    if (r.placed) {
      // ---- objects 0..k
      for (int j = lane; j <= k; j += 32) {
        const float4 p = (j == k) ? r.pose : g.poses[pbase + j];
        float sn, cs;
        sincosf(p.w, &sn, &cs);
        opose[j] = p;
        osc[j] = make_float2(sn, cs);
        off[j] = __ldg(&b.obj_sph_off[o0 + j]) - s0;
      }
      __syncwarp();
      const float4 ref = opose[0];
      // ---- broad phase: earlier objects whose bounding balls come near object k's
      int nkeep = 0;
      {
        const float4 pk = opose[k];
        const float4 Hk = __ldg(reinterpret_cast<const float4*>(b.obj_half) + o0 + k);
        const float rk = sqrtf(Hk.x * Hk.x + Hk.y * Hk.y + Hk.z * Hk.z);
        for (int j0 = 0; j0 < k; j0 += 32) {
          const int j = j0 + lane;
          bool keep = false;
          int cnt = 0;
          if (j < k) {
            const float4 pj = opose[j];
            const float4 Hj = __ldg(reinterpret_cast<const float4*>(b.obj_half) + o0 + j);
            const float rj = sqrtf(Hj.x * Hj.x + Hj.y * Hj.y + Hj.z * Hj.z);
            const float dx = pj.x - pk.x, dy = pj.y - pk.y, dz = pj.z - pk.z;
            const float lim = rj + rk + kBroadMargin;
            keep = dx * dx + dy * dy + dz * dz <= lim * lim;
            cnt = off[j + 1] - off[j];
          }
          const unsigned mask = __ballot_sync(0xFFFFFFFFu, keep);
          // prefix of kept sphere counts within this chunk of 32 objects
          int pre = keep ? cnt : 0;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xFFFFFFFFu, pre, o);
            if (lane >= o) pre += v;
          }
          const int base_sph = nkeep == 0 ? 0 : kpref[nkeep];
          if (keep) {
            const int slot = nkeep + __popc(mask & ((1u << lane) - 1u));
            kobj[slot] = j;
            kpref[slot + 1] = base_sph + pre;
          }
          if (nkeep == 0 && lane == 0) kpref[0] = 0;
          nkeep += __popc(mask);
          __syncwarp();
        }
        if (lane == 0 && nkeep == 0) kpref[0] = 0;
        __syncwarp();
      }
      const int Skeep = kpref[nkeep];
      // ---- object k's spheres (B side)
      {
        const float4 p = opose[k];
        const float2 sc2 = osc[k];
        float r2 = 0.f;
        for (int q = lane; q < Sk + kPad; q += 32) {
          if (q < Sk) {
            const float4 l = __ldg(reinterpret_cast<const float4*>(b.sph_local) + s0 + Sprev + q);
            const float x = (p.x - ref.x) + (sc2.y * l.x - sc2.x * l.y);
            const float y = (p.y - ref.y) + (sc2.x * l.x + sc2.y * l.y);
            const float z = (p.z - ref.z) + l.z;
            const float c2 = x * x + y * y + z * z;
            Bs[q] = make_float4(x, y, z, l.w);
            Bb[q] = c2 - l.w * l.w;
            r2 = fmaxf(r2, c2);
          } else {
            Bs[q] = make_float4(1e6f, 1e6f, 1e6f, 0.f);
            Bb[q] = 3e12f;
          }
        }
        __syncwarp();
        float m = kFarSentinel;
        // ---- object k vs world boxes
        for (int bi = 0; bi < nobb; ++bi) {
          const float* o = b.obb + 12 * (bx0 + bi);
          float qx = __ldg(o + 4), qy = __ldg(o + 5), qz = __ldg(o + 6), qw = __ldg(o + 7);
          const float inv = rsqrtf(qx * qx + qy * qy + qz * qz + qw * qw);
          qx *= inv; qy *= inv; qz *= inv; qw *= inv;
          // columns of R (R maps box frame to world)
          const float c00 = 1.f - 2.f * (qy * qy + qz * qz), c01 = 2.f * (qx * qy + qz * qw), c02 = 2.f * (qx * qz - qy * qw);
          const float c10 = 2.f * (qx * qy - qz * qw), c11 = 1.f - 2.f * (qx * qx + qz * qz), c12 = 2.f * (qy * qz + qx * qw);
          const float c20 = 2.f * (qx * qz + qy * qw), c21 = 2.f * (qy * qz - qx * qw), c22 = 1.f - 2.f * (qx * qx + qy * qy);
          const float ox = __ldg(o + 0) - ref.x, oy = __ldg(o + 1) - ref.y, oz = __ldg(o + 2) - ref.z;
          const float hx = __ldg(o + 8), hy = __ldg(o + 9), hz = __ldg(o + 10);
          for (int q = lane; q < Sk; q += 32) {
            const float4 w = Bs[q];
            const float vx = w.x - ox, vy = w.y - oy, vz = w.z - oz;
            const float px = c00 * vx + c01 * vy + c02 * vz;
            const float py = c10 * vx + c11 * vy + c12 * vz;
            const float pz = c20 * vx + c21 * vy + c22 * vz;
            const float ex = fabsf(px) - hx, ey = fabsf(py) - hy, ez = fabsf(pz) - hz;
            const float em = fmaxf(ex, fmaxf(ey, ez));
            if (em - w.w < kBand) {
              const float ux = fmaxf(ex, 0.f), uy = fmaxf(ey, 0.f), uz = fmaxf(ez, 0.f);
              m = fminf(m, sqrtf(ux * ux + uy * uy + uz * uz) + fminf(em, 0.f) - w.w);
            }
          }
        }
        my_box += (unsigned long long)nobb * (unsigned long long)(lane < Sk ? (Sk - lane + 31) / 32 : 0);
        m = warp_min(m);
        bool alive = !(m < -kBand);
        r2 = -warp_min(-r2);
        // ---- object k vs the kept earlier objects (A side in registers)
        for (int i0 = 0; alive && i0 < Skeep; i0 += 32 * APL) {
          ABlock<APL> A;
          float a2max = 0.f;
          int nval = 0;
#pragma unroll
          for (int s = 0; s < APL; ++s) {
            const int qq = i0 + s * 32 + lane;
            const bool valid = qq < Skeep;
            float x = 0.f, y = 0.f, z = 0.f, rr = 0.f;
            if (valid) {
              const int jj = upper_index(kpref, nkeep + 1, qq);
              const int j = kobj[jj];
              const int q = off[j] + (qq - kpref[jj]);
              const float4 l = __ldg(reinterpret_cast<const float4*>(b.sph_local) + s0 + q);
              const float4 p = opose[j];
              const float2 sc2 = osc[j];
              x = (p.x - ref.x) + (sc2.y * l.x - sc2.x * l.y);
              y = (p.y - ref.y) + (sc2.x * l.x + sc2.y * l.y);
              z = (p.z - ref.z) + l.z;
              rr = l.w;
              ++nval;
            }
            A.ax[s] = -2.f * x; A.ay[s] = -2.f * y; A.az[s] = -2.f * z;
            A.a2[s] = x * x + y * y + z * z;
            A.r[s] = rr;
            A.bst[s] = valid ? 0 : INT_MAX;
            a2max = fmaxf(a2max, A.a2[s]);
          }
          const float eps = 1e-5f * (fmaxf(r2, -warp_min(-a2max)) + 0.01f);
          refresh<APL, true>(A, 0.f, 0.f, eps);
          my_pairs += (unsigned long long)nval * (unsigned long long)Sk;
          sweep<APL, false, true>(A, Bs, Bb, 0, Sk, Sk, m, 0.f, eps, nullptr, nullptr, alive);
        }
        pass = alive && !(m < 0.f);
        bnd = bnd || fabsf(m) <= kBand;
      }
    }
    if (lane == 0) {
      if (bnd) g.band[c] = 1;
      g.tries[c] += 1;
      if (pass) {
        if (g.list_reach && (__ldg(&b.obj_rel[o0 + k]) & SC_REL_REACH)) g.list_reach[atomicAdd(g.n_reach, 1)] = c;
        else if (k + 1 == nt) g.valid[c] = 1;
        else g.list_next[atomicAdd(g.n_next, 1)] = c;
      } else if (g.retry < g.max_retries) {
        g.list_retry[atomicAdd(g.n_retry, 1)] = c;
      }
    }
    __syncwarp();  // the warp's shared memory is reused by its next candidate
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

// ---- reachability stage (Sec. IV-E): the collision-free tries of
// reach-flagged objects, in the reach list, get a top-down grasp target in
// the robot base frame; an optional learned gate sends the ones it predicts
// unreachable back to retry; exact IK decides the rest.
struct ReachArgs {
  sc_scene_batch b;
  int k, retry, max_retries, gated;
  float tol_pos, tol_rot, tau;
  const int32_t* list_reach;
  const int* n_reach;
  float* targets;        // [cap][12]
  const float* logits;   // [cap]
  int32_t* list_ik;      // positions in the reach list the gate passed
  int* n_ik;
  int32_t* list_retry;
  int* n_retry;
  int32_t* list_next;
  int* n_next;
  const float4* poses;
  uint8_t* valid;
  uint8_t* band;
  float* q_reach;        // [P][7] or NULL
  unsigned long long* stats;
  ikc::IkArgs ik;
};

// Top-down grasp of object k: position = top centre of its box, tool z =
// -world z, tool x along the object's yaw; expressed in the template's robot
// base frame (x, y, z, yaw). R row-major, then p.
__global__ void reach_targets_kernel(ReachArgs A) {
  const int n = *(volatile const int*)A.n_reach;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int c = A.list_reach[i];
    const int t = template_of(A.b, c);
    const int o0 = __ldg(&A.b.tmpl_obj_off[t]), nt = __ldg(&A.b.tmpl_obj_off[t + 1]) - o0;
    const int64_t pbase = __ldg(&A.b.tmpl_pose_off[t]) + (int64_t)(c - __ldg(&A.b.cand_tmpl_off[t])) * nt;
    const float4 p = A.poses[pbase + A.k];
    const float hz = __ldg(&A.b.obj_half[4 * (o0 + A.k) + 2]);
    const float4 base = __ldg(reinterpret_cast<const float4*>(A.b.tmpl_base) + t);
    float sb, cb, sp, cp;
    sincosf(base.w, &sb, &cb);
    sincosf(p.w - base.w, &sp, &cp);
    const float wx = p.x - base.x, wy = p.y - base.y, wz = p.z + hz - base.z;
    float* o = A.targets + 12 * (size_t)i;
    o[0] = cp; o[1] = sp; o[2] = 0.f;
    o[3] = sp; o[4] = -cp; o[5] = 0.f;
    o[6] = 0.f; o[7] = 0.f; o[8] = -1.f;
    o[9] = cb * wx + sb * wy;
    o[10] = -sb * wx + cb * wy;
    o[11] = wz;
  }
}

// Gate: logit >= tau goes on to IK, the rest retries (or ends invalid).
__global__ void gate_split_kernel(ReachArgs A) {
  const int n = *(volatile const int*)A.n_reach;
  unsigned long long rejected = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (A.logits[i] >= A.tau) {
      A.list_ik[atomicAdd(A.n_ik, 1)] = i;
    } else {
      ++rejected;
      if (A.retry < A.max_retries) A.list_retry[atomicAdd(A.n_retry, 1)] = A.list_reach[i];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) rejected += __shfl_xor_sync(0xFFFFFFFFu, rejected, o);
  if ((threadIdx.x & 31) == 0 && rejected) atomicAdd(&A.stats[3], rejected);
}

// Exact IK, one warp per entry; seeds keyed by (candidate, object, try).
__global__ void __launch_bounds__(128) reach_ik_kernel(ReachArgs A) {
  const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
  const int n = A.gated ? *(volatile const int*)A.n_ik : *(volatile const int*)A.n_reach;
  unsigned long long solves = 0, seed_iters = 0;
  for (int j = blockIdx.x * warps + (threadIdx.x >> 5); j < n; j += gridDim.x * warps) {
    const int i = A.gated ? A.list_ik[j] : j;
    const int c = A.list_reach[i];
    const ikc::Target T = ikc::load_target(A.targets + 12 * (size_t)i);
    float q[7], pe2, sr, cr;
    const ikc::Solve r = ikc::warp_solve(A.ik, T, (uint32_t)c, ((uint32_t)A.k << 16) | (uint32_t)A.retry, lane, q, pe2,
                                         sr, cr);
    ++solves;
    seed_iters += (unsigned long long)(r.it + 1) * (unsigned long long)A.ik.seeds;
    if (lane == r.winner) {
      const int t = template_of(A.b, c);
      const int o0 = __ldg(&A.b.tmpl_obj_off[t]), nt = __ldg(&A.b.tmpl_obj_off[t + 1]) - o0;
      const int64_t pbase = __ldg(&A.b.tmpl_pose_off[t]) + (int64_t)(c - __ldg(&A.b.cand_tmpl_off[t])) * nt;
      const float pe = sqrtf(pe2), ang = atan2f(sr, cr);
      if (fabsf(pe - A.tol_pos) <= kBand || fabsf(ang - A.tol_rot) <= kBand) A.band[c] = 1;
      if (r.found) {
        if (A.q_reach) {
#pragma unroll
          for (int jq = 0; jq < 7; ++jq) A.q_reach[7 * (pbase + A.k) + jq] = q[jq];
        }
        if (A.k + 1 == nt) A.valid[c] = 1;
        else A.list_next[atomicAdd(A.n_next, 1)] = c;
      } else if (A.retry < A.max_retries) {
        A.list_retry[atomicAdd(A.n_retry, 1)] = c;
      }
    }
  }
  if (lane == 0 && solves) {
    atomicAdd(&A.stats[2], solves);
    atomicAdd(&A.stats[4], seed_iters);
  }
}

// 1 + the largest template-local index of an object carrying the reach flag.
__global__ void reach_extent_kernel(sc_scene_batch b, int* out) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < b.n_templates; t += gridDim.x * blockDim.x) {
    const int o0 = b.tmpl_obj_off[t], o1 = b.tmpl_obj_off[t + 1];
    int ext = 0;
    for (int o = o0; o < o1; ++o)
      if (b.obj_rel[o] & SC_REL_REACH) ext = o - o0 + 1;
    if (ext) atomicMax(out, ext);
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
  if (blockIdx.x == 0 && threadIdx.x < 5 && stats) stats[threadIdx.x] = 0;
}

template <int APL>
cudaError_t prepare_step_kernel(size_t smem, int threads, int ctas_per_sm, int num_sms, int* grid) {
  auto kern = gen_warp_kernel<APL>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  *grid = num_sms * (ctas_per_sm < per_sm ? ctas_per_sm : per_sm);
  return cudaSuccess;
}

template <int APL>
void launch_step(const GenStepArgs& g, int grid, int threads, size_t smem, cudaStream_t s) {
  gen_warp_kernel<APL><<<grid, threads, smem, s>>>(g);
}

}  // namespace

cudaError_t reach_extent(const sc_scene_batch& b, int* scratch_int, int* out_host, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(scratch_int, 0, sizeof(int), s);
  if (e) return e;
  reach_extent_kernel<<<64, 256, 0, s>>>(b, scratch_int);
  if ((e = cudaGetLastError())) return e;
  if ((e = cudaMemcpyAsync(out_host, scratch_int, sizeof(int), cudaMemcpyDeviceToHost, s))) return e;
  return cudaStreamSynchronize(s);
}

// Scratch: 6 int32 lists of n (next x2, retry x2, reach, gate-passed), the
// grasp targets (12 floats) and logits of the reach list, counts
// [K+1] + 3 x [K][R+1], work counters [K][R+1], then the seed scalar.
size_t generate_seed_offset(int n_cand, int max_obj, int max_retries) {
  const size_t n = (size_t)n_cand;
  const size_t lists = 6 * n * sizeof(int32_t) + 13 * n * sizeof(float);
  const size_t counts = (size_t)(max_obj + 1) + 3 * (size_t)max_obj * (max_retries + 1);
  const size_t counters = (size_t)max_obj * (max_retries + 1);
  const size_t body = lists + (counts + counters) * sizeof(int);
  return (body + 255) & ~size_t(255);  // the 8-byte seed sits on a 256-byte boundary
}

size_t generate_scratch_bytes(int n_cand, int max_obj, int max_retries) {
  return generate_seed_offset(n_cand, max_obj, max_retries) + 256;
}

cudaError_t enqueue_generate(const sc_scene_batch& b, const GenerateLaunch& a, const sc_collide_config& cfg,
                             int num_sms, cudaStream_t s, const char** why) {
  *why = check_collide_config(cfg);
  if (*why) return cudaErrorInvalidValue;
  if (cfg.threads > 512) { *why = "generation uses at most 512 threads per CTA"; return cudaErrorInvalidValue; }
  const size_t smem = (size_t)(cfg.threads / 32) * make_warp_layout(b.max_obj).bytes;
  if (smem > 227 * 1024) { *why = "threads x per-warp shared memory exceeds one CTA's (lower threads)"; return cudaErrorInvalidValue; }
  const int n = a.n_items;
  const int K = b.max_obj, R = a.max_retries;
  // scratch carve-up: 4 lists of n ints, counts[K+1] (list sizes per object),
  // retry counts[K][R+1], work counters[K][R+1]
  int32_t* ib = static_cast<int32_t*>(a.scratch);
  int32_t* L[2] = {ib, ib + n};
  int32_t* Rl[2] = {ib + 2 * (size_t)n, ib + 3 * (size_t)n};
  int32_t* list_reach = ib + 4 * (size_t)n;
  int32_t* list_ik = ib + 5 * (size_t)n;
  float* targets = reinterpret_cast<float*>(ib + 6 * (size_t)n);
  float* logits = targets + 12 * (size_t)n;
  int* counts = reinterpret_cast<int*>(logits + n);
  const int n_counts = (K + 1) + 3 * K * (R + 1);
  int* cnt_list = counts;
  int* cnt_retry = counts + (K + 1);
  int* cnt_reach = cnt_retry + K * (R + 1);
  int* cnt_ik = cnt_reach + K * (R + 1);
  unsigned int* counters = reinterpret_cast<unsigned int*>(counts + n_counts);
  const int n_counters = K * (R + 1);
  const unsigned long long* seed_dev = a.seed_dev;

  int grid = 0;
  cudaError_t e;
  switch (cfg.a_per_lane) {
    case 1: e = prepare_step_kernel<1>(smem, cfg.threads, cfg.ctas_per_sm, num_sms, &grid); break;
    case 2: e = prepare_step_kernel<2>(smem, cfg.threads, cfg.ctas_per_sm, num_sms, &grid); break;
    default: e = prepare_step_kernel<4>(smem, cfg.threads, cfg.ctas_per_sm, num_sms, &grid); break;
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
  g.seed = seed_dev;
  g.max_attempts = a.max_attempts;
  g.max_retries = R;
  g.seg_len = cfg.seg_len;
  g.poses = reinterpret_cast<float4*>(a.poses);
  g.valid = a.valid;
  g.band = a.band;
  g.tries = a.tries;
  g.stats = a.stats;
  g.status = a.status;
  ReachArgs ra;
  std::memset(&ra, 0, sizeof(ra));
  const bool reach = a.arm != nullptr;
  if (reach) {
    ra.b = b;
    ra.max_retries = R;
    ra.gated = a.gate != nullptr;
    ra.tol_pos = a.ik->tol_pos;
    ra.tol_rot = a.ik->tol_rot;
    ra.tau = a.tau;
    ra.list_reach = list_reach;
    ra.targets = targets;
    ra.logits = logits;
    ra.list_ik = list_ik;
    ra.poses = reinterpret_cast<const float4*>(a.poses);
    ra.valid = a.valid;
    ra.band = a.band;
    ra.q_reach = a.q_reach;
    ra.stats = a.stats;
    ikc::fill_params(ra.ik, *a.arm, *a.ik);
  }
  int small_blocks = (n + 255) / 256;
  small_blocks = small_blocks < num_sms * 4 ? small_blocks : num_sms * 4;
  if (small_blocks < 1) small_blocks = 1;
  for (int k = 0; k < K; ++k) {
    g.k = k;
    g.list_next = L[(k + 1) & 1];
    g.n_next = cnt_list + k + 1;
    const bool reach_k = reach && k < a.reach_objects;
    for (int r = 0; r <= R; ++r) {
      g.retry = r;
      g.list_in = r == 0 ? L[k & 1] : Rl[(r - 1) & 1];
      g.n_in = r == 0 ? cnt_list + k : cnt_retry + k * (R + 1) + (r - 1);
      g.list_retry = Rl[r & 1];
      g.n_retry = cnt_retry + k * (R + 1) + r;
      g.counter = counters + k * (R + 1) + r;
      g.list_reach = reach_k ? list_reach : nullptr;
      g.n_reach = reach_k ? cnt_reach + k * (R + 1) + r : nullptr;
      if (a.timer) a.timer->begin(0, s);
      switch (cfg.a_per_lane) {
        case 1: launch_step<1>(g, grid, cfg.threads, smem, s); break;
        case 2: launch_step<2>(g, grid, cfg.threads, smem, s); break;
        default: launch_step<4>(g, grid, cfg.threads, smem, s); break;
      }
      if (a.timer) a.timer->end(s);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if (!reach_k) continue;
      ra.k = k;
      ra.retry = r;
      ra.n_reach = g.n_reach;
      ra.n_ik = cnt_ik + k * (R + 1) + r;
      ra.list_retry = g.list_retry;
      ra.n_retry = g.n_retry;
      ra.list_next = g.list_next;
      ra.n_next = g.n_next;
      if (a.timer) a.timer->begin(1, s);
      reach_targets_kernel<<<small_blocks, 256, 0, s>>>(ra);
      if (ra.gated) {
        e = mlp_infer_counted(a.gate, targets, ra.n_reach, n, logits, a.status, num_sms, s);
        if (e != cudaSuccess) return e;
        gate_split_kernel<<<small_blocks, 256, 0, s>>>(ra);
      }
      if (a.timer) {
        a.timer->end(s);
        a.timer->begin(2, s);
      }
      reach_ik_kernel<<<num_sms * 8, 128, 0, s>>>(ra);
      if (a.timer) a.timer->end(s);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace sc
