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
#include "mlp_tc_core.cuh"
#include "sample_core.cuh"
#include "tri_core.cuh"

namespace sc {

namespace {

using namespace core;

// Per-template constants gathered once per generation call (one 64-byte
// record, read with four vector loads instead of a chain of CSR lookups).
struct TmplInfo {
  int o0, nt, s0, bx0;           // first object, objects, first sphere, first world box
  int nobb, v0, nv, cand0;       // world boxes, first polygon vertex, vertices, first candidate
  long long pose0;               // first pose row
  float z, pad;                  // support height
  float xmin, xmax, ymin, ymax;  // support polygon bounding box
};
static_assert(sizeof(TmplInfo) == 64, "TmplInfo is four 16-byte loads");

// Per-candidate progress of the rounds (objects with reachability): the
// object a candidate is on and the try it makes next. A candidate sits in
// exactly one list at a time, so only one kernel touches its state.
struct CandState {
  uint8_t* kc;     // [n_cand] current object
  uint16_t* rc;    // [n_cand] next try of that object
  uint8_t* alive;  // [n_cand] 1: starts the chained launch at object k_begin
  int k_begin;     // objects [0, k_begin) run in rounds
};

struct GenStepArgs {
  sc_scene_batch b;
  const int32_t* cand_t;    // [n_cand] template of each candidate (-1: none)
  const TmplInfo* tinfo;    // [n_templates]
  const float* edge_inv;    // [n_verts] 1 / squared length of the edge ending at each vertex
  const float4* obb_tab;    // [n_obb][4] (R row 0 | cx), (R row 1 | cy), (R row 2 | cz), (hx, hy, hz, 0)
  const float4* tri_chunk;  // [tri_chunk_slots] bounding ball (centre, radius) of 32 triangles (world frame)
  const unsigned long long* seed;  // device scalar, so a replayed graph takes a new seed
  int max_attempts, max_retries, seg_len;
  // reach bounds: a grasp target (t*, R*) fails the exact IK with no check in
  // its band when t* lies farther than sqrt(reach_r2) from the shoulder
  // (0, 0, reach_z0) of the arm's base frame, or when its wrist point
  // t* - R* reach_v lies farther than sqrt(reach_w2) from it; such a try fails
  // right after sampling (its collisions are not decided, its outcome does not
  // depend on them) and is retried in the next round (reach_r2 < 0: none)
  float reach_r2, reach_w2, reach_z0;
  float3 reach_v;
  int max_sk;  // most spheres of one object in the batch (sizes the per-warp B area)
  CandState st;
  const int32_t* list_in;  // this round's candidates
  const int* n_in;
  int32_t* list_gen;       // the next round's candidates (retry, or the next object)
  int* n_gen;
  int32_t* list_reach;     // collision-free tries of reach-flagged objects (NULL: no reach stage)
  float* targets;          // [cap][12] their grasp targets, by position in list_reach
  int* n_reach;
  float4* poses;
  uint8_t* valid;
  uint8_t* band;
  int32_t* tries;
  unsigned int* counter;
  unsigned long long* stats;
  int* status;
};

// Shared memory of one warp: the candidate's objects (absolute sphere
// offsets, poses, sin/cos of yaw, bounding-ball radii), the kept objects of
// the current try, the new object's spheres in the world frame (relative to
// object 0's position) with |c|^2 - r^2, and the A staging area.
struct WarpLayout {
  int tmpl, off, pose, sc, rad, kobj, kball, B, beta, astage, bytes;
};

// max_sk: most spheres of one object in the batch (B side); apl: A spheres
// per lane of the register block (A staging holds one block plus 64).
__host__ __device__ inline WarpLayout make_warp_layout(int max_obj, int max_sk, int apl) {
  WarpLayout W;
  W.tmpl = 0;
  W.off = 64;
  W.pose = align16(W.off + 4 * (max_obj + 1));
  W.sc = align16(W.pose + 16 * max_obj);
  W.rad = align16(W.sc + 8 * max_obj);
  W.kobj = align16(W.rad + 4 * max_obj);
  W.kball = align16(W.kobj + 4 * max_obj);
  W.B = align16(W.kball + 16 * max_obj);
  W.beta = align16(W.B + 16 * (max_sk + kPad));
  W.astage = align16(W.beta + 4 * (max_sk + kPad));
  W.bytes = align16(W.astage + 16 * (32 * apl + 64));
  return W;
}

struct WarpState {
  TmplInfo* tmpl; // the current candidate's template record
  int* off;       // [max_obj + 1] absolute sphere offsets of the candidate's objects
  float4* opose;  // [max_obj] poses of objects 0..k
  float2* osc;    // [max_obj] sin, cos of their yaw
  float* orad;    // [max_obj] bounding-ball radii |H|
  int* kobj;      // kept objects of the current try
  float4* kball;  // their balls (centre relative to object 0, radius)
  float4* Bs;     // object k's spheres
  float* Bb;      // |b|^2 - r^2
  float4* astage; // A survivors
};

__device__ __forceinline__ WarpState warp_state(unsigned char* smem, const WarpLayout& WL) {
  unsigned char* base = smem + (size_t)(threadIdx.x >> 5) * WL.bytes;
  WarpState W;
  W.tmpl = reinterpret_cast<TmplInfo*>(base + WL.tmpl);
  W.off = reinterpret_cast<int*>(base + WL.off);
  W.opose = reinterpret_cast<float4*>(base + WL.pose);
  W.osc = reinterpret_cast<float2*>(base + WL.sc);
  W.orad = reinterpret_cast<float*>(base + WL.rad);
  W.kobj = reinterpret_cast<int*>(base + WL.kobj);
  W.kball = reinterpret_cast<float4*>(base + WL.kball);
  W.Bs = reinterpret_cast<float4*>(base + WL.B);
  W.Bb = reinterpret_cast<float*>(base + WL.beta);
  W.astage = reinterpret_cast<float4*>(base + WL.astage);
  return W;
}

// Copies template t's record into the warp's slot (t < 0: a zeroed record).
__device__ __forceinline__ const TmplInfo& load_tmpl(const TmplInfo* tinfo, int t, TmplInfo* slot, int lane) {
  if (lane < 4) {
    int4 v = make_int4(0, 0, 0, 0);
    if (t >= 0) v = __ldg(reinterpret_cast<const int4*>(tinfo + t) + lane);
    reinterpret_cast<int4*>(slot)[lane] = v;
  }
  __syncwarp();
  return *slot;
}

// Asynchronous global -> shared copies (completed by cp_async_wait_all).
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Decides the staged A spheres [0, fill) (slot s * 32 + lane of the register
// block) against the B spheres [0, Sc) in shared memory (decide mode, fixed
// tolerance eps).
template <int APL>
__device__ __forceinline__ void sweep_block(const float4* astage, int fill, const float4* Bs, const float* Bb, int Sc,
                                            float eps, int lane, float& m, bool& alive) {
  ABlock<APL> A;
#pragma unroll
  for (int s = 0; s < APL; ++s) {
    const bool valid = s * 32 + lane < fill;
    const float4 w = valid ? astage[s * 32 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    A.ax[s] = -2.f * w.x; A.ay[s] = -2.f * w.y; A.az[s] = -2.f * w.z;
    A.a2[s] = w.x * w.x + w.y * w.y + w.z * w.z;
    A.r[s] = w.w;
    A.bst[s] = valid ? 0 : INT_MAX;
  }
  refresh<APL, true>(A, 0.f, 0.f, eps);
  sweep<APL, false, true>(A, Bs, Bb, 0, Sc, Sc, m, 0.f, eps, nullptr, nullptr, alive);
}

// Work counted by lane 0 of a warp.
struct TryCounters {
  unsigned long long pairs = 0, box = 0, cull = 0, exh = 0, tri = 0, far = 0;
};

struct TryOut {
  bool pass;  // placed and collision-free
  bool band;  // a decision of the try lay within the band
};

// Object k (position pk, yaw sine/cosine skn/kcs, ball radius rk, spheres
// [sph0, sph0 + Sk) of the batch) against the world triangles of template t,
// coordinates relative to ref, in three exact culls: chunks of 32 triangles
// whose bounding balls (chunks, world frame) come within the band of object
// k's ball; their triangles within the band of the ball (distance minus its
// radius); each kept triangle's exact distance to every sphere of object k.
// kBroadMargin absorbs FP32 rounding at both cull levels. Chunk tests count
// as ball cull tests (cull_cnt), point-triangle distances in tri_cnt.
// Returns this lane's minimum.
__device__ __forceinline__ float world_tri_min(const sc_scene_batch& b, const float4* chunks, int t, float4 pk,
                                                float4 ref, float rk, float skn, float kcs, int sph0, int Sk,
                                                int lane, unsigned long long& tri_cnt,
                                                unsigned long long& cull_cnt) {
  float m = kFarSentinel;
  const int tq0 = __ldg(&b.tmpl_tri_off[t]), ntri = __ldg(&b.tmpl_tri_off[t + 1]) - tq0;
  const int nch = (ntri + 31) >> 5;
  const float3 r3 = make_float3(ref.x, ref.y, ref.z);
  const float3 ck = make_float3(pk.x - ref.x, pk.y - ref.y, pk.z - ref.z);
  const float3 cw = make_float3(pk.x, pk.y, pk.z);
#pragma unroll 1
  for (int c0 = 0; c0 < nch; c0 += 32) {
    // chunk level: lanes take chunks; a chunk whose ball is farther from
    // object k's ball than the band holds no triangle that matters
    bool chunk_near = false;
    if (c0 + lane < nch) {
      const float4 cb = __ldg(&chunks[tri_chunk_slot(tq0, t, c0 + lane)]);
      const float dx = cw.x - cb.x, dy = cw.y - cb.y, dz = cw.z - cb.z;
      const float lim = cb.w + rk + kBand + kBroadMargin;
      chunk_near = dx * dx + dy * dy + dz * dz <= lim * lim;
    }
    if (lane == 0) cull_cnt += (unsigned long long)min(32, nch - c0);
    unsigned cmask = __ballot_sync(0xFFFFFFFFu, chunk_near);
#pragma unroll 1
    while (cmask) {
      const int j0 = (c0 + __ffs(cmask) - 1) * 32;
      cmask &= cmask - 1;
      // triangle level: lanes take the chunk's triangles
      bool near = false;
      if (j0 + lane < ntri)
        near = sqrtf(point_tri_d2(ck, load_tri(b.tri, tq0 + j0 + lane, r3))) - rk < kBand + kBroadMargin;
      if (lane == 0) tri_cnt += (unsigned long long)min(32, ntri - j0);
      unsigned mask = __ballot_sync(0xFFFFFFFFu, near);
#pragma unroll 1
      while (mask) {
        const Tri Tj = load_tri(b.tri, tq0 + j0 + __ffs(mask) - 1, r3);
        mask &= mask - 1;
#pragma unroll 1
        for (int q = lane; q < Sk; q += 32) {
          const float4 l = __ldg(reinterpret_cast<const float4*>(b.sph_local) + sph0 + q);
          const float3 w = make_float3((pk.x - ref.x) + (kcs * l.x - skn * l.y),
                                       (pk.y - ref.y) + (skn * l.x + kcs * l.y), (pk.z - ref.z) + l.z);
          m = fminf(m, sqrtf(point_tri_d2(w, Tj)) - l.w);
        }
        if (lane == 0) tri_cnt += (unsigned long long)Sk;
      }
    }
  }
  return m;
}

// One try (Sec. IV-A, Fig. 2) of template-local object k of candidate c:
// sample its pose (the pose is written to poses[pbase + k] whatever the
// outcome), then decide it against the kept earlier objects, the world
// boxes and (relation-enabled instances) the world triangles. On entry the
// warp state holds objects 0..k-1 (opose, osc, orad,
// off[0..k]); with PREFETCHED, their poses, half extents (in kball) and
// offsets are cp.async copies still in flight, completed here after the
// sampling, and osc / orad are derived from them. On return, when the pose
// was accepted, opose[k], osc[k] and orad[k] hold object k.
// Broad phase (exact): every sphere of an object lies in the ball of radius
// |H| (its box's half-diagonal) around the object's frame origin, so two
// objects whose origins are farther apart than |H_j| + |H_k| + margin have no
// sphere pair within the band. Sphere-level cull (exact, same argument): a B
// sphere farther than band + margin from every kept object's ball, or an A
// sphere that far from object k's ball, has no pair within the band.
// MODE 0: free / on-top / next-to objects only; 1: the full relation set;
// 2: the full relation set with articulated parts and world triangles.
template <int APL, bool PREFETCHED, int MODE>
__device__ __forceinline__ TryOut gen_try(const GenStepArgs& g, const TmplInfo& T, const WarpState& W, int t, int c, int k,
                                          int retry, int rel, int Sprev, int Sk, int64_t pbase, uint64_t seed,
                                          const float4* ref_poses, int lane, TryCounters& cnt) {
  constexpr bool EXT = MODE >= 1, WORLD = MODE == 2;
  const sc_scene_batch& b = g.b;
  const int o0 = T.o0, s0 = T.s0, nobb = T.nobb, bx0 = T.bx0;
  // ---- sample object k
  Support sup;
  sup.P.v = reinterpret_cast<const float2*>(b.poly_verts) + T.v0;
  sup.P.n = T.nv;
  sup.P.inv = g.edge_inv + T.v0;
  sup.ok = T.nv >= 3 && T.nv <= kMaxPolyVerts;
  sup.z = T.z;
  sup.xmin = T.xmin; sup.xmax = T.xmax; sup.ymin = T.ymin; sup.ymax = T.ymax;
  const ObjectSpec spec = load_object_spec<EXT>(b, o0, k, rel, ref_poses, 0, g.status, lane, t, c);
  SampleResult r;
  r.placed = false;
  r.band = true;
  r.pose = make_float4(0.f, 0.f, 0.f, 0.f);
  if (sup.ok) {
    r = warp_sample_spec<EXT>(sup, spec, seed, g.max_attempts, retry, c, k, lane, b.obj_anchor, ref_poses);
  } else if (lane == 0) {
    latch_error(g.status, kDevBadPolygon);
  }
  if (lane == 0) g.poses[pbase + k] = r.pose;
  if (PREFETCHED) {
    cp_async_wait_all();
    __syncwarp();
#pragma unroll 1
    for (int j = lane; j < k; j += 32) {
      const float4 p = W.opose[j], H = W.kball[j];
      float sn, cs;
      sincos_cw(p.w, &sn, &cs);
      W.osc[j] = make_float2(sn, cs);
      W.orad[j] = sqrtf(H.x * H.x + H.y * H.y + H.z * H.z);
    }
  }
  TryOut out;
  out.pass = false;
  out.band = r.band;
  if (!r.placed) return out;
  const float4 pk = r.pose;
  if (PREFETCHED && g.list_reach && (rel & SC_REL_REACH) && g.reach_r2 >= 0.f) {
    // the reach bounds: the grasp target of this pose no configuration
    // reaches, so the try fails whatever its collisions (which are then not
    // decided); the grasp target as grasp_target_at forms it: position in the
    // base frame, tool rotation rows (cp, sp, 0), (sp, -cp, 0), (0, 0, -1)
    const float4 base = __ldg(reinterpret_cast<const float4*>(b.tmpl_base) + t);
    const float wx = pk.x - base.x, wy = pk.y - base.y;
    const float wz = pk.z + __ldg(&b.obj_half[4 * (o0 + k) + 2]) - base.z - g.reach_z0;
    float sb, cb, sp, cp;
    sincos_cw(base.w, &sb, &cb);  // within 1.5 ulp of the sincosf values the target is formed from
    sincos_cw(pk.w - base.w, &sp, &cp);
    const float tx = cb * wx + sb * wy, ty = -sb * wx + cb * wy;
    const float3 v = g.reach_v;
    const float ux = tx - (cp * v.x + sp * v.y), uy = ty - (sp * v.x - cp * v.y), uz = wz + v.z;
    if (tx * tx + ty * ty + wz * wz > g.reach_r2 || ux * ux + uy * uy + uz * uz > g.reach_w2) {
      cnt.far += lane == 0;
      return out;
    }
  }
  const float rk = sqrtf(spec.H.x * spec.H.x + spec.H.y * spec.H.y + spec.H.z * spec.H.z);
  float skn, kcs;
  sincos_cw(pk.w, &skn, &kcs);
  if (lane == 0) {
    W.opose[k] = pk;
    W.osc[k] = make_float2(skn, kcs);
    W.orad[k] = rk;
  }
  __syncwarp();
  const float4 ref = k == 0 ? pk : W.opose[0];
  // ---- broad phase: earlier objects whose bounding balls come near object
  // k's; the kept ones' balls (relative to ref) go to kball
  int nkeep = 0;
  float a_bound = 0.f;  // bound on |a| over the kept objects' spheres
#pragma unroll 1
  for (int j0 = 0; j0 < k; j0 += 32) {
    const int j = j0 + lane;
    bool keep = false;
    float4 ball = make_float4(0.f, 0.f, 0.f, 0.f);
    if (j < k) {
      const float4 pj = W.opose[j];
      const float rj = W.orad[j];
      const float dx = pj.x - pk.x, dy = pj.y - pk.y, dz = pj.z - pk.z;
      const float lim = rj + rk + kBroadMargin;
      keep = dx * dx + dy * dy + dz * dz <= lim * lim;
      ball = make_float4(pj.x - ref.x, pj.y - ref.y, pj.z - ref.z, rj);
      if (keep) a_bound = fmaxf(a_bound, sqrtf(ball.x * ball.x + ball.y * ball.y + ball.z * ball.z) + rj);
    }
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, keep);
    __syncwarp();  // every ball input of this chunk is read before kball slots are overwritten
    if (keep) {
      const int slot = nkeep + __popc(mask & ((1u << lane) - 1u));
      W.kobj[slot] = j;
      W.kball[slot] = ball;
    }
    nkeep += __popc(mask);
    __syncwarp();
  }
  a_bound = -warp_min(-a_bound);
  // world boxes in the A area (unused until the sweep; instances with
  // parts and triangles): the template's box rows with each part box's centre moved by
  // the candidate's q * axis when they fit (4 rows per box), else the shifts
  // alone, so the box loop reads shared memory instead of global loads (and
  // no chain of dependent loads for a part box)
  const bool shifted = WORLD && b.max_parts > 0 && b.obb_part != nullptr;
  const bool staged = WORLD && nobb > 0 && 4 * nobb <= 32 * APL + 64;
  if (staged) {
#pragma unroll 1
    for (int e = lane; e < 4 * nobb; e += 32) {
      const int bi = e >> 2, row = e & 3;
      float4 v = __ldg(g.obb_tab + 4 * (bx0 + bi) + row);
      if (shifted && row < 3) {
        const float3 sh = box_shift(b, t, c, bx0 + bi, g.status);
        v.w = v.w + (row == 0 ? sh.x : row == 1 ? sh.y : sh.z);
      }
      W.astage[e] = v;
    }
    __syncwarp();
  } else if (shifted) {
#pragma unroll 1
    for (int bi = lane; bi < nobb; bi += 32) {
      const float3 sh = box_shift(b, t, c, bx0 + bi, g.status);
      W.astage[bi] = make_float4(sh.x, sh.y, sh.z, 0.f);
    }
    __syncwarp();
  }
  // ---- object k's spheres (B side), one pass: world frame, world boxes
  // (exact box SDF where the lower bound max(|p| - h) - r is within the
  // band), cull against the kept objects' balls, compacted into Bs as they
  // are produced
  float r2 = 0.f, m = kFarSentinel;
  int Sc = 0;  // B spheres kept
#pragma unroll 1
  for (int q0 = 0; q0 < Sk; q0 += 32) {
    const int q = q0 + lane;
    bool keep = false;
    float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
    float bb = 0.f;
    if (q < Sk) {
      const float4 l = __ldg(reinterpret_cast<const float4*>(b.sph_local) + s0 + Sprev + q);
      const float x = (pk.x - ref.x) + (kcs * l.x - skn * l.y);
      const float y = (pk.y - ref.y) + (skn * l.x + kcs * l.y);
      const float z = (pk.z - ref.z) + l.z;
      const float c2 = x * x + y * y + z * z;
      w = make_float4(x, y, z, l.w);
      bb = c2 - l.w * l.w;
      r2 = fmaxf(r2, c2);
#pragma unroll 1
      for (int bi = 0; bi < nobb; ++bi) {
        float4 R0, R1, R2, Hh;
        // an articulated part's box moves with the candidate's joint value
        float4 sh = make_float4(0.f, 0.f, 0.f, 0.f);
        if (staged) {  // rows with the moved centres
          const float4* o = W.astage + 4 * bi;
          R0 = o[0]; R1 = o[1]; R2 = o[2]; Hh = o[3];
        } else {
          const float4* o = g.obb_tab + 4 * (bx0 + bi);
          R0 = __ldg(o); R1 = __ldg(o + 1); R2 = __ldg(o + 2); Hh = __ldg(o + 3);
          if (shifted) sh = W.astage[bi];
        }
        // box frame: p = R^T (c - centre); rows of R^T are the columns of R,
        // stored as the table's rows
        const float vx = x - ((R0.w + sh.x) - ref.x), vy = y - ((R1.w + sh.y) - ref.y),
                    vz = z - ((R2.w + sh.z) - ref.z);
        const float px = R0.x * vx + R0.y * vy + R0.z * vz;
        const float py = R1.x * vx + R1.y * vy + R1.z * vz;
        const float pz = R2.x * vx + R2.y * vy + R2.z * vz;
        const float ex = fabsf(px) - Hh.x, ey = fabsf(py) - Hh.y, ez = fabsf(pz) - Hh.z;
        const float em = fmaxf(ex, fmaxf(ey, ez));
        if (em - l.w < kBand) {
          const float ux = fmaxf(ex, 0.f), uy = fmaxf(ey, 0.f), uz = fmaxf(ez, 0.f);
          m = fminf(m, sqrtf(ux * ux + uy * uy + uz * uz) + fminf(em, 0.f) - l.w);
        }
      }
#pragma unroll 1
      for (int jj = 0; jj < nkeep && !keep; ++jj) {
        const float4 kb = W.kball[jj];
        const float dx = x - kb.x, dy = y - kb.y, dz = z - kb.z;
        const float lim = kb.w + l.w + kBand + kBroadMargin;
        keep = dx * dx + dy * dy + dz * dz <= lim * lim;
      }
    }
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, keep);
    if (keep) {
      const int pos = Sc + __popc(mask & ((1u << lane) - 1u));
      W.Bs[pos] = w;
      W.Bb[pos] = bb;
    }
    Sc += __popc(mask);
  }
#pragma unroll 1
  for (int q = Sc + lane; q < Sc + kPad; q += 32) {
    W.Bs[q] = make_float4(1e6f, 1e6f, 1e6f, 0.f);
    W.Bb[q] = 3e12f;
  }
  if (lane == 0) {
    cnt.box += (unsigned long long)nobb * (unsigned long long)Sk;
    cnt.exh += (unsigned long long)Sprev * (unsigned long long)Sk;
    cnt.cull += (unsigned long long)Sk * (unsigned long long)nkeep;
  }
  // ---- object k against the world triangles (instances with world features)
  if (WORLD && b.n_tri > 0 && !__any_sync(0xFFFFFFFFu, m < -kBand))
    m = fminf(m, world_tri_min(b, g.tri_chunk, t, pk, ref, rk, skn, kcs, s0 + Sprev, Sk, lane, cnt.tri, cnt.cull));
  m = warp_min(m);
  bool alive = !(m < -kBand);
  r2 = -warp_min(-r2);
  __syncwarp();
  // one tolerance for the whole try, from bounds on |a| and |b|
  const float eps = 1e-5f * (fmaxf(r2, a_bound * a_bound) + 0.01f);
  const float ckx = pk.x - ref.x, cky = pk.y - ref.y, ckz = pk.z - ref.z;
  // ---- object k vs the kept earlier objects: A spheres are read 64 at a
  // time per kept object, culled against object k's ball, staged in shared
  // memory and decided 32 * APL at a time from registers (one sweep site: a
  // full block, or the remainder once nothing is left)
  constexpr int kCap = 32 * APL;
  int fill = 0, jj = 0, qb = 0, q1 = 0;
  bool have_obj = false;
  float px = 0.f, py = 0.f, pz = 0.f;
  float2 osj = make_float2(0.f, 1.f);  // sin, cos of the current kept object's yaw
#pragma unroll 1
  for (;;) {
#pragma unroll 1
    while (!have_obj && jj < nkeep) {
      const int j = W.kobj[jj];
      qb = W.off[j] - s0;
      q1 = W.off[j + 1] - s0;
      const float4 p = W.opose[j];
      osj = W.osc[j];
      px = p.x - ref.x; py = p.y - ref.y; pz = p.z - ref.z;
      have_obj = qb < q1;
      if (!have_obj) ++jj;
    }
    const bool more = Sc > 0 && have_obj;
    if (alive && more && fill < kCap) {
      float4 cand[2];
      bool ck[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int q = qb + u * 32 + lane;
        cand[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        ck[u] = false;
        if (q < q1) {
          const float4 l = __ldg(reinterpret_cast<const float4*>(b.sph_local) + s0 + q);
          cand[u].x = px + (osj.y * l.x - osj.x * l.y);
          cand[u].y = py + (osj.x * l.x + osj.y * l.y);
          cand[u].z = pz + l.z;
          cand[u].w = l.w;
          const float dx = cand[u].x - ckx, dy = cand[u].y - cky, dz = cand[u].z - ckz;
          const float lim = rk + l.w + kBand + kBroadMargin;
          ck[u] = dx * dx + dy * dy + dz * dz <= lim * lim;
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const unsigned mask = __ballot_sync(0xFFFFFFFFu, ck[u]);
        if (ck[u]) W.astage[fill + __popc(mask & ((1u << lane) - 1u))] = cand[u];
        fill += __popc(mask);
      }
      if (lane == 0) cnt.cull += (unsigned long long)min(64, q1 - qb);
      qb += 64;
      if (qb >= q1) {
        have_obj = false;
        ++jj;
      }
    }
    const int n_sw = fill >= kCap ? kCap : (more ? 0 : fill);
    if (alive && n_sw > 0) {
      __syncwarp();
      if (lane == 0) cnt.pairs += (unsigned long long)n_sw * (unsigned long long)Sc;
      sweep_block<APL>(W.astage, n_sw, W.Bs, W.Bb, Sc, eps, lane, m, alive);
      // move the staged overflow (at most 63 spheres) to the front
      const int over = fill - n_sw;
      __syncwarp();
      const float4 v0 = lane < over ? W.astage[n_sw + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 v1 = lane + 32 < over ? W.astage[n_sw + 32 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
      __syncwarp();
      if (lane < over) W.astage[lane] = v0;
      if (lane + 32 < over) W.astage[lane + 32] = v1;
      fill = over;
    }
    if (!alive || (!more && fill == 0)) break;
  }
  __syncwarp();
  out.pass = alive && !(m < 0.f);
  out.band = out.band || fabsf(m) <= kBand;
  return out;
}

// Position of the candidate in the template and the checks every launch
// makes before working on object k (error code, 0 when fine).
__device__ __forceinline__ int check_object(const GenStepArgs& g, const TmplInfo& T, int t, int k, int Sprev,
                                            int Sk) {
  const sc_scene_batch& b = g.b;
  return t < 0 ? kDevBadTemplate
         : (k >= T.nt || T.nt > b.max_obj || T.nt > kMaxObj) ? kDevTooManyObjects
         : (Sk > g.max_sk || Sprev + Sk > b.max_sph) ? kDevTooManySpheres
         : (T.nobb > kMaxObbPerTemplate) ? kDevTooManyBoxes : kDevOk;
}

// Routing of a finished try (warp-uniform).
enum Route : int { kRouteNone = 0, kRouteReach = 1, kRouteGen = 2 };

// Top-down grasp of candidate c's current object k = kc[c] (Sec. IV-E):
// position = top centre of its box, tool z = -world z, tool x along the
// object's yaw; expressed in the template's robot base frame (x, y, z, yaw).
// R row-major, then p, into o[12].
__device__ __forceinline__ void grasp_target_at(const sc_scene_batch& b, const int32_t* cand_t, const TmplInfo* tinfo,
                                                const uint8_t* kc, const float4* poses, int c, float o[12]) {
  const int t = __ldg(&cand_t[c]);
  const TmplInfo& T = tinfo[t];
  const int k = kc[c];
  const int64_t pbase = T.pose0 + (int64_t)(c - T.cand0) * T.nt;
  const float4 p = poses[pbase + k];
  const float hz = __ldg(&b.obj_half[4 * (T.o0 + k) + 2]);
  const float4 base = __ldg(reinterpret_cast<const float4*>(b.tmpl_base) + t);
  float sb, cb, sp, cp;
  sincosf(base.w, &sb, &cb);
  sincosf(p.w - base.w, &sp, &cp);
  const float wx = p.x - base.x, wy = p.y - base.y, wz = p.z + hz - base.z;
  o[0] = cp; o[1] = sp; o[2] = 0.f;
  o[3] = sp; o[4] = -cp; o[5] = 0.f;
  o[6] = 0.f; o[7] = 0.f; o[8] = -1.f;
  o[9] = cb * wx + sb * wy;
  o[10] = -sb * wx + cb * wy;
  o[11] = wz;
}

// Appends the warp's pending routed candidates (lane i holds entry i < npend)
// to their lists: one atomic per list and flush instead of one per try. A
// candidate sent to the reach queue also gets its grasp target at the same
// position (its pose was written by this warp before the flush).
__device__ __forceinline__ void flush_routes(const GenStepArgs& g, int pend_c, int pend_r, int npend, int lane) {
#pragma unroll
  for (int d = kRouteReach; d <= kRouteGen; ++d) {
    const bool mine = lane < npend && pend_r == d;
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, mine);
    if (!mask) continue;
    int* cnt = d == kRouteReach ? g.n_reach : g.n_gen;
    int32_t* list = d == kRouteReach ? g.list_reach : g.list_gen;
    const int leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(cnt, __popc(mask));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    if (mine) {
      const int row = base + __popc(mask & ((1u << lane) - 1u));
      list[row] = pend_c;
      if (d == kRouteReach) {
        float o[12];
        grasp_target_at(g.b, g.cand_t, g.tinfo, g.st.kc, g.poses, pend_c, o);
        float4* dst = reinterpret_cast<float4*>(g.targets + 12 * (size_t)row);
        dst[0] = make_float4(o[0], o[1], o[2], o[3]);
        dst[1] = make_float4(o[4], o[5], o[6], o[7]);
        dst[2] = make_float4(o[8], o[9], o[10], o[11]);
      }
    }
  }
}

__device__ __forceinline__ void add_counters(const GenStepArgs& g, const TryCounters& cnt, int lane) {
  if (lane == 0 && g.stats) {
    atomicAdd(&g.stats[0], cnt.pairs);
    atomicAdd(&g.stats[1], cnt.box);
    atomicAdd(&g.stats[5], cnt.cull);
    atomicAdd(&g.stats[6], cnt.exh);
    if (cnt.tri) atomicAdd(&g.stats[7], cnt.tri);
    if (cnt.far) atomicAdd(&g.stats[8], cnt.far);
  }
}

// One generation round for the objects that carry reachability: each warp
// takes one listed candidate at a time and makes the try its state names
// (object kc[c], try rc[c]). A collision-free try of a reach-flagged object
// goes to this round's reach queue (its state is left for the reach stage);
// otherwise the candidate advances (next try, or next object) into the next
// round's list, to the chained launch (alive) once it reaches k_begin, or
// ends (valid after its last object, invalid after its last try). Work
// distribution: warp w takes item w first, then items claimed from the
// round's counter (the claim for the next item is issued before the current
// one is processed); routed candidates are appended 32 at a time.
template <int APL, int MODE>
__global__ void __launch_bounds__(256, 3) gen_round_kernel(GenStepArgs g) {
  extern __shared__ __align__(16) unsigned char smem[];
  const sc_scene_batch& b = g.b;
  const WarpLayout WL = make_warp_layout(b.max_obj, g.max_sk, APL);
  const WarpState W = warp_state(smem, WL);
  const int lane = threadIdx.x & 31;
  const int warps_per_block = blockDim.x >> 5;
  const int n_items = *(volatile const int*)g.n_in;
  const int warps_total = gridDim.x * warps_per_block;
  int item = blockIdx.x * warps_per_block + (threadIdx.x >> 5);
  if (item >= n_items) return;  // no atomic traffic from warps without work
  const uint64_t seed = *g.seed;
  TryCounters cnt;
  int pend_c = 0, pend_r = kRouteNone, npend = 0;

  while (item < n_items) {
    int next = 0;
    if (lane == 0) next = warps_total + (int)atomicAdd(g.counter, 1u);
    const int c = __ldg(&g.list_in[item]);
    const int t = (c >= 0 && c < b.n_cand) ? __ldg(&g.cand_t[c]) : -1;
    const TmplInfo& T = load_tmpl(g.tinfo, t, W.tmpl, lane);
    const int o0 = T.o0, nt = T.nt;
    const int k = t >= 0 ? (int)g.st.kc[c] : 0;
    const int r = t >= 0 ? (int)g.st.rc[c] : 0;
    int Sprev = 0, Sk = 0, rel = 0;
    if (t >= 0 && k < nt) {
      Sprev = __ldg(&b.obj_sph_off[o0 + k]) - T.s0;
      Sk = __ldg(&b.obj_sph_off[o0 + k + 1]) - T.s0 - Sprev;
      rel = __ldg(&b.obj_rel[o0 + k]);
    }
    const int err = check_object(g, T, t, k, Sprev, Sk);
    int route = kRouteNone;
    if (err != kDevOk) {
      if (lane == 0) {
        latch_error(g.status, err);
        if (t >= 0) g.band[c] = 1;
      }
    } else {
      const int64_t pbase = T.pose0 + (int64_t)(c - T.cand0) * nt;
      // earlier objects' poses, half extents (into the kept-ball slots) and
      // sphere offsets, copied while object k is sampled
#pragma unroll 1
      for (int j = lane; j < k; j += 32) {
        cp_async16(W.opose + j, g.poses + pbase + j);
        cp_async16(W.kball + j, reinterpret_cast<const float4*>(b.obj_half) + o0 + j);
      }
#pragma unroll 1
      for (int j = lane; j <= k + 1; j += 32) cp_async4(W.off + j, b.obj_sph_off + o0 + j);
      cp_async_commit();
      const TryOut res =
          gen_try<APL, true, MODE>(g, T, W, t, c, k, r, rel, Sprev, Sk, pbase, seed, g.poses + pbase, lane, cnt);
      bool done = false;
      const bool placed = res.pass;
      const bool reach_try = placed && g.list_reach && (rel & SC_REL_REACH);
      if (reach_try) {
        route = kRouteReach;
      } else if (placed) {  // object k placed
        done = k + 1 == nt;
        if (!done) route = k + 1 < g.st.k_begin ? kRouteGen : kRouteNone;
      } else if (r < g.max_retries) {
        route = kRouteGen;
      }
      if (lane == 0) {
        if (res.band) g.band[c] = 1;
        atomicAdd(&g.tries[c], 1);
        if (done) {
          g.valid[c] = 1;
        } else if (placed && route != kRouteReach) {
          g.st.kc[c] = (uint8_t)(k + 1);
          g.st.rc[c] = 0;
          if (route == kRouteNone) g.st.alive[c] = 1;
        } else if (!placed && route == kRouteGen) {
          g.st.rc[c] = (uint16_t)(r + 1);
        }
      }
    }
    if (route != kRouteNone) {
      if (lane == npend) {
        pend_c = c;
        pend_r = route;
      }
      ++npend;
    }
    __syncwarp();  // the warp's shared memory is reused by its next candidate
    item = __shfl_sync(0xFFFFFFFFu, next, 0);
    if (npend == 32 || (npend > 0 && item >= n_items)) {
      flush_routes(g, pend_c, pend_r, npend, lane);
      npend = 0;
    }
  }
  add_counters(g, cnt, lane);
}

// The objects after the reachability stage (all objects when there is none):
// one warp runs a candidate's whole remaining placement loop (every object,
// every try) with the candidate's placed objects kept in its shared memory.
// Candidates are taken in the caller's order (heaviest first, candidates of
// a template together, so concurrent warps share the template's spheres in
// the caches), skipping those not alive at object k_begin.
struct ChainArgs {
  const int32_t* order;  // candidate order (NULL: 0..n-1)
  int n;
  int k_begin;
  const uint8_t* alive;  // [n_cand] alive at object k_begin
  unsigned int* counter;
};

template <int APL, int MODE>
__global__ void __launch_bounds__(256, 3) gen_chain_kernel(GenStepArgs g, ChainArgs ca) {
  extern __shared__ __align__(16) unsigned char smem[];
  const sc_scene_batch& b = g.b;
  const WarpLayout WL = make_warp_layout(b.max_obj, g.max_sk, APL);
  const WarpState W = warp_state(smem, WL);
  const int lane = threadIdx.x & 31;
  const int warps_per_block = blockDim.x >> 5;
  const int warps_total = gridDim.x * warps_per_block;
  int item = blockIdx.x * warps_per_block + (threadIdx.x >> 5);
  if (item >= ca.n) return;
  const uint64_t seed = *g.seed;
  TryCounters cnt;
  while (item < ca.n) {
    int next = 0;
    if (lane == 0) next = warps_total + (int)atomicAdd(ca.counter, 1u);
    const int c = ca.order ? __ldg(&ca.order[item]) : item;
    const bool live = c >= 0 && c < b.n_cand && __ldg(&ca.alive[c]);
    const int t = live ? __ldg(&g.cand_t[c]) : -1;
    if (t >= 0) {
      const TmplInfo& T = load_tmpl(g.tinfo, t, W.tmpl, lane);
      const int o0 = T.o0, nt = T.nt;
      const int64_t pbase = T.pose0 + (int64_t)(c - T.cand0) * nt;
      // objects placed before k_begin (by the per-try launches) and the
      // sphere offsets of all objects
      const int k0 = min(ca.k_begin, nt);
#pragma unroll 1
      for (int j = lane; j < k0; j += 32) {
        const float4 p = g.poses[pbase + j];
        const float4 H = __ldg(reinterpret_cast<const float4*>(b.obj_half) + o0 + j);
        float sn, cs;
        sincos_cw(p.w, &sn, &cs);
        W.opose[j] = p;
        W.osc[j] = make_float2(sn, cs);
        W.orad[j] = sqrtf(H.x * H.x + H.y * H.y + H.z * H.z);
      }
      const int n_off = min(nt, b.max_obj) + 1;
#pragma unroll 1
      for (int j = lane; j < n_off; j += 32) W.off[j] = __ldg(&b.obj_sph_off[o0 + j]);
      __syncwarp();
      int ntries = 0;
      bool band = false, dead = false;
#pragma unroll 1
      for (int k = k0; k < nt && !dead; ++k) {
        const int Sprev = W.off[k] - T.s0;
        const int Sk = W.off[k + 1] - W.off[k];
        const int err = check_object(g, T, t, k, Sprev, Sk);
        if (err != kDevOk) {
          if (lane == 0) latch_error(g.status, err);
          band = true;
          dead = true;
          break;
        }
        const int rel = __ldg(&b.obj_rel[o0 + k]);
        bool placed = false;
#pragma unroll 1
        for (int r = 0; r <= g.max_retries && !placed; ++r) {
          const TryOut res =
              gen_try<APL, false, MODE>(g, T, W, t, c, k, r, rel, Sprev, Sk, pbase, seed, W.opose, lane, cnt);
          ++ntries;
          band = band || res.band;
          placed = res.pass;
        }
        dead = !placed;
      }
      if (lane == 0) {
        g.tries[c] += ntries;
        if (band) g.band[c] = 1;
        if (!dead) g.valid[c] = 1;
      }
    } else if (live && lane == 0) {
      latch_error(g.status, kDevBadTemplate);
    }
    __syncwarp();
    item = __shfl_sync(0xFFFFFFFFu, next, 0);
  }
  add_counters(g, cnt, lane);
}

// ---- reachability stage (Sec. IV-E): the collision-free tries of
// reach-flagged objects, in the reach list, get a top-down grasp target in
// the robot base frame; an optional learned gate sends the ones it predicts
// unreachable back to retry; exact IK decides the rest.
// Logit margin above the gate's threshold within which a passed target is
// "doubtful" (likelier unreachable, so likelier to run every IK iteration).
constexpr float kDoubtful = 5.f;

struct ReachArgs {
  sc_scene_batch b;
  const int32_t* cand_t;
  const TmplInfo* tinfo;
  int max_retries, gated;
  float tau;
  CandState st;
  const int32_t* list_reach;  // this round's reach queue
  const int* n_reach;
  float* targets;        // [cap][12]
  int32_t* list_ik;      // positions in the reach list the gate passed: those within
                         // kDoubtful of the threshold from the front, the others
                         // from the back (capacity ik_cap), so IK starts with the
                         // targets likeliest to run every iteration
  int* n_ik;             // [2]: front and back counts
  int ik_cap;
  int32_t* list_gen;     // the round after next: retries and next objects
  int* n_gen;
  unsigned int* claim;   // IK work counter of the round (zeroed at init)
  const uint2* map_counts;  // 4D reachability map gate (NULL: the surrogate or none)
  RmapGrid map_grid;
  int map_tau;
  const float4* poses;
  uint8_t* valid;
  uint8_t* band;
  float* q_reach;        // [P][7] or NULL
  unsigned long long* stats;
  ikc::IkArgs ik;
};

// After the reach decision of try (k, r) of candidate c (one thread): the
// next object (or valid after the last one, or the chained launch from
// k_begin on) when it passed; the next try when it failed and tries remain.
__device__ __forceinline__ void reach_advance(const ReachArgs& A, int c, int k, int r, int nt, bool pass) {
  if (pass) {
    if (k + 1 == nt) {
      A.valid[c] = 1;
      return;
    }
    A.st.kc[c] = (uint8_t)(k + 1);
    A.st.rc[c] = 0;
    if (k + 1 < A.st.k_begin) A.list_gen[atomicAdd(A.n_gen, 1)] = c;
    else A.st.alive[c] = 1;
  } else if (r < A.max_retries) {
    A.st.rc[c] = (uint16_t)(r + 1);
    A.list_gen[atomicAdd(A.n_gen, 1)] = c;
  }
}


// A gate's decision on reach-queue entry `row` (warp-uniform call; `valid`
// false on lanes past the queue): a pass goes to the IK list (a doubtful one
// to its front, the others to its back), a rejection retries (or ends
// invalid); appends aggregated per warp.
__device__ __forceinline__ void gate_route(const ReachArgs& A, int row, bool valid, bool pass, bool doubtful) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  pass = valid && pass;
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const bool mine = pass && (doubtful == (side == 0));
    const unsigned mp = __ballot_sync(0xFFFFFFFFu, mine);
    if (mp) {
      const int leader = __ffs(mp) - 1;
      int base = 0;
      if (lane == leader) base = atomicAdd(A.n_ik + side, __popc(mp));
      base = __shfl_sync(0xFFFFFFFFu, base, leader);
      const int pos = base + __popc(mp & lt);
      if (mine) A.list_ik[side == 0 ? pos : A.ik_cap - 1 - pos] = row;
    }
  }
  const bool rej = valid && !pass;
  int c = 0;
  bool retry = false;
  if (rej) {
    c = A.list_reach[row];
    const int r = A.st.rc[c];
    retry = r < A.max_retries;
    if (retry) A.st.rc[c] = (uint16_t)(r + 1);
  }
  const unsigned mr = __ballot_sync(0xFFFFFFFFu, retry);
  if (mr) {
    const int leader = __ffs(mr) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(A.n_gen, __popc(mr));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    if (retry) A.list_gen[base + __popc(mr & lt)] = c;
  }
  const unsigned mj = __ballot_sync(0xFFFFFFFFu, rej);
  if (lane == 0 && mj) atomicAdd(&A.stats[3], (unsigned long long)__popc(mj));
}

// The learned gate's decision fused into the tensor-core forward pass: its
// rows are the round's reach queue (grasp targets written by the generation
// round), and each logit is decided at once (logit >= tau).
struct GateIO {
  static constexpr int kColGroups = 4;  // 16 epilogue warps (8 left room for more IK blocks but ran slower)
  ReachArgs A;
  __device__ int rows() const { return *(volatile const int*)A.n_reach; }
  __device__ void features(int row, float f[9]) const {
    const float* t = A.targets + 12 * (size_t)row;
    f[0] = __ldg(t + 9); f[1] = __ldg(t + 10); f[2] = __ldg(t + 11);
    f[3] = __ldg(t + 0); f[4] = __ldg(t + 3); f[5] = __ldg(t + 6);
    f[6] = __ldg(t + 1); f[7] = __ldg(t + 4); f[8] = __ldg(t + 7);
  }
  __device__ void emit(int row, bool valid, float logit) const {
    gate_route(A, row, valid, logit >= A.tau, logit < A.tau + kDoubtful);
  }
};

// The 4D reachability map's decision on the round's reach queue (the grasp
// targets were written by the generation round): score >= the map's
// threshold passes to IK, warps walking the queue 32 entries at a time.
__global__ void reach_map_gate_kernel(ReachArgs A) {
  const int n = *(volatile const int*)A.n_reach;
  const int lane = threadIdx.x & 31;
  for (int i0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < n; i0 += gridDim.x * blockDim.x) {
    const int i = i0 + lane;
    const bool valid = i < n;
    bool pass = false;
    if (valid) {
      float o[12];
      const float* t = A.targets + 12 * (size_t)i;
#pragma unroll
      for (int j = 0; j < 12; ++j) o[j] = t[j];
      pass = (int)rmap_score(A.map_counts, rmap_cell(A.map_grid, o)) >= A.map_tau;
    }
    gate_route(A, i, valid, pass, true);
  }
}

// Exact IK, one warp per entry; seeds keyed by (candidate, object, try).
// Entries cost from one check to 100 steps, so warps claim them one at a
// time (first entry static, the claim for the next issued before solving the
// current one) from a grid sized to the resident blocks. kRight: the signed
// forward kinematics of arms whose middle twists are +-pi/2 (ArmK::right).
template <bool kRight>
__global__ void __launch_bounds__(128) reach_ik_kernel(ReachArgs A) {
  const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
  const int nf = A.gated ? *(volatile const int*)A.n_ik : 0;  // front part of the IK list
  const int n = A.gated ? nf + *(volatile const int*)(A.n_ik + 1) : *(volatile const int*)A.n_reach;
  const int warps_total = gridDim.x * warps;
  unsigned long long solves = 0, seed_iters = 0;
  int j = blockIdx.x * warps + (threadIdx.x >> 5);
  while (j < n) {
    int next = 0;
    if (lane == 0) next = warps_total + (int)atomicAdd(A.claim, 1u);
    const int i = A.gated ? A.list_ik[j < nf ? j : A.ik_cap - 1 - (j - nf)] : j;
    const int c = A.list_reach[i];
    const int k = A.st.kc[c], r = A.st.rc[c];
    const ikc::Target T = ikc::load_target(A.targets + 12 * (size_t)i);
    float q[7], pe2, sr, cr;
    const ikc::Solve s =
        ikc::warp_solve<kRight>(A.ik, T, (uint32_t)c, ((uint32_t)k << 16) | (uint32_t)r, lane, q, pe2, sr, cr);
    ++solves;
    seed_iters += (unsigned long long)s.checks * (unsigned long long)A.ik.seeds;
    __syncwarp();  // every lane has read the state before the winner updates it
    if (lane == s.winner) {
      const TmplInfo& Tm = A.tinfo[__ldg(&A.cand_t[c])];
      const int64_t pbase = Tm.pose0 + (int64_t)(c - Tm.cand0) * Tm.nt;
      if (s.band) A.band[c] = 1;
      if (s.found && A.q_reach) {
#pragma unroll
        for (int jq = 0; jq < 7; ++jq) A.q_reach[7 * (pbase + k) + jq] = q[jq];
      }
      reach_advance(A, c, k, r, Tm.nt, s.found);
    }
    j = __shfl_sync(0xFFFFFFFFu, next, 0);
  }
  if (lane == 0 && solves) {
    atomicAdd(&A.stats[2], solves);
    atomicAdd(&A.stats[4], seed_iters);
  }
}

// out[0]: 1 + the largest template-local index of an object carrying the
// reach flag; out[1]: the most spheres of one object; out[2]: 1 if an object
// uses a relation beyond FREE / ON_TOP / NEXT_TO (a DIRECTIONAL or MIDDLE
// kind, or the LOCAL or FACE_TO flag).
__global__ void batch_scan_kernel(sc_scene_batch b, int* out) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < b.n_templates; t += gridDim.x * blockDim.x) {
    const int o0 = b.tmpl_obj_off[t], o1 = b.tmpl_obj_off[t + 1];
    int ext = 0;
    for (int o = o0; o < o1; ++o)
      if (b.obj_rel[o] & SC_REL_REACH) ext = o - o0 + 1;
    if (ext) atomicMax(out, ext);
  }
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < b.n_objects; o += gridDim.x * blockDim.x) {
    atomicMax(out + 1, b.obj_sph_off[o + 1] - b.obj_sph_off[o]);
    const int rel = b.obj_rel[o];
    if ((rel & SC_REL_KIND_MASK) > SC_REL_NEXT_TO || (rel & (SC_REL_LOCAL | SC_REL_FACE_TO))) atomicMax(out + 2, 1);
  }
}

// Per-call tables: the template of every candidate, one TmplInfo record per
// template (with the support polygon's bounding box) and the inverse squared
// length of every polygon edge (edge i runs from vertex i-1 to vertex i,
// cyclically within its polygon; 0 for a zero-length edge).
__global__ void gen_tables_kernel(sc_scene_batch b, int32_t* cand_t, TmplInfo* tinfo, float* edge_inv,
                                  float4* obb_tab, float4* tri_chunk) {
  const int stride = gridDim.x * blockDim.x;
  // triangle chunks (one warp per template): the centre of the chunk's
  // bounding box and the largest vertex distance from it, rounded up by a
  // relative 1e-6 and 1e-6 m so the ball holds every vertex despite FP32
  if (b.n_tri > 0) {
    const int lane = threadIdx.x & 31, nwarp = stride >> 5;
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < b.n_templates; t += nwarp) {
      const int tq0 = b.tmpl_tri_off[t], ntri = b.tmpl_tri_off[t + 1] - tq0;
      for (int j = 0; j * 32 < ntri; ++j) {
        const bool has = j * 32 + lane < ntri;
        float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
        float v[9];
        if (has) {
          const float* q = b.tri + 12 * (int64_t)(tq0 + j * 32 + lane);
          for (int i = 0; i < 3; ++i)
            for (int d = 0; d < 3; ++d) {
              v[3 * i + d] = q[4 * i + d];
              lo[d] = fminf(lo[d], v[3 * i + d]);
              hi[d] = fmaxf(hi[d], v[3 * i + d]);
            }
        }
        for (int d = 0; d < 3; ++d) {
          lo[d] = warp_min(lo[d]);
          hi[d] = -warp_min(-hi[d]);
        }
        const float cx = 0.5f * (lo[0] + hi[0]), cy = 0.5f * (lo[1] + hi[1]), cz = 0.5f * (lo[2] + hi[2]);
        float r2 = 0.f;
        if (has)
          for (int i = 0; i < 3; ++i) {
            const float dx = v[3 * i] - cx, dy = v[3 * i + 1] - cy, dz = v[3 * i + 2] - cz;
            r2 = fmaxf(r2, dx * dx + dy * dy + dz * dz);
          }
        r2 = -warp_min(-r2);
        if (lane == 0) tri_chunk[tri_chunk_slot(tq0, t, j)] = make_float4(cx, cy, cz, sqrtf(r2) * 1.000001f + 1e-6f);
      }
    }
  }
  // world boxes: the transpose of R (box frame -> world, from the normalised
  // quaternion) row by row with the centre, then the half extents
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < b.n_obb; i += stride) {
    const float* o = b.obb + 12 * i;
    float qx = o[4], qy = o[5], qz = o[6], qw = o[7];
    const float inv = rsqrtf(qx * qx + qy * qy + qz * qz + qw * qw);
    qx *= inv; qy *= inv; qz *= inv; qw *= inv;
    // columns of R
    const float c00 = 1.f - 2.f * (qy * qy + qz * qz), c01 = 2.f * (qx * qy + qz * qw), c02 = 2.f * (qx * qz - qy * qw);
    const float c10 = 2.f * (qx * qy - qz * qw), c11 = 1.f - 2.f * (qx * qx + qz * qz), c12 = 2.f * (qy * qz + qx * qw);
    const float c20 = 2.f * (qx * qz + qy * qw), c21 = 2.f * (qy * qz - qx * qw), c22 = 1.f - 2.f * (qx * qx + qy * qy);
    obb_tab[4 * i + 0] = make_float4(c00, c01, c02, o[0]);
    obb_tab[4 * i + 1] = make_float4(c10, c11, c12, o[1]);
    obb_tab[4 * i + 2] = make_float4(c20, c21, c22, o[2]);
    obb_tab[4 * i + 3] = make_float4(o[8], o[9], o[10], 0.f);
  }
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < b.n_cand; c += stride) cand_t[c] = template_of(b, c);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < b.n_templates; t += stride) {
    TmplInfo T;
    T.o0 = b.tmpl_obj_off[t];
    T.nt = b.tmpl_obj_off[t + 1] - T.o0;
    T.s0 = b.obj_sph_off[T.o0];
    T.bx0 = b.tmpl_obb_off[t];
    T.nobb = b.tmpl_obb_off[t + 1] - T.bx0;
    T.v0 = b.tmpl_poly_off[t];
    T.nv = b.tmpl_poly_off[t + 1] - T.v0;
    T.cand0 = b.cand_tmpl_off[t];
    T.pose0 = b.tmpl_pose_off[t];
    T.z = b.tmpl_support_z[t];
    T.pad = 0.f;
    float xmin = 3e38f, xmax = -3e38f, ymin = 3e38f, ymax = -3e38f;
    if (T.nv >= 3 && T.nv <= kMaxPolyVerts) {
      const float2* v = reinterpret_cast<const float2*>(b.poly_verts) + T.v0;
      for (int i = 0; i < T.nv; ++i) {
        const float2 a = v[i == 0 ? T.nv - 1 : i - 1], p = v[i];
        xmin = fminf(xmin, p.x); xmax = fmaxf(xmax, p.x);
        ymin = fminf(ymin, p.y); ymax = fmaxf(ymax, p.y);
        const float ex = p.x - a.x, ey = p.y - a.y, len2 = ex * ex + ey * ey;
        edge_inv[T.v0 + i] = len2 > 0.f ? 1.f / len2 : 0.f;
      }
    }
    T.xmin = xmin; T.xmax = xmax; T.ymin = ymin; T.ymax = ymax;
    tinfo[t] = T;
  }
}

// Initial state of the listed candidates: outputs cleared, poses NaN until
// placed, object 0 / try 0, in round 0's list (the caller's order or
// 0..n-1); alive = 1 when the chained launch starts at object 0. Counts are
// zeroed except round 0's list length; work counters and statistics zeroed.
__global__ void gen_init_kernel(sc_scene_batch b, const int32_t* order, int n, int32_t* list0, int* counts,
                                int n_counts, unsigned int* counters, int n_counters, float4* poses, uint8_t* valid,
                                uint8_t* band, int32_t* tries, unsigned long long* stats, int* status, CandState st) {
  const int stride = gridDim.x * blockDim.x;
  const float nan = __int_as_float(0x7FC00000);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int c = order ? order[i] : i;
    list0[i] = c;
    const int t = template_of(b, c);
    if (t < 0) {  // the step kernels skip it too
      latch_error(status, kDevBadTemplate);
      continue;
    }
    valid[c] = 0;
    band[c] = 0;
    tries[c] = 0;
    st.kc[c] = 0;
    st.rc[c] = 0;
    st.alive[c] = st.k_begin == 0 ? 1 : 0;
    const int o0 = b.tmpl_obj_off[t], nt = b.tmpl_obj_off[t + 1] - o0;
    const int64_t pbase = b.tmpl_pose_off[t] + (int64_t)(c - b.cand_tmpl_off[t]) * nt;
    for (int k = 0; k < nt; ++k) poses[pbase + k] = make_float4(nan, nan, nan, nan);
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_counts; i += stride) counts[i] = (i == 0) ? n : 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_counters; i += stride) counters[i] = 0;
  if (blockIdx.x == 0 && threadIdx.x < 9 && stats) stats[threadIdx.x] = 0;
}

template <int APL, int MODE>
cudaError_t prepare_step_kernel(size_t smem, int threads, int ctas_per_sm, int num_sms, int* grid) {
  auto kern = gen_round_kernel<APL, MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(gen_chain_kernel<APL, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  *grid = num_sms * (ctas_per_sm < per_sm ? ctas_per_sm : per_sm);
  return cudaSuccess;
}

template <int APL>
void launch_round(const GenStepArgs& g, int mode, int grid, int threads, size_t smem, cudaStream_t s) {
  if (mode == 2) gen_round_kernel<APL, 2><<<grid, threads, smem, s>>>(g);
  else if (mode == 1) gen_round_kernel<APL, 1><<<grid, threads, smem, s>>>(g);
  else gen_round_kernel<APL, 0><<<grid, threads, smem, s>>>(g);
}

template <int APL>
void launch_chain(const GenStepArgs& g, const ChainArgs& ca, int mode, int grid, int threads, size_t smem,
                  cudaStream_t s) {
  if (mode == 2) gen_chain_kernel<APL, 2><<<grid, threads, smem, s>>>(g, ca);
  else if (mode == 1) gen_chain_kernel<APL, 1><<<grid, threads, smem, s>>>(g, ca);
  else gen_chain_kernel<APL, 0><<<grid, threads, smem, s>>>(g, ca);
}

}  // namespace

cudaError_t batch_scan(const sc_scene_batch& b, int* scratch_int3, int* out_host3, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(scratch_int3, 0, 3 * sizeof(int), s);
  if (e) return e;
  batch_scan_kernel<<<64, 256, 0, s>>>(b, scratch_int3);
  if ((e = cudaGetLastError())) return e;
  if ((e = cudaMemcpyAsync(out_host3, scratch_int3, 3 * sizeof(int), cudaMemcpyDeviceToHost, s))) return e;
  return cudaStreamSynchronize(s);
}

int generate_rounds(int reach_objects, int max_retries) {
  // a try of a reach-flagged object takes at most two rounds (generation,
  // then the reach stage, whose outcome lands in the round after next)
  return 2 * reach_objects * (max_retries + 1);
}

// Scratch: round lists G[3], reach queues Q[2] and gate-passed lists IK[2]
// (int32 [n] each), two slots of grasp targets (12 floats); counts
// (list lengths per round [NR + 2], reach queue lengths per round [NR], the
// IK list's two part lengths per round [2 NR]); work counters (generation claims per round, the chained
// launch's, IK claims per round); the per-candidate state (object, try,
// alive); the per-call tables (candidate templates, TmplInfo records,
// inverse edge lengths, world-box frames, triangle chunk balls); then the
// seed scalar.
// NR is bounded by generate_rounds(max_obj, max_retries).
struct GenScratch {
  size_t lists, counts, counters, kc, rc, alive, cand_t, tinfo, edge_inv, obb_tab, tri_chunk, seed, total;
};

static GenScratch gen_scratch_layout(const sc_scene_batch& b, int n_items, int max_retries) {
  auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t n = (size_t)n_items;
  const size_t NR = (size_t)generate_rounds(b.max_obj, max_retries);
  GenScratch L;
  L.lists = 0;
  L.counts = up(L.lists + 7 * n * sizeof(int32_t) + 2 * 12 * n * sizeof(float));
  L.counters = up(L.counts + ((NR + 2) + 3 * NR) * sizeof(int));
  L.kc = up(L.counters + (2 * NR + 1) * sizeof(unsigned int));
  L.rc = up(L.kc + (size_t)b.n_cand);
  L.alive = up(L.rc + (size_t)b.n_cand * sizeof(uint16_t));
  L.cand_t = up(L.alive + (size_t)b.n_cand);
  L.tinfo = up(L.cand_t + (size_t)b.n_cand * sizeof(int32_t));
  L.edge_inv = up(L.tinfo + (size_t)b.n_templates * sizeof(TmplInfo));
  L.obb_tab = up(L.edge_inv + (size_t)b.n_verts * sizeof(float));
  L.tri_chunk = up(L.obb_tab + (size_t)b.n_obb * 4 * sizeof(float4));
  L.seed = up(L.tri_chunk + tri_chunk_slots(b) * sizeof(float4));  // the 8-byte seed on a 256-byte boundary
  L.total = L.seed + 256;
  return L;
}

size_t generate_seed_offset(const sc_scene_batch& b, int n_items, int max_retries) {
  return gen_scratch_layout(b, n_items, max_retries).seed;
}

size_t generate_scratch_bytes(const sc_scene_batch& b, int n_items, int max_retries) {
  return gen_scratch_layout(b, n_items, max_retries).total;
}

cudaError_t enqueue_generate(const sc_scene_batch& b, const GenerateLaunch& a, const sc_collide_config& cfg,
                             int num_sms, cudaStream_t s, const char** why) {
  *why = check_collide_config(cfg);
  if (*why) return cudaErrorInvalidValue;
  if (cfg.threads > 512) { *why = "generation uses at most 512 threads per CTA"; return cudaErrorInvalidValue; }
  const int max_sk = a.max_sph_obj > 0 ? a.max_sph_obj : kMaxSphPerObj;
  const size_t smem = (size_t)(cfg.threads / 32) * make_warp_layout(b.max_obj, max_sk, cfg.a_per_lane).bytes;
  if (smem > 227 * 1024) { *why = "threads x per-warp shared memory exceeds one CTA's (lower threads)"; return cudaErrorInvalidValue; }
  const int n = a.n_items;
  const int K = b.max_obj, R = a.max_retries;
  const bool reach = a.arm != nullptr;
  // objects [0, k_begin) carry reachability and run in rounds (generation,
  // then the gate and IK on two side streams, overlapping the next rounds);
  // the rest run in one chained launch
  const int k_begin = reach ? (a.reach_objects < K ? a.reach_objects : K) : 0;
  const int NR = generate_rounds(k_begin, R);
  if (k_begin > 0 && (a.n_events < 2 * NR + 1 || !a.side[0] || !a.side[1])) {
    *why = "internal: too few events or side streams for the rounds";
    return cudaErrorInvalidValue;
  }
  const GenScratch SL = gen_scratch_layout(b, n, R);
  char* sb = static_cast<char*>(a.scratch);
  int32_t* ib = reinterpret_cast<int32_t*>(sb + SL.lists);
  int32_t* G[3] = {ib, ib + n, ib + 2 * (size_t)n};
  int32_t* Q[2] = {ib + 3 * (size_t)n, ib + 4 * (size_t)n};
  int32_t* IK[2] = {ib + 5 * (size_t)n, ib + 6 * (size_t)n};
  float* fb = reinterpret_cast<float*>(ib + 7 * (size_t)n);
  float* targets[2] = {fb, fb + 12 * (size_t)n};
  const int NRmax = generate_rounds(K, R);
  int* counts = reinterpret_cast<int*>(sb + SL.counts);
  const int n_counts = (NRmax + 2) + 3 * NRmax;
  int* cnt_gen = counts;                  // [NR + 2]
  int* cnt_reach = counts + (NRmax + 2);  // [NR]
  int* cnt_ik = cnt_reach + NRmax;        // [NR][2]
  unsigned int* counters = reinterpret_cast<unsigned int*>(sb + SL.counters);
  const int n_counters = 2 * NRmax + 1;  // generation claims per round, the chained launch's, IK claims per round
  CandState st;
  st.kc = reinterpret_cast<uint8_t*>(sb + SL.kc);
  st.rc = reinterpret_cast<uint16_t*>(sb + SL.rc);
  st.alive = reinterpret_cast<uint8_t*>(sb + SL.alive);
  st.k_begin = k_begin;
  int32_t* cand_t = reinterpret_cast<int32_t*>(sb + SL.cand_t);
  TmplInfo* tinfo = reinterpret_cast<TmplInfo*>(sb + SL.tinfo);
  float* edge_inv = reinterpret_cast<float*>(sb + SL.edge_inv);
  float4* obb_tab = reinterpret_cast<float4*>(sb + SL.obb_tab);
  float4* tri_chunk = reinterpret_cast<float4*>(sb + SL.tri_chunk);

  int grid = 0;
  cudaError_t e;
  switch (cfg.a_per_lane) {
    case 1:
      e = a.ext_rel == 2   ? prepare_step_kernel<1, 2>(smem, cfg.threads, cfg.ctas_per_sm, num_sms, &grid)
          : a.ext_rel == 1 ? prepare_step_kernel<1, 1>(smem, cfg.threads, cfg.ctas_per_sm, num_sms, &grid)
                           : prepare_step_kernel<1, 0>(smem, cfg.threads, cfg.ctas_per_sm, num_sms, &grid);
      break;
    case 2:
      e = a.ext_rel == 2   ? prepare_step_kernel<2, 2>(smem, cfg.threads, cfg.ctas_per_sm, num_sms, &grid)
          : a.ext_rel == 1 ? prepare_step_kernel<2, 1>(smem, cfg.threads, cfg.ctas_per_sm, num_sms, &grid)
                           : prepare_step_kernel<2, 0>(smem, cfg.threads, cfg.ctas_per_sm, num_sms, &grid);
      break;
    default:
      e = a.ext_rel == 2   ? prepare_step_kernel<4, 2>(smem, cfg.threads, cfg.ctas_per_sm, num_sms, &grid)
          : a.ext_rel == 1 ? prepare_step_kernel<4, 1>(smem, cfg.threads, cfg.ctas_per_sm, num_sms, &grid)
                           : prepare_step_kernel<4, 0>(smem, cfg.threads, cfg.ctas_per_sm, num_sms, &grid);
      break;
  }
  if (e != cudaSuccess) return e;
  {
    int blocks = (n + 255) / 256;
    blocks = blocks < num_sms * 4 ? blocks : num_sms * 4;
    if (blocks < 1) blocks = 1;
    gen_init_kernel<<<blocks, 256, 0, s>>>(b, a.order, n, G[0], counts, n_counts, counters, n_counters,
                                           reinterpret_cast<float4*>(a.poses), a.valid, a.band, a.tries, a.stats,
                                           a.status, st);
    int tmax = b.n_cand > b.n_templates ? b.n_cand : b.n_templates;
    tmax = tmax > b.n_obb ? tmax : b.n_obb;
    int tb = (tmax + 255) / 256;
    tb = tb < num_sms * 4 ? tb : num_sms * 4;
    gen_tables_kernel<<<tb < 1 ? 1 : tb, 256, 0, s>>>(b, cand_t, tinfo, edge_inv, obb_tab, tri_chunk);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  GenStepArgs g;
  std::memset(&g, 0, sizeof(g));
  g.b = b;
  g.cand_t = cand_t;
  g.tinfo = tinfo;
  g.edge_inv = edge_inv;
  g.obb_tab = obb_tab;
  g.tri_chunk = tri_chunk;
  g.seed = a.seed_dev;
  g.max_attempts = a.max_attempts;
  g.max_retries = R;
  g.reach_r2 = -1.f;
  g.reach_w2 = 0.f;
  g.reach_z0 = 0.f;
  g.reach_v = make_float3(0.f, 0.f, 0.f);
  if (reach) {
    // DH rows 0..6. Every frame origin of the chain lies within |a_0| + the
    // sum over the rows after the first of sqrt(a_i^2 + d_i^2) of the
    // shoulder (0, 0, d_0) (row i adds a_i x_i + d_i z_i, x_i perpendicular
    // to z_i): the tool within r7 (rows 1..6), the wrist p6 (origin of frame
    // 6) within r6 (rows 1..5). The tool sits at p6 + R v, v = (a_6, d_6 sin
    // alpha_6, d_6 cos alpha_6) in the tool frame R, so a check of q passing
    // or inside the band (position error <= tol_pos + 1e-5, angle <= tol_rot
    // + 1e-5) puts t* - R* v within tol_pos + 1e-5 + 2 sin((tol_rot + 1e-5) /
    // 2) |v| of p6. The 1e-4 margins cover FP32 rounding.
    auto link = [&](int i) {
      return sqrt((double)a.arm->dh_a[i] * a.arm->dh_a[i] + (double)a.arm->dh_d[i] * a.arm->dh_d[i]);
    };
    double r6 = fabs((double)a.arm->dh_a[0]);
    for (int i = 1; i < 6; ++i) r6 += link(i);
    const double r7 = r6 + link(6);
    const double tp = (double)a.ik->tol_pos + 1e-5, tr = (double)a.ik->tol_rot + 1e-5;
    const double al = (double)a.arm->dh_alpha[6];
    const double vx = a.arm->dh_a[6], vy = a.arm->dh_d[6] * sin(al), vz = a.arm->dh_d[6] * cos(al);
    const double vn = sqrt(vx * vx + vy * vy + vz * vz);
    const double b7 = r7 + tp + 1e-4;
    const double b6 = r6 + tp + 2.0 * sin(tr < 3.14159 ? tr / 2.0 : 1.5707963) * vn + 1e-4;
    g.reach_r2 = (float)(b7 * b7);
    g.reach_w2 = (float)(b6 * b6);
    g.reach_z0 = a.arm->dh_d[0];
    g.reach_v = make_float3((float)vx, (float)vy, (float)vz);
  }
  g.max_sk = max_sk;
  g.seg_len = cfg.seg_len;
  g.st = st;
  g.poses = reinterpret_cast<float4*>(a.poses);
  g.valid = a.valid;
  g.band = a.band;
  g.tries = a.tries;
  g.stats = a.stats;
  g.status = a.status;
  ReachArgs ra;
  std::memset(&ra, 0, sizeof(ra));
  if (reach) {
    ra.b = b;
    ra.cand_t = cand_t;
    ra.tinfo = tinfo;
    ra.max_retries = R;
    ra.gated = a.gate != nullptr || a.map_counts != nullptr;
    ra.map_counts = a.map_counts;
    ra.map_grid = a.map_grid;
    ra.map_tau = a.map_tau;
    ra.tau = a.tau;
    ra.st = st;
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
  const MlpTcWeights gate_w = a.gate ? mlp_tc_weights(a.gate) : MlpTcWeights{};
  int ik_per_sm = 0;
  const bool ik_right = a.arm && ra.ik.arm.right;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
           &ik_per_sm, ik_right ? reach_ik_kernel<true> : reach_ik_kernel<false>, 128, 0)) != cudaSuccess)
    return e;
  const int ik_blocks = num_sms * (ik_per_sm > 0 ? ik_per_sm : 1);
  // ---- rounds. Round i: generation on s reads G[i % 3] (filled by round
  // i-1's generation and round i-2's reach stage) and writes G[(i+1) % 3]
  // and the reach queue Q[i % 2]; the reach stage of round i runs on side
  // stream i % 2 after it and writes G[(i+2) % 3]. Generation of round i
  // waits for the reach stage of round i-2, so reach stages overlap the next
  // rounds' generation and each other.
  cudaEvent_t* ev_gen = a.events + 1;
  cudaEvent_t* ev_reach = a.events + 1 + NR;
  if (NR > 0) {
    if ((e = cudaEventRecord(a.events[0], s)) != cudaSuccess) return e;
    for (int j = 0; j < 2; ++j)
      if ((e = cudaStreamWaitEvent(a.side[j], a.events[0], 0)) != cudaSuccess) return e;
  }
  for (int i = 0; i < NR; ++i) {
    if (i >= 2 && (e = cudaStreamWaitEvent(s, ev_reach[i - 2], 0)) != cudaSuccess) return e;
    g.list_in = G[i % 3];
    g.n_in = cnt_gen + i;
    g.list_gen = G[(i + 1) % 3];
    g.n_gen = cnt_gen + i + 1;
    g.list_reach = Q[i % 2];
    g.n_reach = cnt_reach + i;
    g.targets = targets[i % 2];  // free: this round waited for the reach stage of round i - 2
    g.counter = counters + i;
    if (a.timer) a.timer->begin(0, s);
    switch (cfg.a_per_lane) {
      case 1: launch_round<1>(g, a.ext_rel, grid, cfg.threads, smem, s); break;
      case 2: launch_round<2>(g, a.ext_rel, grid, cfg.threads, smem, s); break;
      default: launch_round<4>(g, a.ext_rel, grid, cfg.threads, smem, s); break;
    }
    if (a.timer) a.timer->end(s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaEventRecord(ev_gen[i], s)) != cudaSuccess) return e;
    cudaStream_t sr = a.side[i % 2];
    if ((e = cudaStreamWaitEvent(sr, ev_gen[i], 0)) != cudaSuccess) return e;
    ra.list_reach = Q[i % 2];
    ra.n_reach = cnt_reach + i;
    ra.targets = targets[i % 2];
    ra.list_ik = IK[i % 2];
    ra.n_ik = cnt_ik + 2 * i;
    ra.ik_cap = n;
    ra.list_gen = G[(i + 2) % 3];
    ra.n_gen = cnt_gen + i + 2;
    ra.claim = counters + NRmax + 1 + i;
    if (a.timer) a.timer->begin(1, sr);
    if (a.map_counts) reach_map_gate_kernel<<<small_blocks, 256, 0, sr>>>(ra);
    if (a.gate) {  // gate forward pass and decision in one launch
      e = launch_mlp_tc(gate_w, GateIO{ra}, n, a.status, num_sms, sr);
      if (e != cudaSuccess) return e;
    }
    if (a.timer) {
      a.timer->end(sr);
      a.timer->begin(2, sr);
    }
    if (ik_right)
      reach_ik_kernel<true><<<ik_blocks, 128, 0, sr>>>(ra);
    else
      reach_ik_kernel<false><<<ik_blocks, 128, 0, sr>>>(ra);
    if (a.timer) a.timer->end(sr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaEventRecord(ev_reach[i], sr)) != cudaSuccess) return e;
  }
  for (int i = NR - 2; i < NR; ++i)  // join the side streams
    if (i >= 0 && (e = cudaStreamWaitEvent(s, ev_reach[i], 0)) != cudaSuccess) return e;
  // ---- objects [k_begin, max_obj): one chained launch
  if (k_begin < K) {
    if (a.timer) a.timer->begin(0, s);
    ChainArgs ca;
    ca.order = a.order;
    ca.n = n;
    ca.k_begin = k_begin;
    ca.alive = st.alive;
    ca.counter = counters + NRmax;
    switch (cfg.a_per_lane) {
      case 1: launch_chain<1>(g, ca, a.ext_rel, grid, cfg.threads, smem, s); break;
      case 2: launch_chain<2>(g, ca, a.ext_rel, grid, cfg.threads, smem, s); break;
      default: launch_chain<4>(g, ca, a.ext_rel, grid, cfg.threads, smem, s); break;
    }
    if (a.timer) a.timer->end(s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace sc
