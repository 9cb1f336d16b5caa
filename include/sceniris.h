/*
 * sceniris.h - C ABI of libsceniris_b300.so, the B300 (sm_103a) hot path of
 * Sceniris (arXiv 2512.16896): batched pose sampling and collision rejection
 * over many scene variations at once, plus the reachability check.
 *
 * Conventions (apply to every call unless stated otherwise):
 *  - Units are metres and radians; frames are right-handed with z up.
 *  - Every array argument is a DEVICE pointer owned by the caller. Inputs are
 *    read-only during the call; outputs are written in full. The library
 *    never frees or keeps a caller pointer after the call is enqueued.
 *  - Calls are asynchronous on the context's CUDA stream unless they return
 *    host data. sc_ctx_synchronize() waits and reports device-side errors.
 *  - No call aborts and no exception crosses the ABI: failures return a
 *    non-zero sc_status and a message readable with sc_last_error().
 *  - Arguments are validated on the host before anything is launched; a call
 *    that returns SC_ERR_INVALID has enqueued no work.
 *  - Random numbers are Philox4x32-10 (Salmon et al., SC'11) with key = the
 *    64-bit seed (low word, high word) and a counter that names the draw,
 *    so every result is a pure function of (seed, indices) and is
 *    reproducible in any order, on any device and across calls.
 */
#ifndef SCENIRIS_H
#define SCENIRIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SC_OK = 0,
  SC_ERR_INVALID = 1,     /* bad argument; nothing was launched */
  SC_ERR_OOM = 2,         /* a context allocation failed */
  SC_ERR_CUDA = 3,        /* a CUDA runtime call failed (message has the CUDA error) */
  SC_ERR_TIMEOUT = 4,     /* a bounded device wait gave up */
  SC_ERR_UNSUPPORTED = 5, /* valid request this build does not handle (message says what) */
  SC_ERR_DEVICE = 6       /* a kernel latched an error in the device status word */
} sc_status;

/* ---------------------------------------------------------------- context */

/* Opaque context: one device, one stream, owns the library's scratch memory
 * (work counters, per-launch statistics, device status word). Not thread-safe:
 * use one context per host thread. */
typedef struct sc_ctx sc_ctx;

/* Create a context on `device` that enqueues on `cuda_stream` (a cudaStream_t;
 * NULL = the legacy default stream). *out receives the context.
 * Errors: SC_ERR_INVALID (out NULL, bad device), SC_ERR_CUDA, SC_ERR_OOM. */
sc_status sc_ctx_create(int device, void* cuda_stream, sc_ctx** out);
/* Destroy a context (NULL is ignored). Waits for the context's stream first. */
void sc_ctx_destroy(sc_ctx* ctx);
/* Change the stream later calls enqueue on. */
sc_status sc_ctx_set_stream(sc_ctx* ctx, void* cuda_stream);
/* Wait for the stream, then read and clear the device status word.
 * Returns SC_ERR_DEVICE if a kernel latched an error since the last check. */
sc_status sc_ctx_synchronize(sc_ctx* ctx);
/* Message of the last failing call on this host thread ("" if none). The
 * pointer stays valid until the next library call on the same thread. */
const char* sc_last_error(void);
/* ABI version (major * 10000 + minor * 100 + patch). */
int32_t sc_version(void);
/* Number of SMs of the context's device (read at creation). */
int32_t sc_ctx_num_sms(const sc_ctx* ctx);

/* ---------------------------------------------------------- scene batch */

/* Relation kinds stored in obj_rel (low 4 bits) and flags, see sc_sample_poses. */
enum {
  SC_REL_FREE = 0,
  SC_REL_ON_TOP = 1,
  SC_REL_NEXT_TO = 2,
  SC_REL_DIRECTIONAL = 3, /* one anchor, partial annulus (direction, half-angle, radii) */
  SC_REL_MIDDLE = 4,      /* two or more anchors: inside the polygon of their positions */
  SC_REL_INSIDE = 5,      /* on the inside support of an articulated part (reference = part index) */
  SC_REL_KIND_MASK = 0xF,
  SC_REL_REACH = 0x10,    /* reachability check (sc_generate) */
  SC_REL_LOCAL = 0x20,    /* DIRECTIONAL: direction angle in the anchor's frame */
  SC_REL_FACE_TO = 0x40   /* yaw faces the reference object instead of a uniform draw */
};

/* A batch of scene templates and the candidates (scene variations) drawn
 * from them, CSR-packed (Sec. IV-B: one transform per instance per edge; here
 * one pose per (candidate, object)). All pointers are DEVICE pointers.
 *
 *  tmpl_obj_off  int32 [T+1]  objects of template t: [tmpl_obj_off[t], tmpl_obj_off[t+1]);
 *                             template-local object k is global object tmpl_obj_off[t]+k.
 *                             Placement order = local index order.
 *  obj_sph_off   int32 [O+1]  collision spheres of object o (spheres of one template
 *                             are contiguous, in object order).
 *  sph_local     float [S][4] sphere (x, y, z, r) in its object's frame.
 *  obj_half      float [O][4] (Hx, Hy, Hz, rho): half extents of the object's box in its
 *                             frame (its bottom face rests on the support) and the
 *                             radius of its xy bounding circle. The box must contain
 *                             every sphere of the object: sc_generate skips pairs of
 *                             objects whose bounding balls (radius |H|) are apart.
 *  obj_rel       int32 [O]    kind | flags | (reference local index << 8); the
 *                             reference (parent / anchor / faced object) is an EARLIER
 *                             object.
 *  obj_rel_param float [O][4] (dmin, dmax, ratio_on_support, unused); DIRECTIONAL:
 *                             (min_r, max_r, ratio_on_support, theta), max_r may be +inf.
 *  obj_rel_dir   float [O]    DIRECTIONAL: direction angle of v (radians); may be NULL
 *                             when no object is DIRECTIONAL.
 *  obj_anchor_off int32 [O+1], obj_anchor int32 [A]: MIDDLE: the anchors (2..16
 *                             template-local indices of earlier objects, polygon order)
 *                             of object o are obj_anchor[obj_anchor_off[o] ..
 *                             obj_anchor_off[o+1]); may be NULL when no object is MIDDLE.
 *  Articulated parts (prismatic, e.g. drawers; all NULL / 0 when there are none):
 *  tmpl_part_off int32 [T+1]  parts of template t: [tmpl_part_off[t], tmpl_part_off[t+1]), at
 *                             most 16 per template; template-local part j is part
 *                             tmpl_part_off[t] + j.
 *  part_param    float [n_parts][12]  (ax, ay, az, qmin), (qmax, cx, cy, cz), (hx, hy, yaw, -):
 *                             joint axis (unit, template frame) and range; the part's
 *                             inside support at q = 0, a rectangle of half extents hx, hy
 *                             turned by yaw about z, centred at (cx, cy) on the plane z = cz.
 *                             At joint value q the part and its support move by q * axis.
 *  obb_part      int32 [n_obb] template-local part a world box moves with (-1: static).
 *  part_q        float [n_cand][max_parts] joint value of every part per candidate
 *                             (sc_sample_parts writes them); read by sampling (INSIDE),
 *                             collision and generation.
 *  tmpl_poly_off int32 [T+1], poly_verts float [V][2]: support polygon of template t
 *                             (closed, any orientation, >= 3 vertices) on the plane
 *                             z = tmpl_support_z[t].
 *  tmpl_obb_off  int32 [T+1], obb float [n_obb][12]: world boxes of template t,
 *                             each (cx, cy, cz, -, qx, qy, qz, qw, hx, hy, hz, -); the
 *                             quaternion need not be normalised. A box of an articulated
 *                             part (obb_part >= 0) is centred at c + q * axis for each
 *                             candidate's joint value q of that part.
 *  World meshes (NULL / 0 when there are none):
 *  tmpl_tri_off  int32 [T+1], tri float [n_tri][12]: triangles of template t's world
 *                             meshes, (ax, ay, az, -, bx, by, bz, -, cx, cy, cz, -) in the
 *                             world frame, at most 65,536 per template; 16-byte aligned.
 *                             A mesh is a surface: a sphere's distance to it is the
 *                             distance from its centre to the nearest point of any
 *                             triangle, minus r (unsigned; a sphere wholly inside a
 *                             closed mesh does not touch it).
 *  cand_tmpl_off int32 [T+1]  candidates of template t: [cand_tmpl_off[t], cand_tmpl_off[t+1]);
 *                             the global candidate index is the Philox counter word 0.
 *  tmpl_pose_off int64 [T+1]  start of template t's block in the pose array; candidate
 *                             c of template t (l = c - cand_tmpl_off[t]) owns the
 *                             n_t poses at tmpl_pose_off[t] + l * n_t + k.
 *  tmpl_base     float [T][4] robot base (x, y, z, yaw) per template; may be NULL
 *                             when no reachability check is requested.
 * Host-known sizes: n_* are the lengths above, max_obj / max_sph the largest object
 * and sphere count of any template (they size on-chip buffers: max_sph <= 8192,
 * max_obj <= 256, at most 64 vertices per polygon and 64 boxes per template). */
typedef struct {
  int32_t n_templates, n_objects, n_spheres, n_verts, n_obb, n_cand;
  int32_t max_obj, max_sph;
  const int32_t* tmpl_obj_off;
  const int32_t* obj_sph_off;
  const float* sph_local;
  const float* obj_half;
  const int32_t* obj_rel;
  const float* obj_rel_param;
  const int32_t* tmpl_poly_off;
  const float* poly_verts;
  const float* tmpl_support_z;
  const int32_t* tmpl_obb_off;
  const float* obb;
  const int32_t* cand_tmpl_off;
  const int64_t* tmpl_pose_off;
  const float* tmpl_base;
  const float* obj_rel_dir;
  const int32_t* obj_anchor_off;
  const int32_t* obj_anchor;
  int32_t n_parts, max_parts;
  const int32_t* tmpl_part_off;
  const float* part_param;
  const int32_t* obb_part;
  const float* part_q;
  int32_t n_tri;
  const int32_t* tmpl_tri_off;
  const float* tri;
} sc_scene_batch;

/* ------------------------------------------------------------- sampling */

typedef struct {
  uint64_t seed;        /* Philox key */
  int32_t max_attempts; /* proposals per object per try (point-in-polygon rejection), 1..1024 */
  int32_t retry;        /* try index r >= 0 (Philox counter word 2) */
  int32_t first_obj;    /* first template-local object to sample */
  int32_t n_obj;        /* how many objects from first_obj (clipped to each template) */
} sc_sample_params;

/* Sample object poses for the listed candidates (Sec. III position sampling,
 * Sec. IV-C batch sampling with the canonical polygon moved per instance,
 * Sec. IV-F relations and ratio_on_support). For every listed candidate c and
 * object k in [first_obj, first_obj + n_obj) (in order; earlier objects of c
 * must already hold poses), attempt a = 0..max_attempts-1 draws
 * u = Philox(seed; c, k, retry, a), u_i = (word_i >> 8) 2^-24, and proposes:
 *   FREE    xy uniform in the support polygon's bounding box;
 *   NEXT_TO around the anchor: angle 2 pi u0, distance rho_anchor + rho + dmin +
 *           (dmax - dmin) u1 (the annulus between min_r and max_r of Sec. IV-F, v = Null);
 *   ON_TOP  xy uniform in the parent's top face (its frame) moved by the parent's pose,
 *           z = parent z + parent Hz + Hz; accepted at attempt 0 (may overhang).
 *   DIRECTIONAL (one anchor, the partial annulus S_r of Sec. IV-F): area-uniform
 *           in the sector of half-angle theta around phi = dir (+ the anchor's yaw
 *           with SC_REL_LOCAL) between radii min_r and R = min(max_r, largest
 *           distance from the anchor to a corner of the support's bounding box):
 *           r = sqrt(min_r^2 + (R^2 - min_r^2) u0), angle phi + theta (2 u1 - 1),
 *           measured from the anchor's position;
 *   MIDDLE  (anchors A_1..A_n, Sec. IV-F 'middle'): n = 2: A_1 + u0 (A_2 - A_1);
 *           n >= 3: uniform in the anchors' bounding box, kept only inside the
 *           polygon A_1..A_n (crossing number, boundary inside).
 *   INSIDE  (Sec. IV-F 'inside', reference = part j): like ON_TOP on the part's
 *           inside support at the candidate's joint value (the rectangle shrunk
 *           by e = ratio_on_support * min(Hx, Hy) on each side), z = its plane + Hz;
 *           accepted at attempt 0.
 * FREE / NEXT_TO / DIRECTIONAL / MIDDLE proposals are accepted when inside the
 * support polygon and at least e = ratio_on_support * min(Hx, Hy) from its
 * boundary (S' = S_r n S); z = support + Hz. yaw = 2 pi u2, or with
 * SC_REL_FACE_TO the direction from the object towards the reference object,
 * atan2(y_ref - y, x_ref - x). The first accepted attempt wins; if none is
 * accepted the pose of the last attempt is written and the object counts as
 * failed. A relation that names a later object, a missing array, or a MIDDLE
 * object without 2..16 anchors latches a device error and is sampled free.
 * poses   float [P][4] (x, y, z, yaw), CSR layout of the batch; read (earlier
 *         objects) and written (sampled objects).
 * active  int32 [n_active] candidate indices to sample, or NULL for all n_cand
 *         (then n_active is ignored). Duplicates are not allowed.
 * sample_ok [n] u8: 1 if every sampled object of the candidate was accepted.
 * band      [n] u8: 1 if an accept/reject decision that fixed the outcome lay
 *           within 1e-5 m of the polygon boundary or of the erosion distance (or,
 *           for MIDDLE, of the anchor polygon's boundary).
 * Errors: SC_ERR_INVALID for NULL outputs, max_attempts outside 1..1024,
 * retry < 0, n_obj < 0 or sizes beyond the limits of sc_scene_batch. */
sc_status sc_sample_poses(sc_ctx* ctx, const sc_scene_batch* batch, const sc_sample_params* params,
                          const int32_t* active, int32_t n_active, float* poses, uint8_t* sample_ok,
                          uint8_t* band);

/* Joint value of every articulated part of the listed candidates (Sec. IV-B:
 * a batched forward kinematics sets each instance's articulation, e.g. how
 * far each drawer is open; a prismatic part's FK is the translation q * axis):
 * part_q[c * max_parts + j] = qmin + (qmax - qmin) u0 with
 * u = Philox(seed; c, 0xFFFF0000 + j, 0, 0), u0 as in sc_sample_poses.
 * part_q: device float [n_cand][max_parts]; entries of other candidates and
 * of j >= the template's part count are left unchanged. Errors:
 * SC_ERR_INVALID (NULL part_q, a batch without parts). */
sc_status sc_sample_parts(sc_ctx* ctx, const sc_scene_batch* batch, uint64_t seed, const int32_t* active,
                          int32_t n_active, float* part_q);

/* ------------------------------------------------------------ collision */

/* Launch shape and mode of the persistent collision kernel. A field left 0
 * (or a NULL config) takes the built-in default: {128, 1, 32, 8} for a batch
 * with max_sph <= 256, else {256, 4, 256, 4}. threads: 128..1024, multiple
 * of 32. a_per_lane: spheres each lane holds from the A side (1, 2 or 4).
 * seg_len: B-sphere segment per work unit (multiple of 8, 8..4096).
 * ctas_per_sm: resident CTAs per SM the grid is sized for (1..8).
 * decide_only: 0 = exact minimum distance for every candidate; 1 = decide
 * only: a candidate stops at its first pair closer than -1e-5 m (a certain
 * collision); collide and band are the same as in mode 0. min_dist is the
 * exact minimum inside the band (|d| <= 1e-5 m); a certain collision reports
 * some distance below -1e-5 m, a clear candidate some distance above 1e-5 m
 * or FLT_MAX.
 * stage_bulk: 0 = each lane loads the local spheres it transforms; 1 = one
 * thread copies the candidate's whole local sphere block (contiguous per
 * template) into shared memory with a bulk asynchronous copy
 * (cp.async.bulk, completion on an mbarrier) and the lanes transform it in
 * place. Results are identical; only the time differs (sc_collide only;
 * sc_generate ignores it). */
typedef struct {
  int32_t threads, a_per_lane, seg_len, ctas_per_sm;
  int32_t decide_only;
  int32_t stage_bulk;
} sc_collide_config;

/* Collision check of the listed candidates (Sec. IV-D; the paper uses cuRobo
 * meshes, this build per-object sphere sets against oriented boxes and world
 * triangle meshes). Each sphere
 * is moved by its object's pose (rotation about z by yaw, then translation),
 * and the minimum signed distance
 *   min( |c_i - c_j| - r_i - r_j  over spheres i of object a, j of object b,
 *                                  a < b, b >= first_new_obj,
 *        sdf_box(c_i) - r_i       over spheres of objects >= first_new_obj and
 *                                  the template's world boxes,
 *        dist_tri(c_i) - r_i      over the same spheres and the template's
 *                                  world triangles (unsigned distance) )
 * is reduced per candidate; the empty set gives FLT_MAX. Touching (d = 0) is
 * free: collide = min_dist < 0. band = |min_dist| <= 1e-5 m.
 * first_new_obj = 0 checks the whole scene; k re-checks object k (and later)
 * against everything placed before it (Sec. IV-D re-checks only what changed).
 * The kernel is persistent: CTAs take candidates from `active` in list order
 * through an atomic counter, so list the heaviest candidates first (see
 * sc_order_by_work) for ragged batches.
 * Outputs [n]: collide u8, min_dist float, band u8 (n = n_active, or n_cand
 * when active is NULL). A candidate the kernel cannot check (its template,
 * sphere, object, box or triangle counts beyond the limits, or a world box
 * naming a part its template lacks) gets collide = 0, min_dist = NaN and
 * band = 1, and the device error is latched into the context's status word.
 * Errors: SC_ERR_INVALID (NULL outputs, first_new_obj < 0, bad config, limits
 * of sc_scene_batch). */
sc_status sc_collide(sc_ctx* ctx, const sc_scene_batch* batch, const float* poses, const int32_t* active,
                     int32_t n_active, int32_t first_new_obj, uint8_t* collide, float* min_dist, uint8_t* band);
sc_status sc_collide_ex(sc_ctx* ctx, const sc_scene_batch* batch, const float* poses, const int32_t* active,
                        int32_t n_active, int32_t first_new_obj, const sc_collide_config* config, uint8_t* collide,
                        float* min_dist, uint8_t* band);

/* Number of sphere pairs (and sphere-box pairs) the last sc_collide,
 * sc_collide_ex or sc_generate call on this context evaluated in its inner
 * loop, read back after the call completes (synchronises the stream). Pairs
 * that the kernel proved unable to change the result are not counted. */
sc_status sc_collide_last_work(sc_ctx* ctx, int64_t* sphere_pairs, int64_t* sphere_box_pairs);
/* Point-triangle distances (ball culls and exact sphere distances) of the
 * last sc_collide / sc_collide_ex / sc_generate call (synchronises). */
sc_status sc_collide_last_tri_work(sc_ctx* ctx, int64_t* sphere_tri_pairs);

/* --------------------------------------------------------- reachability */

/* 7-DoF serial arm in standard Denavit-Hartenberg form:
 * T_i = Rz(q_i) Tz(d_i) Tx(a_i) Rx(alpha_i), tool frame = frame 7, joint
 * limits [qmin_i, qmax_i]. Targets are expressed in the arm's base frame. */
typedef struct {
  float dh_d[7], dh_a[7], dh_alpha[7], qmin[7], qmax[7];
} sc_arm;

typedef struct {
  float lambda;   /* damping (0.05) */
  float tol_pos;  /* success: position error <= tol_pos (metres) */
  float tol_rot;  /* and rotation angle <= tol_rot (radians, in (0, pi/2)) */
  int32_t iters;  /* DLS steps per seed (100) */
  int32_t seeds;  /* seeds per target, 1..32 */
  uint64_t seed;  /* Philox key of the seeds */
} sc_ik_params;

/* Can the arm reach each target? (Sec. IV-E: the sampled pose is rejected when
 * the robot cannot reach it; the paper looks the answer up in an RM4D map,
 * this build solves damped-least-squares IK.) Seeds q_j = qmin_j + (qmax_j -
 * qmin_j) u_j with u from Philox(seed; target id, seed index, j / 4, 0), word
 * j % 4. All seeds of a target iterate in lock step: check every seed (position
 * error <= tol_pos and angle(R^T R*) <= tol_rot), and stop at the first check
 * where one succeeds, returning the lowest such seed; otherwise take one step
 * dq = J^T (J J^T + lambda^2 I)^-1 e with e = [p* - p; 1/2 sum_k r_k x r*_k] and
 * clamp q to the limits. After `iters` steps and a final check the target is
 * unreachable and the seed with the smallest position error is returned.
 * targets    float [n][12] (R row-major, p), base frame.
 * target_ids uint32 [n] Philox counter word of each target, or NULL (= index).
 * reachable  u8 [n]; q_out float [n][7]; err float [n][2] = (position error,
 *            rotation angle) of the returned configuration.
 * band       u8 [n] or NULL: 1 when a success check of some seed, at any
 *            check up to the one that ended the target, could flip under a
 *            perturbation of 1e-5 (both errors at most 1e-5 above their
 *            tolerances and one within 1e-5 of its tolerance). FP32 and FP64
 *            solvers can decide such targets differently.
 * Errors: SC_ERR_INVALID (NULL pointers, seeds outside 1..32, iters < 0,
 * non-positive tolerances or tol_rot >= pi/2). */
sc_status sc_ik_reach(sc_ctx* ctx, const sc_arm* arm, const sc_ik_params* params, const float* targets,
                      const uint32_t* target_ids, int32_t n, uint8_t* reachable, float* q_out, float* err,
                      uint8_t* band);

/* Seed-iterations (checks evaluated x seeds, summed over targets) of the
 * last sc_ik_reach call on this context, read back after the call completes
 * (synchronises the stream). */
sc_status sc_ik_last_work(sc_ctx* ctx, int64_t* seed_iterations);

/* One damped-least-squares step (the update of sc_ik_reach, including the
 * clamp) for n independent (target, configuration) pairs: q_out[i] = step of
 * q_in[i] towards targets[i]. tool (optional, float [n][12]) receives the
 * forward kinematics of q_in[i] (R row-major, p). */
sc_status sc_ik_dls_step(sc_ctx* ctx, const sc_arm* arm, float lambda, const float* targets, const float* q_in,
                         int32_t n, float* q_out, float* tool);

/* ------------------------------------------------------------ surrogate */

/* Learned reachability gate (not in the paper, which queries RM4D for
 * Sec. IV-E): an MLP 9 -> 256 -> 256 -> 256 -> 1 with SiLU activations on the
 * features x = (p, R[:,0], R[:,1]) of a target (position and the first two
 * columns of its rotation, base frame), standardised by a stored mean / std.
 * BF16 weights and activations on the tensor cores, FP32 accumulation, biases
 * and Adam state; the bf16 rounding points are: standardised input, every
 * SiLU output, the weight copies, and every dL/da in the backward pass.
 * Parameters are packed FP32: W1 [256][9], b1 [256], W2 [256][256], b2, W3
 * [256][256], b3, W4 [256], b4 [1] (sc_mlp_param_count() = 134401). */
typedef struct sc_mlp sc_mlp;

int32_t sc_mlp_param_count(void);
/* New network: weights and biases U(-1/sqrt(fan_in), +1/sqrt(fan_in)) from
 * Philox(seed), mean 0 / std 1 standardisation, threshold 0, Adam step 0. */
sc_status sc_mlp_create(sc_ctx* ctx, uint64_t seed, sc_mlp** out);
void sc_mlp_destroy(sc_mlp* mlp);
/* Copy parameters / standardisation / threshold to or from HOST memory (any
 * pointer may be NULL to skip it). Synchronises the context's stream. */
sc_status sc_mlp_get(sc_ctx* ctx, const sc_mlp* mlp, float* params, float* mu, float* sigma, float* tau);
sc_status sc_mlp_set(sc_ctx* ctx, sc_mlp* mlp, const float* params, const float* mu, const float* sigma, float tau);
/* logits[i] of targets[i] (float [n][12], device). */
sc_status sc_surrogate_infer(sc_ctx* ctx, const sc_mlp* mlp, const float* targets, int32_t n, float* logits);
/* Gradients of the mean binary cross-entropy on logits,
 * BCE(z, y) = max(z, 0) - z y + log(1 + exp(-|z|)), over all n targets
 * (labels u8 [n], 1 = reachable): grads (device, packed like the parameters,
 * may be NULL) and the loss (host, may be NULL). n <= 2^20. */
sc_status sc_surrogate_grads(sc_ctx* ctx, sc_mlp* mlp, const float* targets, const uint8_t* labels, int32_t n,
                             float* grads, float* loss);

typedef struct {
  int32_t epochs, batch;  /* passes over the data; minibatch size (16..65536) */
  float lr, beta1, beta2, eps;  /* Adam (1e-3, 0.9, 0.999, 1e-8) */
  uint64_t seed;          /* epoch shuffles */
} sc_train_params;

/* One Adam step with the given gradients (device, packed; NULL = the last
 * gradients sc_surrogate_grads or training computed):
 * m = b1 m + (1 - b1) g; v = b2 v + (1 - b2) g^2;
 * w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps). */
sc_status sc_mlp_adam_step(sc_ctx* ctx, sc_mlp* mlp, const float* grads, const sc_train_params* params);
/* One training step on n labelled targets (device, rows in the given order):
 * the gradients of sc_surrogate_grads and the Adam update of
 * sc_mlp_adam_step in one pass (the weight-gradient kernel applies the
 * update to each gradient as it writes it), leaving the same parameters,
 * moments, step count and gradients as those two calls. The batch limits of
 * sc_surrogate_grads apply (params->batch is not used). loss (host, may be
 * NULL) receives the mean BCE. */
sc_status sc_mlp_train_step(sc_ctx* ctx, sc_mlp* mlp, const float* targets, const uint8_t* labels, int32_t n,
                            const sc_train_params* params, float* loss);
/* Train on n labelled targets (device): a fresh network (Adam step 0) first
 * takes its standardisation from the training set; every epoch visits the
 * targets in a shuffled order (an affine permutation mod n) in whole
 * minibatches, each one gradient + Adam step. loss_per_epoch (host, may be
 * NULL) receives the mean BCE of each epoch's last minibatch. */
sc_status sc_surrogate_train(sc_ctx* ctx, sc_mlp* mlp, const float* targets, const uint8_t* labels, int32_t n,
                             const sc_train_params* params, float* loss_per_epoch);
/* Set the gate threshold to the largest tau whose recall on these labelled
 * targets is >= min_recall (ties included: keep z >= tau); report the recall
 * and the fraction of targets that pass. */
sc_status sc_surrogate_tune_threshold(sc_ctx* ctx, sc_mlp* mlp, const float* targets, const uint8_t* labels, int32_t n,
                                      float min_recall, float* tau, float* recall, float* pass_rate);
/* Checkpoint: parameters, Adam moments and step, standardisation and
 * threshold in one little-endian file ("SCMLP001" header). */
sc_status sc_mlp_save(sc_ctx* ctx, const sc_mlp* mlp, const char* path);
sc_status sc_mlp_load(sc_ctx* ctx, const char* path, sc_mlp** out);

/* ---------------------------------------------- 4D reachability map */

/* A reachability map in the manner of RM4D, the map the paper queries for
 * its reachability check (Sec. IV-E), built here from labelled IK outcomes
 * (sc_ik_reach) instead of the paper's precomputed map. A target (R, p) in
 * the base frame ([12] floats: R row-major, then p) falls in one cell of a
 * 4D grid over
 *   - its height p_z, in [z_lo, z_hi), nz bins;
 *   - the cosine a_z of its approach axis a = R e_z, in [-1, 1], nc bins
 *     (the top bin closed);
 *   - its position (x*, y*) in the frame turned about the base z axis until
 *     the azimuth reference h lies on +x, each in [-r_max, r_max), nxy bins.
 *     h = the horizontal direction of a, or, for a vertical approach
 *     (a_x^2 + a_y^2 <= 1e-6), of the tool x axis R e_x.
 * Every key step is one IEEE-rounded FP32 operation in a fixed order:
 *   u = tilted ? (a_x, a_y) : ((R e_x)_x, (R e_x)_y); n2 = u_x u_x + u_y u_y;
 *   inv = 1 / sqrt(n2); h = u inv; x* = p_x h_x + p_y h_y; y* = p_y h_x - p_x h_y;
 *   bin = floor((v - lo) s) with s = nz / (z_hi - z_lo), nc / 2, nxy / (2 r_max)
 * (each s one FP32 division on the host). A target outside the grid, or
 * with n2 = 0 or a NaN, has no cell. Each cell holds two counts (uint32):
 * reachable labels and labels. */
typedef struct {
  int32_t nz, nc, nxy;   /* bins; nz * nc * nxy^2 <= 2^27 */
  float z_lo, z_hi;      /* height range (metres), z_hi > z_lo */
  float r_max;           /* half-width of the x*, y* range (metres), > 0 */
} sc_rmap_params;

typedef struct sc_rmap sc_rmap;

/* New map with zero counts and threshold 1 (a target passes when its score
 * is >= the threshold). SC_ERR_INVALID for bad params, SC_ERR_OOM. */
sc_status sc_rmap_create(sc_ctx* ctx, const sc_rmap_params* params, sc_rmap** out);
void sc_rmap_destroy(sc_rmap* map);
/* Number of cells (0 for NULL). */
int64_t sc_rmap_cells(const sc_rmap* map);
/* Add n labelled targets (device: targets float [n][12], labels u8 [n], 1 =
 * reachable) to the counts; targets without a cell are skipped. Counts are
 * integers, so the result does not depend on the order of the additions. */
sc_status sc_rmap_build(sc_ctx* ctx, sc_rmap* map, const float* targets, const uint8_t* labels, int32_t n);
/* score[i] (device u16 [n]) = floor(65535 * reachable / labels) of target
 * i's cell; 65535 for a cell without labels (no evidence there, and a gate
 * must not reject without it); 0 for a target without a cell (choose the
 * grid to cover the arm's workspace). */
sc_status sc_rmap_query(sc_ctx* ctx, const sc_rmap* map, const float* targets, int32_t n, uint16_t* score);
/* Set the threshold to the largest tau whose recall on these labelled
 * targets is >= min_recall (ties included: pass when score >= tau) and report
 * the recall and the fraction of targets that pass. Synchronises. */
sc_status sc_rmap_tune_threshold(sc_ctx* ctx, sc_rmap* map, const float* targets, const uint8_t* labels, int32_t n,
                                 float min_recall, int32_t* tau, float* recall, float* pass_rate);
/* Set the threshold directly (0 passes every target, 65536 none). */
sc_status sc_rmap_set_threshold(sc_rmap* map, int32_t tau);
/* Counts to HOST memory, uint32 [cells][2] = (reachable, labels) per cell
 * in the order cell = ((iz * nc + ic) * nxy + ix) * nxy + iy. Synchronises. */
sc_status sc_rmap_get_counts(sc_ctx* ctx, const sc_rmap* map, uint32_t* counts);

/* ----------------------------------------------------------- generation */

typedef struct {
  uint64_t seed;        /* Philox key of the pose draws */
  int32_t max_attempts; /* proposals per object per try, 1..1024 (as sc_sample_params) */
  int32_t max_retries;  /* retries per object after its first try, 0..1000 (the paper uses 10) */
  int32_t use_graph;    /* 1: capture the launch sequence into a CUDA graph once (per batch, order,
                           output pointers, retries and launch shape) and replay it; 0: launch eagerly */
} sc_gen_params;

/* Optional reachability stage of sc_generate (Sec. IV-E: a sampled pose the
 * robot cannot reach is rejected). Objects with the SC_REL_REACH flag are,
 * after a collision-free try, checked for a top-down grasp: position = top
 * centre of the object's box, tool z = -world z, tool x along the object's
 * yaw, expressed in the template's robot base frame (tmpl_base). With a gate,
 * the surrogate's logit must reach the gate's threshold (sc_mlp_set /
 * sc_surrogate_tune_threshold) first; a rejected try retries like a
 * collision. Exact IK (sc_ik_reach semantics, seeds keyed by (candidate,
 * seed, block, object << 16 | try)) then decides; an unreachable grasp
 * retries too. Every emitted scene is thus verified by exact collision and
 * exact IK decisions; the gate only skips IK on tries it predicts to fail.
 * Before any of this, right after the pose is sampled, a try whose grasp
 * target lies beyond the arm's reach fails without collision checks, gate
 * or IK: its position farther than |a_0| + sum_{i>0} sqrt(a_i^2 + d_i^2)
 * + tol_pos from (0, 0, d_0) of the base frame, or its wrist point t - R v
 * (v = (a_6, d_6 sin alpha_6, d_6 cos alpha_6)) farther than the same sum
 * over links 1..5 + tol_pos + 2 sin(tol_rot / 2) |v| (each with the band's
 * 1e-5 and a 1e-4 margin). The exact IK would fail such a target with no
 * check in its band, so valid flags and tries are those of running it.
 * A 4D reachability map (sc_rmap) can gate instead of the surrogate: the
 * grasp target's map score must reach the map's threshold
 * (sc_rmap_tune_threshold), decided where the target is formed. */
typedef struct {
  const sc_arm* arm;       /* NULL: no reachability stage */
  const sc_ik_params* ik;  /* exact IK settings */
  const sc_mlp* gate;      /* NULL: exact IK on every collision-free try */
  const sc_rmap* map;      /* map gate instead (at most one of gate and map) */
} sc_gen_reach;

/* Generate scenes: the paper's placement loop (Sec. IV-A, Fig. 2) over the
 * listed candidates. Objects are placed in template order. For object k each
 * candidate still alive tries r = 0..max_retries: sample object k's pose with
 * try index r (exactly sc_sample_poses for that object), then check object k
 * against objects 0..k-1, the world boxes (part boxes at the candidate's
 * joint values) and the world triangles (the decision of sc_collide with
 * first_new_obj = k; only the scenes that retry are re-checked, Sec. IV-D).
 * Joint values are read from batch->part_q, written before the call (for
 * example by sc_sample_parts).
 * The first try whose proposal is accepted and collision-free fixes the
 * pose; a candidate that exhausts its tries is invalid (Sec. V-A) and its
 * later objects are not placed.
 * order   int32 [n_order] candidates to generate (NULL: all n_cand; then
 *         n_order is ignored); the heaviest first balances the first steps.
 * config  launch shape of the per-step kernel (NULL: default {256, 1, 256, 4};
 *         zero fields keep their default; decide_only is implied).
 * Outputs, indexed by candidate (only listed candidates are written):
 * poses   float [P][4] CSR pose layout; objects never placed are NaN.
 * valid   u8 [n_cand]: 1 when every object was placed.
 * band    u8 [n_cand]: 1 when any decision on the candidate's path (a support
 *         test of an attempt that fixed an outcome, a minimum distance, or
 *         an IK success check as sc_ik_reach's band) lay within 1e-5 of its
 *         threshold.
 * tries   int32 [n_cand]: tries spent over all objects.
 * reach   optional reachability stage (NULL: none).
 * q_reach float [P][7] (may be NULL): for every reach-checked object that was
 *         placed, the IK solution that verified it (pose-slot layout).
 * Schedule: objects before the last reach-flagged one run in rounds — each
 * round one generation launch over the candidates due a try (each candidate
 * carries its own object and try), then the reach stage of that round on one
 * of two context-owned side streams, overlapping the next rounds (at most
 * 2 x reach objects x (max_retries + 1) rounds; empty ones exit at once);
 * the remaining objects run in one launch where a warp takes a candidate
 * through all its later objects and tries. All of it is one graph launch
 * when use_graph = 1 (the seed is read from device memory, so a replay with
 * a new seed is not re-captured); the side streams are joined back into the
 * caller's stream before the call's work ends.
 * The first call (or one with more candidates than before) allocates the
 * context's generation scratch (candidate lists, per-candidate state,
 * counters, per-call tables); later calls reuse it. A call with
 * use_graph = 1 must not itself be issued inside another stream capture.
 * Errors: SC_ERR_INVALID (NULL outputs, max_attempts / max_retries out of
 * range, bad config, batch limits), SC_ERR_OOM, SC_ERR_CUDA. */
sc_status sc_generate(sc_ctx* ctx, const sc_scene_batch* batch, const sc_gen_params* params, const int32_t* order,
                      int32_t n_order, const sc_collide_config* config, const sc_gen_reach* reach, float* poses,
                      uint8_t* valid, uint8_t* band, int32_t* tries, float* q_reach);

/* Work and time of the last sc_generate call (synchronises the stream). */
typedef struct {
  int64_t sphere_pairs;        /* sphere pairs the collision stage evaluated (after the cull) */
  int64_t sphere_box_pairs;
  int64_t ik_solves;           /* targets the exact IK solved */
  int64_t gate_rejections;     /* tries the learned gate sent back without IK */
  int64_t ik_seed_iterations;  /* sum over solves of seeds x (checks made) */
  float ms_stage[3];           /* with timing on: device time of the generation launches, the
                                  grasp-target + gate launches, and the IK launches (stages run
                                  concurrently on different streams, so these may overlap) */
  int32_t launches_stage[3];
  int64_t cull_tests;          /* sphere-vs-bounding-ball tests of the exact sphere-level cull
                                  (and triangle-chunk ball tests) */
  int64_t exhaustive_pairs;    /* sphere pairs of every decision without any cull (object k's
                                  spheres x all spheres of the objects placed before it) */
  int64_t sphere_tri_pairs;    /* point-triangle distances: ball culls and exact sphere distances */
  int64_t reach_bound_rejections; /* tries of reach-flagged objects whose grasp target lies beyond
                                     the arm's reach (see sc_gen_reach): they fail right after
                                     sampling, without collision checks, gate or IK */
} sc_gen_stats;
sc_status sc_generate_stats(sc_ctx* ctx, sc_gen_stats* out);
/* Turn per-stage CUDA-event timing of sc_generate on or off (a graph captured
 * with one setting is re-captured for the other). */
sc_status sc_ctx_set_timing(sc_ctx* ctx, int32_t on);
/* Per-launch trace of the last timed sc_generate call (timing on): for each
 * timed launch i < *n (at most cap are written), stage[i] (0 generation,
 * 1 grasp targets + gate, 2 exact IK), start_ms[i] and end_ms[i] relative to
 * the first recorded event. HOST arrays [cap]. Synchronises the stream. */
sc_status sc_generate_trace(sc_ctx* ctx, int32_t cap, int32_t* n, int32_t* stage, float* start_ms, float* end_ms);

/* Host helper: order candidates heaviest first (LPT) by their exhaustive
 * pair count. HOST arrays: tmpl_obj_off [T+1], obj_sph_off [O+1],
 * cand_tmpl_off [T+1]; out_order [n_cand] receives candidate indices. */
sc_status sc_order_by_work(int32_t n_templates, const int32_t* tmpl_obj_off, const int32_t* obj_sph_off,
                           const int32_t* cand_tmpl_off, int32_t* out_order);

/* ------------------------------------------------- allocation-free variant */

/* Largest candidate list one sc_collide_noalloc call accepts: CTAs claim
 * candidates through a 32-bit work counter that runs past the end by up to
 * the grid size, and the kernel reads it as a signed index. */
#define SC_NOALLOC_MAX_ITEMS (1 << 30)

/* The collision check of sc_collide for callers that cannot allocate device
 * memory. The paper has no counterpart: this exists for users of the library.
 * Creating an sc_ctx calls cudaMalloc for the kernel's scratch (its work
 * counter and pair statistics); some callers cannot do that, for example code
 * whose device memory is owned by a framework's own pool, per-frame loops in
 * which a cudaMalloc would synchronise the device and stall, or code that
 * keeps no library context. This entry point takes no context and allocates
 * nothing: the scratch is a 256-byte array compiled into the library, which
 * every GPU that loads the library holds until the process exits.
 *  - Runs on the CURRENT device, enqueued on `cuda_stream` (a cudaStream_t;
 *    NULL = legacy default stream).
 *  - The first call on a device looks up that array's device address
 *    (cudaGetSymbolAddress) and the SM count; make that first call before any
 *    stream capture on that device. The address is kept for the life of the
 *    process: do not call this entry point on a device after a
 *    cudaDeviceReset of it (the library's module, and the array with it, is
 *    loaded again at a new address).
 *  - Every call shares the one array per device; the launch zeroes the work
 *    counter before the kernel runs. Calls that overlap on the GPU (on two
 *    streams, or from two host threads at once) race on it and must not be
 *    issued; calls in order on one stream are fine.
 *  - Arguments, layouts, outputs and results are those of sc_collide (the same
 *    kernel, default launch shape). Candidates the kernel's own checks reject
 *    come back with min_dist = NaN and band = 1 (no status word is kept).
 *  - Errors: SC_ERR_INVALID for the cases of sc_collide and for more than
 *    SC_NOALLOC_MAX_ITEMS candidates; SC_ERR_CUDA if the set-up or the launch
 *    fails. Messages through sc_last_error(). */
sc_status sc_collide_noalloc(void* cuda_stream, const sc_scene_batch* batch, const float* poses,
                             const int32_t* active, int32_t n_active, int32_t first_new_obj, uint8_t* collide,
                             float* min_dist, uint8_t* band);

#ifdef __cplusplus
}
#endif
#endif /* SCENIRIS_H */
