// Sceniris hot-path oracle: plain, slow, FP64 CPU implementation.
//
// THIS IS TEST INFRASTRUCTURE. Only the test suite, the smoke check and the
// benchmark's CPU-baseline leg may load it. The product path (the CUDA library
// under paper_2512_16896_b300/) never calls, links or includes anything here,
// and this file includes nothing from there.
//
// Every quantity is computed in double precision from the same float32 input
// arrays the GPU library receives. Nothing is blocked, fused or reordered
// beyond the definitions below: all pairs are evaluated, every PIP test walks
// every edge, every IK step is the textbook formula.
//
// Paper: Sceniris: A Fast Procedural Scene Generation Framework (arXiv 2512.16896).
//   Sec. III  (Scene Synthesizer)  rejection sampling loop, 2D position in a support polygon
//                                  plus a z offset, yaw rule.
//   Sec. IV-A (System overview)    per-object sample -> collision check -> limited retries.
//   Sec. IV-B (Batched repr.)      N transforms per scene-graph edge.
//   Sec. IV-C (Batch sampling)     canonical polygon sampled once, rigidly transformed per instance.
//   Sec. IV-D (Collision checking) batch check, re-check only the scenes that retry.
//   Sec. IV-E (Reachability)       reject a sampled pose the robot cannot reach.
//   Sec. IV-F (Spatial relations)  annulus min_r/max_r (unnumbered equation), ratio_on_support erosion.
//   Sec. V-A  (Experiments)        10 retries per object, failing instances marked invalid.
//
// Parity status of each function is stated beside it ("pinned by ..." names the
// non-self test that fixes it; see tests/test_oracle_pins.py).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <cfloat>
#include <thread>
#include <vector>
#include <algorithm>
#include <array>

extern "C" {

// ---------------------------------------------------------------------------
// Philox4xW-10 counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel
// random numbers: as easy as 1, 2, 3", SC'11). One template serves the 32-bit
// and the 64-bit word widths so that the 64-bit instance can be checked against
// numpy.random.Philox (a library implementation of Philox4x64-10): the round
// structure, the S-box permutation and the key schedule are shared code.
// Pinned by: 4x64 instance == numpy.random.Philox outputs; 4x32 instance ==
// the published Philox4x32-10 known-answer vectors (tests/golden), plus
// uniformity / independence statistics.
// ---------------------------------------------------------------------------
}  // extern "C"

template <typename W> struct PhiloxConst;
template <> struct PhiloxConst<uint32_t> {
  // multipliers and Weyl key increments for W = 32 as published in SC'11
  static constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  static constexpr uint32_t K0 = 0x9E3779B9u, K1 = 0xBB67AE85u;
  static void mulhilo(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
  }
};
template <> struct PhiloxConst<uint64_t> {
  static constexpr uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  static constexpr uint64_t K0 = 0x9E3779B97F4A7C15ull, K1 = 0xBB67AE8584CAA73Bull;
  static void mulhilo(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
  }
};

// One Philox4 round: two multiplications, the high halves XORed with the other
// two counter words and the key, the result permuted (SC'11, Sec. 5 of that paper).
template <typename W>
static void philox4_round(W ctr[4], const W key[2]) {
  W hi0, lo0, hi1, lo1;
  PhiloxConst<W>::mulhilo(PhiloxConst<W>::M0, ctr[0], &hi0, &lo0);
  PhiloxConst<W>::mulhilo(PhiloxConst<W>::M1, ctr[2], &hi1, &lo1);
  W out0 = hi1 ^ ctr[1] ^ key[0];
  W out1 = lo1;
  W out2 = hi0 ^ ctr[3] ^ key[1];
  W out3 = lo0;
  ctr[0] = out0; ctr[1] = out1; ctr[2] = out2; ctr[3] = out3;
}

template <typename W>
static void philox4_10(const W in_ctr[4], const W in_key[2], W out[4]) {
  W ctr[4] = {in_ctr[0], in_ctr[1], in_ctr[2], in_ctr[3]};
  W key[2] = {in_key[0], in_key[1]};
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {  // key bump between rounds
      key[0] = (W)(key[0] + PhiloxConst<W>::K0);
      key[1] = (W)(key[1] + PhiloxConst<W>::K1);
    }
    philox4_round<W>(ctr, key);
  }
  for (int i = 0; i < 4; ++i) out[i] = ctr[i];
}

extern "C" {

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  philox4_10<uint32_t>(ctr, key, out);
}
void or_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  philox4_10<uint64_t>(ctr, key, out);
}

// Uniform in [0,1) from the top 24 bits of a 32-bit word: exact in float and double.
static double u01(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

// Draw for one (candidate, object, retry, attempt) counter: 4 uniforms.
// key = (seed low word, seed high word); counter = (cand, obj, retry, attempt).
static void draw4(uint64_t seed, uint32_t cand, uint32_t obj, uint32_t retry, uint32_t attempt, double u[4]) {
  uint32_t ctr[4] = {cand, obj, retry, attempt};
  uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
  uint32_t x[4];
  philox4_10<uint32_t>(ctr, key, x);
  for (int i = 0; i < 4; ++i) u[i] = u01(x[i]);
}

void or_uniform4(uint64_t seed, uint32_t cand, uint32_t obj, uint32_t retry, uint32_t attempt, double* u) {
  draw4(seed, cand, obj, retry, attempt, u);
}

// ---------------------------------------------------------------------------
// Point in polygon (Sec. III, "Position sampling": a 2D point is sampled inside
// the support polygon). Crossing-number test on the closed polygon; a point on
// the boundary counts as inside. Also returns the unsigned Euclidean distance
// from the point to the polygon boundary (minimum over edge segments), which
// drives both the ratio_on_support erosion (Sec. IV-F) and the 1e-5 m decision
// band. Pinned by: unit square, concave L-shape, vertices/edges, CW vs CCW.
// ---------------------------------------------------------------------------
static double seg_dist(double px, double py, double ax, double ay, double bx, double by) {
  double ex = bx - ax, ey = by - ay;
  double len2 = ex * ex + ey * ey;
  double t = 0.0;
  if (len2 > 0.0) t = ((px - ax) * ex + (py - ay) * ey) / len2;
  if (t < 0.0) t = 0.0;
  if (t > 1.0) t = 1.0;
  double qx = ax + t * ex - px, qy = ay + t * ey - py;
  return std::sqrt(qx * qx + qy * qy);
}

int or_point_in_polygon(const double* vx, const double* vy, int n, double px, double py, double* dist) {
  double dmin = INFINITY;
  int crossings = 0;
  for (int i = 0; i < n; ++i) {
    int j = (i + 1) % n;
    double d = seg_dist(px, py, vx[i], vy[i], vx[j], vy[j]);
    if (d < dmin) dmin = d;
    // edge (i,j) crosses the horizontal ray to +x from p?
    bool yi_above = vy[i] > py, yj_above = vy[j] > py;
    if (yi_above != yj_above) {
      double xcross = vx[i] + (py - vy[i]) * (vx[j] - vx[i]) / (vy[j] - vy[i]);
      if (px < xcross) crossings++;
    }
  }
  if (dist) *dist = dmin;
  if (dmin == 0.0) return 1;  // on the boundary
  return crossings & 1;
}

// ---------------------------------------------------------------------------
// Scene batch description (host copies of the arrays the GPU library takes).
// ---------------------------------------------------------------------------
typedef struct {
  int32_t n_templates, n_objects, n_spheres, n_verts, n_obb, n_cand;
  const int32_t* tmpl_obj_off;   // [T+1] objects of template t: [off[t], off[t+1])
  const int32_t* obj_sph_off;    // [O+1]
  const float* sph_local;        // [S][4] x,y,z,r in the object frame
  const float* obj_half;         // [O][4] AABB half extents Hx,Hy,Hz and xy radius rho
  const int32_t* obj_rel;        // [O] kind | (reference local index << 8)
  const float* obj_rel_param;    // [O][4] dmin, dmax, ratio_on_support, unused
  const int32_t* tmpl_poly_off;  // [T+1]
  const float* poly_verts;       // [V][2]
  const float* tmpl_support_z;   // [T]
  const int32_t* tmpl_obb_off;   // [T+1]
  const float* obb;              // [n_obb][12] centre(x,y,z,-), quaternion(x,y,z,w), half(x,y,z,-)
  const int32_t* cand_tmpl_off;  // [T+1] candidates of template t: [off[t], off[t+1])
  const float* tmpl_base;        // [T][4] robot base pose x,y,z,yaw (reachability only; may be NULL)
  const float* obj_rel_dir;      // [O] direction angle of a DIRECTIONAL relation (may be NULL)
  const int32_t* obj_anchor_off; // [O+1] anchors of a MIDDLE relation (may be NULL)
  const int32_t* obj_anchor;     // [A] template-local indices of earlier objects
  int32_t n_parts, max_parts;    // articulated (prismatic) parts; 0 when there are none
  const int32_t* tmpl_part_off;  // [T+1] parts of template t
  const float* part_param;       // [n_parts][12] axis, qmin | qmax, support centre | half x, y, yaw, -
  const int32_t* obb_part;       // [n_obb] template-local part a box moves with, -1 static (may be NULL)
  const float* part_q;           // [n_cand][max_parts] joint values
  int32_t n_tri;                 // world mesh triangles; 0 when there are none
  const int32_t* tmpl_tri_off;   // [T+1] triangles of template t
  const float* tri;              // [n_tri][12] vertices a | b | c (x, y, z, -)
} or_scene;

enum {
  REL_FREE = 0, REL_ON_TOP = 1, REL_NEXT_TO = 2, REL_DIRECTIONAL = 3, REL_MIDDLE = 4, REL_INSIDE = 5,
  REL_KIND_MASK = 0xF,
  REL_REACH = 0x10, REL_LOCAL = 0x20, REL_FACE_TO = 0x40
};

static const double BAND = 1e-5;         // decision band of the parity contract (metres)
static const double TWO_PI = 6.283185307179586476925286766559;

static int template_of(const or_scene* s, int c) {
  // plain linear scan over the candidate ranges
  for (int t = 0; t < s->n_templates; ++t)
    if (c >= s->cand_tmpl_off[t] && c < s->cand_tmpl_off[t + 1]) return t;
  return -1;
}

// Offset of candidate c's first pose in the CSR pose array: templates are laid
// out one after another, each holding n_cand(t) x n_obj(t) poses.
static int64_t pose_offset(const or_scene* s, int c, int t) {
  int64_t off = 0;
  for (int u = 0; u < t; ++u)
    off += (int64_t)(s->cand_tmpl_off[u + 1] - s->cand_tmpl_off[u]) *
           (s->tmpl_obj_off[u + 1] - s->tmpl_obj_off[u]);
  return off + (int64_t)(c - s->cand_tmpl_off[t]) * (s->tmpl_obj_off[t + 1] - s->tmpl_obj_off[t]);
}

int64_t or_pose_offset(const or_scene* s, int c) { return pose_offset(s, c, template_of(s, c)); }

// Number of articulated parts of template t (0 without parts).
static int parts_of(const or_scene* s, int t) {
  if (s->n_parts <= 0 || !s->tmpl_part_off) return 0;
  return s->tmpl_part_off[t + 1] - s->tmpl_part_off[t];
}

// Joint value of template-local part j of candidate c (a prismatic joint:
// the part translates by q along its axis).
static double part_value(const or_scene* s, int c, int j) { return s->part_q[(int64_t)c * s->max_parts + j]; }

// Support-polygon acceptance for a sampled xy (Sec. III position sampling +
// Sec. IV-F ratio_on_support): inside the polygon and at least e from its
// boundary, e = ratio * half of the shorter edge of the object's projection.
// band = the decision is within 1e-5 m of flipping.
static bool support_accept(const or_scene* s, int t, double x, double y, double e, bool* band) {
  int v0 = s->tmpl_poly_off[t], nv = s->tmpl_poly_off[t + 1] - v0;
  std::vector<double> vx(nv), vy(nv);
  for (int i = 0; i < nv; ++i) {
    vx[i] = s->poly_verts[2 * (v0 + i)];
    vy[i] = s->poly_verts[2 * (v0 + i) + 1];
  }
  double dist;
  int inside = or_point_in_polygon(vx.data(), vy.data(), nv, x, y, &dist);
  *band = (dist <= BAND) || (inside && std::fabs(dist - e) <= BAND);
  return inside && dist >= e;
}

// Sample the pose of object k (template-local index) of candidate c for one
// try `retry`, given the poses of earlier objects already in pose[].
// pose[k] <- (x, y, z, yaw). Returns accepted; *band set if any attempt that
// decided the outcome lies in the decision band.
//   FREE    : Sec. III + IV-C, 2D point uniform in the support polygon (bounding-box
//             proposal, PIP rejection), z = support plane + half height, yaw uniform.
//   ON_TOP  : Sec. IV-C canonical polygon + per-instance rigid transform: the pivot
//             is uniform in the parent's top face (its own frame), then moved by the
//             parent's pose; 'on' support (Sec. IV-F) is the parent's top face.
//   NEXT_TO : Sec. IV-F one-anchor relation with v = Null: the annulus between
//             min_r = contact + dmin and max_r = contact + dmax around the anchor,
//             intersected with the support polygon S (S' = S_r n S) by rejection.
//   DIRECTIONAL : Sec. IV-F one anchor with a direction v and angle threshold
//             theta: the partial annulus between min_r and max_r (from the
//             distance type; max_r may be infinite) around the anchor's
//             position, v turned by the anchor's yaw when LOCAL; points drawn
//             uniformly over its area (radius from the area fraction, angle
//             uniform in v +- theta) with max_r cut at the support's farthest
//             bounding-box corner, then S' = S_r n S by rejection.
//   MIDDLE  : Sec. IV-F two or more anchors: the polygon of their positions
//             (for two, the segment between them), proposals uniform over it
//             (over its bounding box, kept when inside), then S by rejection.
//   INSIDE  : Sec. IV-F 'inside': the support is the inside floor of an
//             articulated part (a drawer), a rectangle given at joint value 0
//             and translated by q * axis at the candidate's joint value q; the
//             position is uniform in the rectangle shrunk by the erosion e on
//             every side (to a line or point when e exceeds a half extent),
//             z = the moved floor + half height, yaw uniform, and the
//             placement is accepted at once, like ON_TOP; the walls are left
//             to the collision check.
//   FACE_TO : the yaw points from the object to the reference object (not
//             for ON_TOP or INSIDE).
// A relation naming a later object, a missing array or a MIDDLE object
// without 2..16 earlier anchors, or an INSIDE object naming a part its
// template lacks, is sampled as a free object.
static bool sample_object(const or_scene* s, int t, int c, int k, int retry, int max_attempts, uint64_t seed,
                          double (*pose)[4], bool* band_out) {
  int o = s->tmpl_obj_off[t] + k;
  int rel = s->obj_rel[o];
  int kind = rel & REL_KIND_MASK, ref = (rel >> 8) & 0xFF;
  bool face_to = (rel & REL_FACE_TO) != 0;
  std::vector<int> anchors;
  if (kind == REL_INSIDE) face_to = false;
  bool bad = (kind != REL_FREE || face_to) && kind != REL_INSIDE && ref >= k;
  bad = bad || kind > REL_INSIDE || (kind == REL_DIRECTIONAL && !s->obj_rel_dir);
  bad = bad || (kind == REL_INSIDE && (!s->part_param || !s->part_q || ref >= parts_of(s, t) || ref >= s->max_parts));
  if (kind == REL_MIDDLE) {
    if (!s->obj_anchor_off) {
      bad = true;
    } else {
      for (int i = s->obj_anchor_off[o]; i < s->obj_anchor_off[o + 1]; ++i) anchors.push_back(s->obj_anchor[i]);
      bad = bad || anchors.size() < 2 || anchors.size() > 16;
      for (int j : anchors) bad = bad || j < 0 || j >= k;
    }
  }
  if (bad) {
    kind = REL_FREE;
    face_to = false;
  }
  const float* H = &s->obj_half[4 * o];
  const float* P = &s->obj_rel_param[4 * o];
  double Hx = H[0], Hy = H[1], Hz = H[2], rho = H[3];
  double e = (double)P[2] * std::min(Hx, Hy);  // ratio_on_support erosion
  double zs = s->tmpl_support_z[t];
  bool band = false;

  if (kind == REL_INSIDE) {
    double u[4];
    draw4(seed, (uint32_t)c, (uint32_t)k, (uint32_t)retry, 0u, u);
    const float* pp = &s->part_param[12 * (s->tmpl_part_off[t] + ref)];
    double q = part_value(s, c, ref);
    double cx = pp[5] + q * pp[0], cy0 = pp[6] + q * pp[1], cz = pp[7] + q * pp[2];
    double hx = std::max((double)pp[8] - e, 0.0), hy = std::max((double)pp[9] - e, 0.0), yaw = pp[10];
    double xl = hx * (2.0 * u[0] - 1.0), yl = hy * (2.0 * u[1] - 1.0);
    double cs = std::cos(yaw), sn = std::sin(yaw);
    pose[k][0] = cx + cs * xl - sn * yl;
    pose[k][1] = cy0 + sn * xl + cs * yl;
    pose[k][2] = cz + Hz;
    pose[k][3] = TWO_PI * u[2];
    *band_out = false;
    return true;
  }

  if (kind == REL_ON_TOP) {
    double u[4];
    draw4(seed, (uint32_t)c, (uint32_t)k, (uint32_t)retry, 0u, u);
    int po = s->tmpl_obj_off[t] + ref;
    double pHx = s->obj_half[4 * po], pHy = s->obj_half[4 * po + 1], pHz = s->obj_half[4 * po + 2];
    double xl = pHx * (2.0 * u[0] - 1.0), yl = pHy * (2.0 * u[1] - 1.0);
    double cy = std::cos(pose[ref][3]), sy = std::sin(pose[ref][3]);
    pose[k][0] = pose[ref][0] + cy * xl - sy * yl;
    pose[k][1] = pose[ref][1] + sy * xl + cy * yl;
    pose[k][2] = pose[ref][2] + pHz + Hz;
    pose[k][3] = TWO_PI * u[2];
    *band_out = false;
    return true;
  }

  // bounding box of the support polygon (FREE proposals)
  int v0 = s->tmpl_poly_off[t], nv = s->tmpl_poly_off[t + 1] - v0;
  double xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
  for (int i = 0; i < nv; ++i) {
    double vx = s->poly_verts[2 * (v0 + i)], vy = s->poly_verts[2 * (v0 + i) + 1];
    xmin = std::min(xmin, vx); xmax = std::max(xmax, vx);
    ymin = std::min(ymin, vy); ymax = std::max(ymax, vy);
  }
  // DIRECTIONAL: direction and outer radius; MIDDLE: the anchors' polygon and bounding box
  double dir = 0.0, r1 = 0.0;
  if (kind == REL_DIRECTIONAL) {
    dir = (double)s->obj_rel_dir[o] + ((rel & REL_LOCAL) ? pose[ref][3] : 0.0);
    double dx = std::max(std::fabs(xmin - pose[ref][0]), std::fabs(xmax - pose[ref][0]));
    double dy = std::max(std::fabs(ymin - pose[ref][1]), std::fabs(ymax - pose[ref][1]));
    r1 = std::min((double)P[1], std::sqrt(dx * dx + dy * dy));
  }
  std::vector<double> ax, ay;
  double bx0 = INFINITY, bx1 = -INFINITY, by0 = INFINITY, by1 = -INFINITY;
  for (int j : anchors) {
    ax.push_back(pose[j][0]);
    ay.push_back(pose[j][1]);
    bx0 = std::min(bx0, pose[j][0]); bx1 = std::max(bx1, pose[j][0]);
    by0 = std::min(by0, pose[j][1]); by1 = std::max(by1, pose[j][1]);
  }
  for (int a = 0; a < max_attempts; ++a) {
    double u[4];
    draw4(seed, (uint32_t)c, (uint32_t)k, (uint32_t)retry, (uint32_t)a, u);
    double x, y;
    bool in_rel = true, rel_band = false;
    if (kind == REL_DIRECTIONAL) {
      double r0 = P[0], th = P[3];
      double rr = std::sqrt(std::max(0.0, r0 * r0 + (r1 * r1 - r0 * r0) * u[0]));
      double phi = dir + th * (2.0 * u[1] - 1.0);
      x = pose[ref][0] + rr * std::cos(phi);
      y = pose[ref][1] + rr * std::sin(phi);
    } else if (kind == REL_MIDDLE && anchors.size() == 2) {
      x = ax[0] + u[0] * (ax[1] - ax[0]);
      y = ay[0] + u[0] * (ay[1] - ay[0]);
    } else if (kind == REL_MIDDLE) {
      x = bx0 + (bx1 - bx0) * u[0];
      y = by0 + (by1 - by0) * u[1];
      double d;
      in_rel = or_point_in_polygon(ax.data(), ay.data(), (int)ax.size(), x, y, &d) != 0;
      rel_band = d <= BAND;
    } else if (kind == REL_NEXT_TO) {
      int ao = s->tmpl_obj_off[t] + ref;
      double rho_a = s->obj_half[4 * ao + 3];
      double phi = TWO_PI * u[0];
      double r = rho_a + rho + (double)P[0] + ((double)P[1] - (double)P[0]) * u[1];
      x = pose[ref][0] + r * std::cos(phi);
      y = pose[ref][1] + r * std::sin(phi);
    } else {
      x = xmin + (xmax - xmin) * u[0];
      y = ymin + (ymax - ymin) * u[1];
    }
    bool b;
    bool ok = support_accept(s, t, x, y, e, &b) && in_rel;
    band = band || b || rel_band;
    pose[k][0] = x;
    pose[k][1] = y;
    pose[k][2] = zs + Hz;
    pose[k][3] = face_to ? std::atan2(pose[ref][1] - y, pose[ref][0] - x) : TWO_PI * u[2];
    if (ok) { *band_out = band; return true; }
  }
  *band_out = band;
  return false;
}

}  // extern "C"

// Run f(i) for i in [0, n) on nthreads std::threads (contiguous chunks).
template <typename F>
static void parallel_for(int n, int nthreads, F f) {
  if (nthreads <= 1 || n < 2) {
    for (int i = 0; i < n; ++i) f(i);
    return;
  }
  nthreads = std::min(nthreads, n);
  std::vector<std::thread> th;
  for (int w = 0; w < nthreads; ++w) {
    int lo = (int)((int64_t)n * w / nthreads), hi = (int)((int64_t)n * (w + 1) / nthreads);
    th.emplace_back([=]() { for (int i = lo; i < hi; ++i) f(i); });
  }
  for (auto& x : th) x.join();
}

extern "C" {

// Sample objects [first_obj, first_obj + n_obj) of every listed candidate
// (active == NULL: all candidates) for try `retry`. poses: [P][4] double, CSR
// pose layout; objects before first_obj must already hold their poses.
// ok[i] / band[i] are per listed candidate (AND / OR over its sampled objects).
int or_sample_poses(const or_scene* s, uint64_t seed, int max_attempts, int retry, int first_obj, int n_obj,
                    const int32_t* active, int n_active, double* poses, uint8_t* ok, uint8_t* band, int nthreads) {
  int n = active ? n_active : s->n_cand;
  parallel_for(n, nthreads, [&](int i) {
    int c = active ? active[i] : i;
    int t = template_of(s, c);
    int nt = s->tmpl_obj_off[t + 1] - s->tmpl_obj_off[t];
    double(*pose)[4] = (double(*)[4]) & poses[4 * pose_offset(s, c, t)];
    bool all_ok = true, any_band = false;
    for (int k = first_obj; k < first_obj + n_obj && k < nt; ++k) {
      bool b;
      bool a = sample_object(s, t, c, k, retry, max_attempts, seed, pose, &b);
      all_ok = all_ok && a;
      any_band = any_band || b;
    }
    ok[i] = all_ok;
    band[i] = any_band;
  });
  return 0;
}

// Randomised articulation (Sec. IV-B batched forward kinematics; the 'inside'
// supports of Sec. IV-F sit on the parts): the
// joint value of part j of candidate c is uniform in [qmin, qmax], drawn from
// the Philox counter (c, 0xFFFF0000 + j, 0, 0), which no pose draw uses.
int or_sample_parts(const or_scene* s, uint64_t seed, const int32_t* active, int n_active, double* part_q) {
  int n = active ? n_active : s->n_cand;
  for (int i = 0; i < n; ++i) {
    int c = active ? active[i] : i;
    int t = template_of(s, c);
    for (int j = 0; j < parts_of(s, t); ++j) {
      const float* pp = &s->part_param[12 * (s->tmpl_part_off[t] + j)];
      double u[4];
      draw4(seed, (uint32_t)c, 0xFFFF0000u + (uint32_t)j, 0u, 0u, u);
      part_q[(int64_t)c * s->max_parts + j] = (double)pp[3] + ((double)pp[4] - (double)pp[3]) * u[0];
    }
  }
  return 0;
}

// ---------------------------------------------------------------------------
// Collision (Sec. IV-D): per-object sphere sets moved by the object's pose
// (Sec. IV-B: one transform per instance), sphere-sphere signed distance
// |c_i - c_j| - r_i - r_j over pairs of spheres of different objects, and the
// exact box signed distance minus r against the static world's OBBs.
// Pinned by: closed forms (two spheres, box face/edge/corner/interior), rigid-
// motion invariance, brute force on hand-computed tiny scenes.
// ---------------------------------------------------------------------------
void or_sphere_world(const float* sph, const double* pose, double* out) {
  double cy = std::cos(pose[3]), sy = std::sin(pose[3]);
  double x = sph[0], y = sph[1], z = sph[2];
  out[0] = pose[0] + cy * x - sy * y;
  out[1] = pose[1] + sy * x + cy * y;
  out[2] = pose[2] + z;
  out[3] = sph[3];
}

double or_sphere_sphere(const double* a, const double* b) {
  double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
  return std::sqrt(dx * dx + dy * dy + dz * dz) - a[3] - b[3];
}

// Rotation matrix (row-major) of the quaternion (x, y, z, w), normalised first.
static void quat_to_matrix(const double q_in[4], double R[9]) {
  double n = std::sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
  double x = q_in[0] / n, y = q_in[1] / n, z = q_in[2] / n, w = q_in[3] / n;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - z * w);     R[2] = 2 * (x * z + y * w);
  R[3] = 2 * (x * y + z * w);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - x * w);
  R[6] = 2 * (x * z - y * w);     R[7] = 2 * (y * z + x * w);     R[8] = 1 - 2 * (x * x + y * y);
}

// Signed distance from sphere (c, r) to the oriented box (12 floats as in
// or_scene.obb) whose centre is moved by `shift` (NULL: not moved).
static double sphere_obb_moved(const double* sphere, const float* box, const double* shift) {
  double q[4] = {box[4], box[5], box[6], box[7]};
  double R[9];
  quat_to_matrix(q, R);
  double ctr[3] = {box[0], box[1], box[2]};
  if (shift)
    for (int i = 0; i < 3; ++i) ctr[i] += shift[i];
  double d[3] = {sphere[0] - ctr[0], sphere[1] - ctr[1], sphere[2] - ctr[2]};
  double p[3];  // R^T d: the sphere centre in the box frame
  for (int i = 0; i < 3; ++i) p[i] = R[0 + i] * d[0] + R[3 + i] * d[1] + R[6 + i] * d[2];
  double h[3] = {box[8], box[9], box[10]};
  double qx = std::fabs(p[0]) - h[0], qy = std::fabs(p[1]) - h[1], qz = std::fabs(p[2]) - h[2];
  double ox = std::max(qx, 0.0), oy = std::max(qy, 0.0), oz = std::max(qz, 0.0);
  double outside = std::sqrt(ox * ox + oy * oy + oz * oz);
  double inside = std::min(std::max(qx, std::max(qy, qz)), 0.0);
  return outside + inside - sphere[3];
}

double or_sphere_obb(const double* sphere, const float* box) { return sphere_obb_moved(sphere, box, nullptr); }

// Distance from point p to segment [a, b]: the nearest point a + t (b - a)
// with t the projection parameter clamped to [0, 1].
static double point_segment(const double* p, const double* a, const double* b) {
  double ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, ap[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
  double l2 = ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2];
  double t = l2 > 0.0 ? (ap[0] * ab[0] + ap[1] * ab[1] + ap[2] * ab[2]) / l2 : 0.0;
  t = std::min(1.0, std::max(0.0, t));
  double d[3] = {ap[0] - t * ab[0], ap[1] - t * ab[1], ap[2] - t * ab[2]};
  return std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
}

// Distance from point p to the (closed, filled) triangle abc: the distance
// to its plane when p's orthogonal projection falls inside the triangle (all
// three barycentric coordinates >= 0), else the distance to the nearest of
// its three edges. A zero-area triangle is its edges.
double or_point_triangle(const double* p, const double* a, const double* b, const double* c) {
  double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
  double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
  double nn = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
  double edges = std::min(point_segment(p, a, b), std::min(point_segment(p, b, c), point_segment(p, c, a)));
  if (!(nn > 0.0)) return edges;
  double ap[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
  double h = (ap[0] * n[0] + ap[1] * n[1] + ap[2] * n[2]) / nn;  // signed height over |n|^2
  double q[3] = {ap[0] - h * n[0], ap[1] - h * n[1], ap[2] - h * n[2]};  // projection, relative to a
  // barycentric coordinates of the projection: q = s e1 + t e2
  double d11 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2], d22 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
  double d12 = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2];
  double q1 = q[0] * e1[0] + q[1] * e1[1] + q[2] * e1[2], q2 = q[0] * e2[0] + q[1] * e2[1] + q[2] * e2[2];
  double det = d11 * d22 - d12 * d12;
  double s = (q1 * d22 - q2 * d12) / det, t = (q2 * d11 - q1 * d12) / det;
  if (s >= 0.0 && t >= 0.0 && s + t <= 1.0) return std::fabs(h) * std::sqrt(nn);
  return edges;
}

// Signed distance of sphere (c, r) to triangle `t` (12 floats as in or_scene.tri).
double or_sphere_triangle(const double* sphere, const float* t) {
  double a[3] = {t[0], t[1], t[2]}, b[3] = {t[4], t[5], t[6]}, c[3] = {t[8], t[9], t[10]};
  return or_point_triangle(sphere, a, b, c) - sphere[3];
}

// Where world box `ob` of candidate c (template t) sits: a box of an
// articulated part is moved by q * axis, q the candidate's joint value of it.
static void box_shift(const or_scene* s, int t, int c, int ob, double shift[3]) {
  shift[0] = shift[1] = shift[2] = 0.0;
  if (!s->obb_part || s->n_parts <= 0) return;
  int j = s->obb_part[ob];
  if (j < 0 || j >= parts_of(s, t) || j >= s->max_parts) return;
  const float* pp = &s->part_param[12 * (s->tmpl_part_off[t] + j)];
  double q = part_value(s, c, j);
  for (int i = 0; i < 3; ++i) shift[i] = q * pp[i];
}

// Minimum signed distance of candidate c whose poses are pose[0..n_t):
// sphere pairs (i in object a, j in object b, a < b, b >= first_new) and
// (sphere in object >= first_new, world OBB). Empty set: +FLT_MAX.
static double candidate_min_dist(const or_scene* s, int t, int c, const double (*pose)[4], int first_new,
                                 int last_obj) {
  int o0 = s->tmpl_obj_off[t];
  int nt = std::min(s->tmpl_obj_off[t + 1] - o0, last_obj);
  // world-frame spheres of every object, per object
  std::vector<std::vector<std::array<double, 4>>> W(nt);
  for (int k = 0; k < nt; ++k) {
    int o = o0 + k;
    for (int q = s->obj_sph_off[o]; q < s->obj_sph_off[o + 1]; ++q) {
      std::array<double, 4> w;
      or_sphere_world(&s->sph_local[4 * q], pose[k], w.data());
      W[k].push_back(w);
    }
  }
  double m = (double)FLT_MAX;
  for (int b = std::max(first_new, 0); b < nt; ++b)
    for (int a = 0; a < b; ++a)
      for (auto& si : W[a])
        for (auto& sj : W[b]) m = std::min(m, or_sphere_sphere(si.data(), sj.data()));
  for (int b = std::max(first_new, 0); b < nt; ++b)
    for (auto& sj : W[b])
      for (int ob = s->tmpl_obb_off[t]; ob < s->tmpl_obb_off[t + 1]; ++ob) {
        double sh[3];
        box_shift(s, t, c, ob, sh);
        m = std::min(m, sphere_obb_moved(sj.data(), &s->obb[12 * ob], sh));
      }
  if (s->n_tri > 0 && s->tmpl_tri_off && s->tri)
    for (int b = std::max(first_new, 0); b < nt; ++b)
      for (auto& sj : W[b])
        for (int q = s->tmpl_tri_off[t]; q < s->tmpl_tri_off[t + 1]; ++q)
          m = std::min(m, or_sphere_triangle(sj.data(), &s->tri[12 * q]));
  return m;
}

// Collision check of every listed candidate. collide = min_dist < 0 (touching
// is free); band = |min_dist| <= 1e-5 m.
int or_collide(const or_scene* s, const double* poses, const int32_t* active, int n_active, int first_new,
               uint8_t* collide, double* min_dist, uint8_t* band, int nthreads) {
  int n = active ? n_active : s->n_cand;
  parallel_for(n, nthreads, [&](int i) {
    int c = active ? active[i] : i;
    int t = template_of(s, c);
    const double(*pose)[4] = (const double(*)[4]) & poses[4 * pose_offset(s, c, t)];
    double m = candidate_min_dist(s, t, c, pose, first_new, 1 << 30);
    min_dist[i] = m;
    collide[i] = m < 0.0;
    band[i] = std::fabs(m) <= BAND;
  });
  return 0;
}

}  // extern "C"

extern "C" {

// ---------------------------------------------------------------------------
// Reachability (Sec. IV-E: reject a sampled pose the robot cannot reach). The
// paper queries an RM4D map; this build answers the same question exactly with
// damped-least-squares IK on a 7-DoF arm given by standard DH parameters.
//   T_i = Rz(q_i) Tz(d_i) Tx(a_i) Rx(alpha_i), tool frame = frame 7, base = identity
//   (targets are given in the robot base frame).
//   Geometric Jacobian: column i = [z_{i-1} x (p_7 - p_{i-1}); z_{i-1}].
//   Error e = [p* - p; 1/2 sum_k r_k x r*_k] (columns of R and R*).
//   Step  dq = J^T (J J^T + lambda^2 I)^-1 e, then q clamped to [qmin, qmax].
//   Success (checked before every step and after the last one):
//     |p* - p| <= tol_pos and angle(R^T R*) <= tol_rot.
//   Seeds: q0_j = qmin_j + (qmax_j - qmin_j) u_j, u from Philox4x32-10 with
//   key = IK seed, counter = (target, seed index, j / 4, hi), word j % 4;
//   hi = 0 for a plain target list, object << 16 | try inside generation.
//   All seeds of a target iterate in lock step; the target is reachable at the
//   first check where any seed succeeds and returns the lowest such seed index;
//   otherwise it returns the seed with the smallest position error at the end.
//   Band: a check of some seed whose position error or angle lies within
//   1e-5 of its tolerance (the other not failing by more than 1e-5) could
//   flip under FP32 rounding; the target is then flagged.
// Pinned by: FK at q = 0 against a hand-multiplied DH chain, Jacobian against
// central differences, the push-through identity of the damped inverse, the
// reach bound (targets beyond sum |d_i| + |a_i| never succeed), the seed
// draw against an independent Philox4x32-10 checked on its known answers,
// and the selection rule at zero iterations (the lowest seed whose own FK,
// from scipy, is the target wins; else the seed of least scipy-FK position
// error); the band flag by targets placed at tol_pos +- 5e-6 and +- 2e-5.
// ---------------------------------------------------------------------------
typedef struct {
  float dh_d[7], dh_a[7], dh_alpha[7], qmin[7], qmax[7];
} or_arm;

typedef struct {
  float lambda, tol_pos, tol_rot;
  int32_t iters, seeds;
  uint64_t seed;
} or_ik_params;

// Forward kinematics: frames[i] (i = 0..7) as row-major 4x4, frame 0 = base.
void or_fk_frames(const or_arm* arm, const double* q, double* frames) {
  double T[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
  std::memcpy(frames, T, sizeof(T));
  for (int i = 0; i < 7; ++i) {
    double ct = std::cos(q[i]), st = std::sin(q[i]);
    double ca = std::cos((double)arm->dh_alpha[i]), sa = std::sin((double)arm->dh_alpha[i]);
    double a = arm->dh_a[i], d = arm->dh_d[i];
    // A = Rz(theta) Tz(d) Tx(a) Rx(alpha)
    double A[16] = {ct, -st * ca, st * sa, a * ct,
                    st, ct * ca, -ct * sa, a * st,
                    0, sa, ca, d,
                    0, 0, 0, 1};
    double N[16];
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) {
        double acc = 0;
        for (int k = 0; k < 4; ++k) acc += T[4 * r + k] * A[4 * k + c];
        N[4 * r + c] = acc;
      }
    std::memcpy(T, N, sizeof(T));
    std::memcpy(frames + 16 * (i + 1), T, sizeof(T));
  }
}

// 6x7 geometric Jacobian (row-major) at q.
void or_jacobian(const or_arm* arm, const double* q, double* J) {
  double F[8 * 16];
  or_fk_frames(arm, q, F);
  double pe[3] = {F[16 * 7 + 3], F[16 * 7 + 7], F[16 * 7 + 11]};
  for (int i = 0; i < 7; ++i) {
    const double* Fi = F + 16 * i;  // frame i-1 of joint i (0-based: frame i)
    double z[3] = {Fi[2], Fi[6], Fi[10]};
    double p[3] = {Fi[3], Fi[7], Fi[11]};
    double r[3] = {pe[0] - p[0], pe[1] - p[1], pe[2] - p[2]};
    J[0 * 7 + i] = z[1] * r[2] - z[2] * r[1];
    J[1 * 7 + i] = z[2] * r[0] - z[0] * r[2];
    J[2 * 7 + i] = z[0] * r[1] - z[1] * r[0];
    J[3 * 7 + i] = z[0];
    J[4 * 7 + i] = z[1];
    J[5 * 7 + i] = z[2];
  }
}

// Position error norm and rotation angle of the tool at q against target
// (R* row-major 3x3, p*), both in the base frame.
void or_pose_error(const or_arm* arm, const double* q, const double* Rt, const double* pt, double* pos_err, double* rot_err) {
  double F[8 * 16];
  or_fk_frames(arm, q, F);
  const double* T = F + 16 * 7;
  double dx = pt[0] - T[3], dy = pt[1] - T[7], dz = pt[2] - T[11];
  *pos_err = std::sqrt(dx * dx + dy * dy + dz * dz);
  double M[9];  // R^T R*
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double acc = 0;
      for (int k = 0; k < 3; ++k) acc += T[4 * k + r] * Rt[3 * k + c];
      M[3 * r + c] = acc;
    }
  double vx = 0.5 * (M[7] - M[5]), vy = 0.5 * (M[2] - M[6]), vz = 0.5 * (M[3] - M[1]);
  double s = std::sqrt(vx * vx + vy * vy + vz * vz);
  double c = 0.5 * (M[0] + M[4] + M[8] - 1.0);
  *rot_err = std::atan2(s, c);
}

// Solve (A) y = e for symmetric positive definite 6x6 A by Cholesky.
static void chol_solve6(const double* A, const double* e, double* y) {
  double L[36] = {0};
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = A[6 * i + j];
      for (int k = 0; k < j; ++k) s -= L[6 * i + k] * L[6 * j + k];
      if (i == j) L[6 * i + i] = std::sqrt(s);
      else L[6 * i + j] = s / L[6 * j + j];
    }
  double z[6];
  for (int i = 0; i < 6; ++i) {
    double s = e[i];
    for (int k = 0; k < i; ++k) s -= L[6 * i + k] * z[k];
    z[i] = s / L[6 * i + i];
  }
  for (int i = 5; i >= 0; --i) {
    double s = z[i];
    for (int k = i + 1; k < 6; ++k) s -= L[6 * k + i] * y[k];
    y[i] = s / L[6 * i + i];
  }
}

// Task-space error at q: e = [p* - p; 1/2 sum_k r_k x r*_k] (6 values).
void or_ik_error(const or_arm* arm, const double* q, const double* Rt, const double* pt, double* e) {
  double F[8 * 16];
  or_fk_frames(arm, q, F);
  const double* T = F + 16 * 7;
  e[0] = pt[0] - T[3];
  e[1] = pt[1] - T[7];
  e[2] = pt[2] - T[11];
  e[3] = e[4] = e[5] = 0.0;
  for (int k = 0; k < 3; ++k) {
    double r[3] = {T[0 + k], T[4 + k], T[8 + k]};
    double rs[3] = {Rt[0 + k], Rt[3 + k], Rt[6 + k]};
    e[3] += 0.5 * (r[1] * rs[2] - r[2] * rs[1]);
    e[4] += 0.5 * (r[2] * rs[0] - r[0] * rs[2]);
    e[5] += 0.5 * (r[0] * rs[1] - r[1] * rs[0]);
  }
}

// One damped-least-squares step from q (in place), clamped to the joint limits.
void or_dls_step(const or_arm* arm, double lambda, const double* Rt, const double* pt, double* q) {
  double e[6];
  or_ik_error(arm, q, Rt, pt, e);
  double J[42];
  or_jacobian(arm, q, J);
  double A[36];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double acc = 0;
      for (int k = 0; k < 7; ++k) acc += J[7 * i + k] * J[7 * j + k];
      A[6 * i + j] = acc + (i == j ? lambda * lambda : 0.0);
    }
  double y[6];
  chol_solve6(A, e, y);
  for (int k = 0; k < 7; ++k) {
    double dq = 0;
    for (int i = 0; i < 6; ++i) dq += J[7 * i + k] * y[i];
    double v = q[k] + dq;
    v = std::min(std::max(v, (double)arm->qmin[k]), (double)arm->qmax[k]);
    q[k] = v;
  }
}

static void ik_seed_words(const or_arm* arm, uint64_t seed, uint32_t target, uint32_t target_hi, uint32_t s,
                          double* q) {
  for (int b = 0; b < 2; ++b) {
    double u[4];
    draw4(seed, target, s, (uint32_t)b, target_hi, u);
    for (int w = 0; w < 4; ++w) {
      int j = 4 * b + w;
      if (j < 7) q[j] = (double)arm->qmin[j] + ((double)arm->qmax[j] - (double)arm->qmin[j]) * u[w];
    }
  }
}

void or_ik_seed(const or_arm* arm, uint64_t seed, uint32_t target, uint32_t s, double* q) {
  ik_seed_words(arm, seed, target, 0u, s, q);
}

// Is one seed's success decision at one check within the band? The decision
// is (position error <= tol_pos) and (angle <= tol_rot); it could flip under
// a perturbation of BAND when one error lies within BAND of its tolerance
// while the other does not fail by more than BAND.
static bool ik_check_banded(double pe, double re, const or_ik_params* P) {
  const double tp = P->tol_pos, tr = P->tol_rot;
  return (std::fabs(pe - tp) <= BAND && re <= tr + BAND) || (std::fabs(re - tr) <= BAND && pe <= tp + BAND);
}

// IK for one target (12 floats: R row-major, p). Returns reachable; q_out[7],
// err[2] = (position error, rotation angle) of the returned configuration,
// *iter_out = the check index at which it ended, *band_out = 1 if any check
// of any seed up to that one was within the band (ik_check_banded): every
// such check took part in deciding the outcome, since the seeds move in lock
// step and the first success ends all of them.
static int ik_one(const or_arm* arm, const or_ik_params* P, const float* target, uint32_t tid, uint32_t tid_hi,
                  double* q_out, double* err, int* iter_out, int* band_out) {
  double Rt[9], pt[3];
  for (int i = 0; i < 9; ++i) Rt[i] = target[i];
  for (int i = 0; i < 3; ++i) pt[i] = target[9 + i];
  int S = P->seeds;
  std::vector<double> q(7 * S);
  for (int s = 0; s < S; ++s) ik_seed_words(arm, P->seed, tid, tid_hi, (uint32_t)s, &q[7 * s]);
  std::vector<double> pe(S), re(S);
  int banded = 0;
  for (int it = 0; it <= P->iters; ++it) {
    int hit = -1;
    for (int s = 0; s < S; ++s) {
      or_pose_error(arm, &q[7 * s], Rt, pt, &pe[s], &re[s]);
      if (ik_check_banded(pe[s], re[s], P)) banded = 1;
      if (hit < 0 && pe[s] <= (double)P->tol_pos && re[s] <= (double)P->tol_rot) hit = s;
    }
    if (hit >= 0) {
      for (int k = 0; k < 7; ++k) q_out[k] = q[7 * hit + k];
      err[0] = pe[hit];
      err[1] = re[hit];
      *iter_out = it;
      *band_out = banded;
      return 1;
    }
    if (it == P->iters) break;
    for (int s = 0; s < S; ++s) or_dls_step(arm, (double)P->lambda, Rt, pt, &q[7 * s]);
  }
  int best = 0;
  for (int s = 1; s < S; ++s)
    if (pe[s] < pe[best]) best = s;
  for (int k = 0; k < 7; ++k) q_out[k] = q[7 * best + k];
  err[0] = pe[best];
  err[1] = re[best];
  *iter_out = P->iters;
  *band_out = banded;
  return 0;
}

// target_ids: Philox counter index of each target (NULL: 0..n-1). band
// (optional) receives ik_one's band flag of each target.
int or_ik_reach(const or_arm* arm, const or_ik_params* P, const float* targets, const uint32_t* target_ids, int n,
                uint8_t* reach, double* q_out, double* err, int32_t* iters, uint8_t* band, int nthreads) {
  parallel_for(n, nthreads, [&](int i) {
    int it, b;
    reach[i] = (uint8_t)ik_one(arm, P, targets + 12 * i, target_ids ? target_ids[i] : (uint32_t)i, 0u, q_out + 7 * i,
                               err + 2 * i, &it, &b);
    if (iters) iters[i] = it;
    if (band) band[i] = (uint8_t)b;
  });
  return 0;
}

// Top-down grasp target of an object at world pose (x, y, z, yaw) with half
// height Hz, for a robot base at (bx, by, bz, byaw): position = top centre of
// the object's box, tool z = -world z, tool x along the object's yaw. Output
// in the base frame: 12 floats (R row-major, p).
void or_grasp_target(const double* pose, double Hz, const float* base, double* out) {
  double cb = std::cos((double)base[3]), sb = std::sin((double)base[3]);
  double wx = pose[0] - base[0], wy = pose[1] - base[1], wz = pose[2] + Hz - base[2];
  double px = cb * wx + sb * wy, py = -sb * wx + cb * wy, pz = wz;
  double psi = pose[3] - (double)base[3];
  double c = std::cos(psi), s = std::sin(psi);
  // columns x = (c, s, 0), y = (s, -c, 0), z = (0, 0, -1)
  double R[9] = {c, s, 0, s, -c, 0, 0, 0, -1};
  for (int i = 0; i < 9; ++i) out[i] = R[i];
  out[9] = px; out[10] = py; out[11] = pz;
}

// ---------------------------------------------------------------------------
// Generation loop (Sec. IV-A and Fig. 2; Sec. IV-D re-checks only retrying
// scenes; Sec. V-A 10 retries per object, failures marked invalid). Objects
// are placed in template order. For object k, try r = 0..max_retries: sample
// (retry index r in the Philox counter), then check object k against objects
// 0..k-1 and the static world, then (if the object is marked for reachability
// and an arm is given) solve IK for its top-down grasp. The first try that
// passes every check fixes the pose; if none does the scene is invalid and its
// remaining objects are not placed.
// band[c] = some decision on the candidate's path was within 1e-5 m (a
// support test, a collision minimum or an IK success check).
// tries[c] = total tries spent.
// Pinned by: valid scenes re-checked collision-free, zero retries equal to a
// whole-scene check, and for the reachability branch: tolerances every seed
// meets at once give the scenes of the run without an arm; a base from which
// every grasp lies beyond the arm's reach spends all max_retries + 1 tries on
// the first designated object and places nothing after it.
// ---------------------------------------------------------------------------
typedef struct {
  uint64_t seed;
  int32_t max_attempts, max_retries;
} or_gen_params;

int or_generate(const or_scene* s, const or_gen_params* G, const or_arm* arm, const or_ik_params* ikp,
                const int32_t* active, int n_active, double* poses, uint8_t* valid, uint8_t* band, int32_t* tries,
                int nthreads) {
  int n = active ? n_active : s->n_cand;
  parallel_for(n, nthreads, [&](int i) {
    int c = active ? active[i] : i;
    int t = template_of(s, c);
    int o0 = s->tmpl_obj_off[t];
    int nt = s->tmpl_obj_off[t + 1] - o0;
    double(*pose)[4] = (double(*)[4]) & poses[4 * pose_offset(s, c, t)];
    bool ok_scene = true, any_band = false;
    int ntries = 0;
    for (int k = 0; k < nt && ok_scene; ++k) {
      bool placed = false;
      for (int r = 0; r <= G->max_retries && !placed; ++r) {
        ntries++;
        bool b;
        bool ok = sample_object(s, t, c, k, r, G->max_attempts, G->seed, pose, &b);
        any_band = any_band || b;
        if (!ok) continue;
        double m = candidate_min_dist(s, t, c, pose, k, k + 1);
        any_band = any_band || std::fabs(m) <= BAND;
        if (m < 0.0) continue;
        if (arm && (s->obj_rel[o0 + k] & REL_REACH)) {
          double tgt[12];
          or_grasp_target(pose[k], s->obj_half[4 * (o0 + k) + 2], &s->tmpl_base[4 * t], tgt);
          float tf[12];
          for (int q = 0; q < 12; ++q) tf[q] = (float)tgt[q];
          double qo[7], e2[2];
          int it, ikb;
          // IK seeds of this try: counter (candidate, seed, block, object << 16 | try)
          const int reach_ok = ik_one(arm, ikp, tf, (uint32_t)c, ((uint32_t)k << 16) | (uint32_t)r, qo, e2, &it, &ikb);
          any_band = any_band || ikb;
          if (!reach_ok) continue;
        }
        placed = true;
      }
      if (!placed) ok_scene = false;
    }
    valid[i] = ok_scene;
    band[i] = any_band;
    if (tries) tries[i] = ntries;
  });
  return 0;
}

}  // extern "C"
