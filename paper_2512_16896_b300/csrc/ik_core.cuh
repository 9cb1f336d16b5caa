// Device core of the batched damped-least-squares IK (Sec. IV-E reachability,
// solved exactly instead of the paper's RM4D lookup): forward kinematics of
// a standard-DH 7-DoF arm, the success test, one DLS step, and the warp-level
// lock-step solve over the seeds of one target. Shared by the IK kernels and
// the reachability stage of the generation loop.
#pragma once

#include "common.cuh"

namespace sc {
namespace ikc {

// Arm constants. Twists within 1e-6 of a multiple of pi/2 are snapped to it
// (cos and sin exactly 0 and +-1), and when the twists of joints 2..6 are all
// +-pi/2 (right != 0; most 7-DoF arms) the forward kinematics runs in a
// signed form: Rx(+-pi/2) maps (c1, c2) to (+-c2, -+n1), a renaming of the
// columns up to sign, so the columns are carried as c_k = g_k ch_k with the
// signs g_k tracked here on the host and folded into the constants below.
// The last joint's twist is folded into the target (see target_frame), so no
// step applies it.
struct ArmK {
  float d[7], a[7], ca[7], sa[7], qmin[7], qmax[7];
  int right;
  uint32_t sflip[7];  // sign bit that turns sin q_i into g0 g1 sin q_i (right form; 0 otherwise)
  float as[7], ds[7];  // a_i g0 and d_i g2 at joint i
  float zsign[7];      // g2 at joint i: z_i = zsign_i * (stored axis)
  float gs[3];         // g of the columns of the frame fk returns
};

struct IkArgs {
  ArmK arm;
  float lambda2, tol_pos2, cos2_tol, sin2_tol;  // squared cosine / sine of the angle tolerance
  // band of the success decision: squared position bounds (tol_pos -+ 1e-5)^2
  // and squared cosine / sine of the angles tol_rot -+ 1e-5 (see check_banded)
  float pos_lo2, pos_hi2, cos2_lo, sin2_lo, cos2_hi, sin2_hi;
  int iters, seeds;
  uint64_t seed;
  const float* targets;
  const uint32_t* target_ids;
  int n;
  uint8_t* reach;
  float* q_out;
  float* err;
  int32_t* iters_out;
  uint8_t* band;        // optional: band flag of each target (Solve::band)
  unsigned long long* seed_iters;  // optional: checks evaluated x seeds, summed (zeroed before the launch)
  unsigned int* claim;  // work counter (zeroed before the launch): warps claim targets dynamically
};

// Forward kinematics; z[i], p[i] = axis and origin of frame i (i = 0..6,
// the frame joint i+1 rotates about; z[i] up to the sign A.zsign[i]); Rh, t =
// the tool frame before the last twist, Rh row-major with its columns up to
// the signs A.gs (tool_rotation gives the tool's rotation).
// T_i = Rz(q_i) Tz(d_i) Tx(a_i) Rx(alpha_i) acts on the frame's columns
// c0, c1, c2 in three steps: Rz turns c0, c1 by q; the translation adds
// a c0 + d c2; Rx turns c1, c2 by alpha (4 + 2 + 4 multiply-adds per row;
// none in the signed form of ArmK). Rows 0 and 1 go through the packed
// two-lane FP32 instructions (each multiply-add above is one instruction for
// both rows), row 2 is scalar; every product rounds as its scalar form. The
// first joint acts on the base frame (c0, c1, c2 = e_x, e_y, e_z, origin 0),
// where those steps reduce to one product per entry: the products with the
// zero and unit entries they skip are exact, so the values are the general
// step's.
template <bool kRight>
__device__ __forceinline__ void fk(const ArmK& A, const float q[7], float z[7][3], float p[7][3], float Rh[9],
                                   float t[3]) {
  float sq[7], cq[7];
#pragma unroll
  for (int i = 0; i < 6; i += 2) {  // joints in pairs, the seventh alone
    float2 s2, c2;
    sincos_cw2(make_float2(q[i], q[i + 1]), &s2, &c2);
    sq[i] = s2.x; cq[i] = c2.x;
    sq[i + 1] = s2.y; cq[i + 1] = c2.y;
  }
  sincos_cw(q[6], &sq[6], &cq[6]);
  z[0][0] = 0.f; z[0][1] = 0.f; z[0][2] = 1.f;
  p[0][0] = 0.f; p[0][1] = 0.f; p[0][2] = 0.f;
  const float ca0 = A.ca[0], sa0 = A.sa[0];
  float2 c0 = make_float2(cq[0], sq[0]);
  float2 c1 = __fmul2_rn(make_float2(-sq[0], cq[0]), make_float2(ca0, ca0));
  float2 c2 = __fmul2_rn(make_float2(sq[0], -cq[0]), make_float2(sa0, sa0));
  float2 t01 = __fmul2_rn(c0, make_float2(A.a[0], A.a[0]));
  float c0z = 0.f, c1z = sa0, c2z = ca0, tz = A.d[0];  // row 2
#pragma unroll
  for (int i = 1; i < 7; ++i) {
    z[i][0] = c2.x; z[i][1] = c2.y; z[i][2] = c2z;
    p[i][0] = t01.x; p[i][1] = t01.y; p[i][2] = tz;
    float st = sq[i];
    if constexpr (kRight) st = __int_as_float(__float_as_int(st) ^ A.sflip[i]);
    const float ct = cq[i], a = A.as[i], d = A.ds[i];
    const float2 n0 = __ffma2_rn(c1, make_float2(st, st), __fmul2_rn(c0, make_float2(ct, ct)));
    const float2 n1 = __ffma2_rn(c1, make_float2(ct, ct), __fmul2_rn(c0, make_float2(-st, -st)));
    t01 = __ffma2_rn(n0, make_float2(a, a), __ffma2_rn(c2, make_float2(d, d), t01));
    const float m0 = fmaf(c1z, st, c0z * ct), m1 = fmaf(c1z, ct, -c0z * st);
    tz = fmaf(m0, a, fmaf(c2z, d, tz));
    if (i == 6) {
      Rh[0] = n0.x; Rh[1] = n1.x; Rh[2] = c2.x;
      Rh[3] = n0.y; Rh[4] = n1.y; Rh[5] = c2.y;
      Rh[6] = m0; Rh[7] = m1; Rh[8] = c2z;
    } else {
      c0 = n0;
      c0z = m0;
      if constexpr (kRight) {  // (ch1, ch2) <- (ch2, nh1); the signs are A's
        c1 = c2; c1z = c2z;
        c2 = n1; c2z = m1;
      } else {
        const float ca = A.ca[i], sa = A.sa[i];
        c1 = __ffma2_rn(c2, make_float2(sa, sa), __fmul2_rn(n1, make_float2(ca, ca)));
        c2 = __ffma2_rn(c2, make_float2(ca, ca), __fmul2_rn(n1, make_float2(-sa, -sa)));
        c1z = fmaf(c2z, sa, m1 * ca);
        c2z = fmaf(c2z, ca, -m1 * sa);
      }
    }
  }
  t[0] = t01.x; t[1] = t01.y; t[2] = tz;
}

// The tool's rotation (row-major) from fk's Rh: the signs A.gs, then the
// last joint's Rx.
__device__ __forceinline__ void tool_rotation(const ArmK& A, const float Rh[9], float R[9]) {
  const float ca = A.ca[6], sa = A.sa[6];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float n0 = A.gs[0] * Rh[3 * r], n1 = A.gs[1] * Rh[3 * r + 1], c2 = A.gs[2] * Rh[3 * r + 2];
    R[3 * r] = n0;
    R[3 * r + 1] = fmaf(c2, sa, n1 * ca);
    R[3 * r + 2] = fmaf(c2, ca, -n1 * sa);
  }
}

struct Target {
  float R[9], p[3];
};

// The target as rot_error compares it with fk's Rh: R* X^T (X = Rx of the
// last joint's twist) with its columns times A.gs / 2. With R = R0 X the
// tool's rotation (R0 = the columns of Rh times A.gs), sum_k r_k x r*_k =
// R0's columns crossed with R* X^T's (X X^T = I) and likewise the trace, so
// the errors are those of R against R*; the factor 1/2 of the error and of
// the cosine is applied here once per solve (exact: a power of two).
__device__ __forceinline__ Target target_frame(const ArmK& A, const Target& T) {
  const float ca = A.ca[6], sa = A.sa[6];
  Target H;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float r0 = T.R[3 * r], r1 = T.R[3 * r + 1], r2 = T.R[3 * r + 2];
    H.R[3 * r] = (0.5f * A.gs[0]) * r0;
    H.R[3 * r + 1] = (0.5f * A.gs[1]) * fmaf(ca, r1, -sa * r2);
    H.R[3 * r + 2] = (0.5f * A.gs[2]) * fmaf(sa, r1, ca * r2);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) H.p[i] = T.p[i];
  return H;
}

// Orientation error of R against the target's R*, in the world frame: w =
// 1/2 sum_k r_k x r*_k over the columns (|w| = sine of the angle of R^T R*,
// since w = R vee(M - M^T) / 2 with M = R^T R*), and c = (tr(R^T R*) - 1) / 2
// = (sum_ij R_ij R*_ij - 1) / 2 (its cosine). T is the target as
// target_frame gives it, its columns already halved.
__device__ __forceinline__ void rot_error(const Target& T, const float R[9], float w[3], float* c) {
  float wx = 0.f, wy = 0.f, wz = 0.f, tr = -0.5f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float ax = R[k], ay = R[3 + k], az = R[6 + k];        // column k of R
    const float bx = T.R[k], by = T.R[3 + k], bz = T.R[6 + k];  // column k of R*
    wx = fmaf(ay, bz, fmaf(-az, by, wx));
    wy = fmaf(az, bx, fmaf(-ax, bz, wy));
    wz = fmaf(ax, by, fmaf(-ay, bx, wz));
    tr = fmaf(ax, bx, fmaf(ay, by, fmaf(az, bz, tr)));
  }
  w[0] = wx;
  w[1] = wy;
  w[2] = wz;
  *c = tr;
}

// Success test of one configuration; v (world-frame error), s2 = |v|^2 and c
// as rot_error.
__device__ __forceinline__ bool check(const IkArgs& K, const Target& T, const float R[9], const float t[3],
                                      float* pos_err2, float v[3], float* s2_out, float* c_out) {
  const float dx = T.p[0] - t[0], dy = T.p[1] - t[1], dz = T.p[2] - t[2];
  const float pe2 = dx * dx + dy * dy + dz * dz;
  float c;
  rot_error(T, R, v, &c);
  const float s2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  *pos_err2 = pe2;
  *s2_out = s2;
  *c_out = c;
  // angle <= tol  <=>  s cos(tol) <= c sin(tol)  <=>  c >= 0 and s^2 cos^2(tol) <= c^2 sin^2(tol)
  // (angle in [0, pi], s = |v| >= 0, tol in (0, pi/2))
  return pe2 <= K.tol_pos2 && c >= 0.f && s2 * K.cos2_tol <= c * c * K.sin2_tol;
}

// Could this success decision flip under a perturbation of 1e-5? It could
// when both errors are within 1e-5 above their tolerances at most and one of
// them lies within 1e-5 of its tolerance:
//   pe <= tol_pos + b  and  angle <= tol_rot + b  and
//   (pe >= tol_pos - b  or  angle >= tol_rot - b),   b = 1e-5,
// in squared form as check (angle <= x  <=>  c >= 0 and s^2 cos^2 x <= c^2 sin^2 x).
__device__ __forceinline__ bool check_banded(const IkArgs& K, float pe2, float s2, float c) {
  const float c2 = c * c;
  const bool rot_hi = c >= 0.f && s2 * K.cos2_hi <= c2 * K.sin2_hi;
  const bool rot_below_lo = c > 0.f && s2 * K.cos2_lo < c2 * K.sin2_lo;
  return pe2 <= K.pos_hi2 && rot_hi && (pe2 >= K.pos_lo2 || !rot_below_lo);
}

// One damped-least-squares step of q (in place) towards T, given the forward
// kinematics (z, p, R, t) of q and the world-frame orientation error v =
// 1/2 sum_k r_k x r*_k of rot_error.
__device__ __forceinline__ void dls_step(const ArmK& A, float lambda2, const Target& T, float q[7],
                                         const float z[7][3], const float p[7][3], const float R[9], const float t[3],
                                         const float v[3]) {
  float e[6];
  e[0] = T.p[0] - t[0];
  e[1] = T.p[1] - t[1];
  e[2] = T.p[2] - t[2];
  e[3] = v[0];
  e[4] = v[1];
  e[5] = v[2];
  // A = J J^T + lambda^2 I accumulated column by column (column i of J is
  // j_i = (z_i x (t - p_i), z_i)); J itself is not kept, J^T y below
  // rebuilds it from z and p. The first column
  // (z_0 = e_z, p_0 = 0) is (-t_y, t_x, 0, 0, 0, 1): its products are
  // written out (those with its zero and unit entries are exact). The other
  // columns update 18 of the 21 entries in pairs on the packed instructions,
  // with the column's entries paired as b0 = (j0, j1), b1 = (j3, j4), b2 =
  // (j2, j5) and the swaps s1 = (j4, j3), s2 = (j5, j2); each entry gets the
  // same multiply-adds in the same order as one by one.
  const float l2 = lambda2;
  float2 P00_11 = make_float2(fmaf(t[1], t[1], l2), fmaf(t[0], t[0], l2));
  float2 P33_44 = make_float2(l2, l2), P22_55 = make_float2(l2, 1.f + l2);
  float2 P30_41 = make_float2(0.f, 0.f), P20_51 = make_float2(0.f, t[0]), P32_54 = make_float2(0.f, 0.f);
  float2 P40_31 = make_float2(0.f, 0.f), P50_21 = make_float2(-t[1], 0.f), P53_42 = make_float2(0.f, 0.f);
  float L10 = -(t[0] * t[1]), L43 = 0.f, L52 = 0.f;
#pragma unroll
  for (int i = 1; i < 7; ++i) {
    const float ux = t[0] - p[i][0], uy = t[1] - p[i][1], uz = t[2] - p[i][2];
    const float j0 = z[i][1] * uz - z[i][2] * uy, j1 = z[i][2] * ux - z[i][0] * uz,
                j2 = z[i][0] * uy - z[i][1] * ux;
    const float2 b0 = make_float2(j0, j1), b1 = make_float2(z[i][0], z[i][1]), b2 = make_float2(j2, z[i][2]);
    const float2 s1 = make_float2(z[i][1], z[i][0]), s2 = make_float2(z[i][2], j2);
    P00_11 = __ffma2_rn(b0, b0, P00_11);
    P33_44 = __ffma2_rn(b1, b1, P33_44);
    P22_55 = __ffma2_rn(b2, b2, P22_55);
    P30_41 = __ffma2_rn(b0, b1, P30_41);
    P20_51 = __ffma2_rn(b0, b2, P20_51);
    P32_54 = __ffma2_rn(b1, b2, P32_54);
    P40_31 = __ffma2_rn(b0, s1, P40_31);
    P50_21 = __ffma2_rn(b0, s2, P50_21);
    P53_42 = __ffma2_rn(b1, s2, P53_42);
    L10 = fmaf(j1, j0, L10);
    L43 = fmaf(z[i][1], z[i][0], L43);
    L52 = fmaf(z[i][2], j2, L52);
  }
  float L[6][6];
  L[0][0] = P00_11.x; L[1][1] = P00_11.y; L[3][3] = P33_44.x; L[4][4] = P33_44.y;
  L[2][2] = P22_55.x; L[5][5] = P22_55.y; L[3][0] = P30_41.x; L[4][1] = P30_41.y;
  L[2][0] = P20_51.x; L[5][1] = P20_51.y; L[3][2] = P32_54.x; L[5][4] = P32_54.y;
  L[4][0] = P40_31.x; L[3][1] = P40_31.y; L[5][0] = P50_21.x; L[2][1] = P50_21.y;
  L[5][3] = P53_42.x; L[4][2] = P53_42.y; L[1][0] = L10; L[4][3] = L43; L[5][2] = L52;
  // Cholesky A = L L^T (lower, in place); 1 / L_jj from one reciprocal square root
  float inv_diag[6];
#pragma unroll
  for (int jc = 0; jc < 6; ++jc) {
    float d = L[jc][jc];
#pragma unroll
    for (int k = 0; k < jc; ++k) d -= L[jc][k] * L[jc][k];
    const float inv = rsqrtf(d);
    inv_diag[jc] = inv;
    L[jc][jc] = d * inv;
#pragma unroll
    for (int r = jc + 1; r < 6; ++r) {
      float v = L[r][jc];
#pragma unroll
      for (int k = 0; k < jc; ++k) v -= L[r][k] * L[jc][k];
      L[r][jc] = v * inv;
    }
  }
  float y[6];
#pragma unroll
  for (int r = 0; r < 6; ++r) {  // L w = e
    float v = e[r];
#pragma unroll
    for (int k = 0; k < r; ++k) v -= L[r][k] * y[k];
    y[r] = v * inv_diag[r];
  }
#pragma unroll
  for (int r = 5; r >= 0; --r) {  // L^T y = w
    float v = y[r];
#pragma unroll
    for (int k = r + 1; k < 6; ++k) v -= L[k][r] * y[k];
    y[r] = v * inv_diag[r];
  }
  // dq = J^T y, with the columns of J as above (the cross products are the
  // ones A was built from); with the axes up to the signs zsign, dq_i comes
  // out times zsign_i
  q[0] = fminf(fmaxf(q[0] + (fmaf(t[0], y[1], -(t[1] * y[0])) + y[5]), A.qmin[0]), A.qmax[0]);
#pragma unroll
  for (int i = 1; i < 7; ++i) {
    const float ux = t[0] - p[i][0], uy = t[1] - p[i][1], uz = t[2] - p[i][2];
    float dq = (z[i][1] * uz - z[i][2] * uy) * y[0];
    dq = fmaf(z[i][2] * ux - z[i][0] * uz, y[1], dq);
    dq = fmaf(z[i][0] * uy - z[i][1] * ux, y[2], dq);
    dq = fmaf(z[i][0], y[3], dq);
    dq = fmaf(z[i][1], y[4], dq);
    dq = fmaf(z[i][2], y[5], dq);
    q[i] = fminf(fmaxf(fmaf(A.zsign[i], dq, q[i]), A.qmin[i]), A.qmax[i]);
  }
}

__device__ __forceinline__ Target load_target(const float* tg) {
  Target T;
#pragma unroll
  for (int i = 0; i < 9; ++i) T.R[i] = __ldg(tg + i);
#pragma unroll
  for (int i = 0; i < 3; ++i) T.p[i] = __ldg(tg + 9 + i);
  return T;
}


struct Solve {
  bool found;
  bool band;   // some seed's check up to the last one was within the band (check_banded)
  int winner;  // lane holding the returned configuration
  int it;      // check index at which the solve ended
  int checks;  // checks evaluated (it + 1)
};

// Lock-step solve of one target by the whole warp (seed = lane). Returns the
// winning lane; that lane's q, pe2, s, c hold the returned configuration and
// its errors. Philox counter of seed lane: (id_lo, lane, block, id_hi).
template <bool kRight>
__device__ __forceinline__ Solve warp_solve(const IkArgs& K, const Target& T0, uint32_t id_lo, uint32_t id_hi, int lane,
                                            float q[7], float& pe2, float& s, float& c) {
  const Target T = target_frame(K.arm, T0);
  const bool active = lane < K.seeds;
  {
    const float4 u0 = draw_uniform4(K.seed, id_lo, (uint32_t)lane, 0u, id_hi);
    const float4 u1 = draw_uniform4(K.seed, id_lo, (uint32_t)lane, 1u, id_hi);
    const float u[7] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z};
#pragma unroll
    for (int j = 0; j < 7; ++j) q[j] = K.arm.qmin[j] + (K.arm.qmax[j] - K.arm.qmin[j]) * u[j];
  }
  Solve r{false, false, -1, 0, 0};
  pe2 = 0.f;
  float s2 = 0.f;
  c = 1.f;
  bool near = false;
  for (;; ++r.it) {
    float z[7][3], p[7][3], R[9], t[3], v[3];
    fk<kRight>(K.arm, q, z, p, R, t);
    const bool ok = active && check(K, T, R, t, &pe2, v, &s2, &c);
    // check_banded needs pe2 <= pos_hi2: skipped while no lane is that close
    if (__any_sync(0xFFFFFFFFu, active && pe2 <= K.pos_hi2)) near = near || (active && check_banded(K, pe2, s2, c));
    const unsigned m = __ballot_sync(0xFFFFFFFFu, ok);
    r.checks = r.it + 1;
    if (m) {
      r.winner = __ffs(m) - 1;
      r.found = true;
      r.band = __any_sync(0xFFFFFFFFu, near);
      s = sqrtf(s2);
      return r;
    }
    if (r.it == K.iters) break;
    if (active) dls_step(K.arm, K.lambda2, T, q, z, p, R, t, v);
  }
  r.band = __any_sync(0xFFFFFFFFu, near);
  s = sqrtf(s2);
  // smallest position error, lowest index on ties
  float best = active ? pe2 : 3e38f;
  int who = lane;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ob = __shfl_xor_sync(0xFFFFFFFFu, best, o);
    const int ow = __shfl_xor_sync(0xFFFFFFFFu, who, o);
    if (ob < best || (ob == best && ow < who)) { best = ob; who = ow; }
  }
  r.winner = who;
  return r;
}

// Host: arm constants (cos / sin of the twist angles) and solver parameters.
inline ArmK make_arm(const sc_arm& a) {
  ArmK k;
  const double snap = 1e-6;  // a float twist within this of a multiple of pi/2 means that multiple
  bool half_pi[7];
  for (int i = 0; i < 7; ++i) {
    k.d[i] = a.dh_d[i];
    k.a[i] = a.dh_a[i];
    const double ca = cos((double)a.dh_alpha[i]), sa = sin((double)a.dh_alpha[i]);
    half_pi[i] = fabs(ca) < snap;
    if (half_pi[i]) {
      k.ca[i] = 0.f; k.sa[i] = sa > 0.0 ? 1.f : -1.f;
    } else if (fabs(sa) < snap) {
      k.ca[i] = ca > 0.0 ? 1.f : -1.f; k.sa[i] = 0.f;
    } else {
      k.ca[i] = (float)ca; k.sa[i] = (float)sa;
    }
    k.qmin[i] = a.qmin[i];
    k.qmax[i] = a.qmax[i];
  }
  k.right = 1;
  for (int i = 1; i < 6; ++i) k.right &= half_pi[i] ? 1 : 0;
  // signs of the carried columns entering joint i (the first joint's frame is exact)
  float g0 = 1.f, g1 = 1.f, g2 = 1.f;
  k.sflip[0] = 0u; k.as[0] = k.a[0]; k.ds[0] = k.d[0]; k.zsign[0] = 1.f;
  for (int i = 1; i < 7; ++i) {
    k.sflip[i] = (k.right && g0 * g1 < 0.f) ? 0x80000000u : 0u;
    k.as[i] = k.a[i] * g0;
    k.ds[i] = k.d[i] * g2;
    k.zsign[i] = g2;
    if (k.right && i < 6) {  // (c1, c2) <- (s c2, -s n1), s = sin alpha_i
      const float sg = k.sa[i], ng1 = sg * g2, ng2 = -sg * g1;
      g1 = ng1;
      g2 = ng2;
    }
  }
  k.gs[0] = g0; k.gs[1] = g1; k.gs[2] = g2;
  return k;
}

inline void fill_params(IkArgs& K, const sc_arm& arm, const sc_ik_params& P) {
  K.arm = make_arm(arm);
  K.lambda2 = P.lambda * P.lambda;
  K.tol_pos2 = P.tol_pos * P.tol_pos;
  K.cos2_tol = (float)(cos((double)P.tol_rot) * cos((double)P.tol_rot));
  K.sin2_tol = (float)(sin((double)P.tol_rot) * sin((double)P.tol_rot));
  const double b = 1e-5, tp = P.tol_pos, tr = P.tol_rot, half_pi = 1.5707963267948966;
  K.pos_lo2 = tp > b ? (float)((tp - b) * (tp - b)) : -1.f;  // -1: no position is below the band
  K.pos_hi2 = (float)((tp + b) * (tp + b));
  const double lo = tr - b, hi = tr + b;
  K.cos2_lo = lo > 0.0 ? (float)(cos(lo) * cos(lo)) : 1.f;  // (1, 0): no angle is below the band
  K.sin2_lo = lo > 0.0 ? (float)(sin(lo) * sin(lo)) : 0.f;
  K.cos2_hi = hi < half_pi ? (float)(cos(hi) * cos(hi)) : 0.f;  // (0, 1): every angle <= pi/2 passes
  K.sin2_hi = hi < half_pi ? (float)(sin(hi) * sin(hi)) : 1.f;
  K.iters = P.iters;
  K.seeds = P.seeds;
  K.seed = P.seed;
}

}  // namespace ikc
}  // namespace sc
