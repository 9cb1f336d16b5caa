// 4D reachability map (RM4D-style, Sec. IV-E): the cell key and score
// (device) and the launchers used by the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace sc {

// Cell grid over (height, cosine of the approach tilt, x*, y*); the scale
// factors are FP32 values the host computes once (bins per metre, per unit
// of cosine) so that every cell index is one fixed sequence of IEEE
// operations.
struct RmapGrid {
  int nz, nc, nxy;
  float z_lo, sz;   // height bin = floor((z - z_lo) * sz)
  float sc;         // tilt bin = floor((a_z + 1) * sc), the top bin closed
  float r_max, sxy; // x* / y* bin = floor((x* + r_max) * sxy)
  size_t cells;     // nz * nc * nxy * nxy
};

// 4D reachability map in the manner of RM4D (Sec. IV-E: the paper queries an
// RM4D map, batched on the GPU). A pose's reachability by an arm whose first
// joint turns about the base z axis does not change when the pose turns about
// that axis, so a target (R, p) in the base frame is keyed by four numbers:
// its height p_z, the cosine a_z of the tilt of its approach axis a = R e_z,
// and its position (x*, y*) in the frame turned about z until the azimuth
// reference h lies on +x. h is the horizontal direction of a; for a vertical
// approach (|a_xy|^2 <= 1e-6), where that direction is undefined, the
// horizontal direction of the tool x axis R e_x, which carries the grasp's
// yaw. Every step is an IEEE-rounded FP32 operation (no contraction), so a
// host implementation of the same sequence gets the same cell. Returns the
// cell of t ([12]: R row-major, then p), or -1 outside the grid.
__device__ __forceinline__ int rmap_cell(const RmapGrid& g, const float t[12]) {
  const float ax = t[2], ay = t[5], az = t[8];  // third column of R
  const float bx = t[0], by = t[3];             // first column of R
  const bool tilted = __fadd_rn(__fmul_rn(ax, ax), __fmul_rn(ay, ay)) > 1e-6f;
  const float ux = tilted ? ax : bx, uy = tilted ? ay : by;
  const float n2 = __fadd_rn(__fmul_rn(ux, ux), __fmul_rn(uy, uy));
  if (!(n2 > 0.f)) return -1;
  const float inv = __fdiv_rn(1.f, __fsqrt_rn(n2));
  const float hx = __fmul_rn(ux, inv), hy = __fmul_rn(uy, inv);
  const float px = t[9], py = t[10], pz = t[11];
  const float xs = __fadd_rn(__fmul_rn(px, hx), __fmul_rn(py, hy));
  const float ys = __fsub_rn(__fmul_rn(py, hx), __fmul_rn(px, hy));
  const float fz = __fmul_rn(__fsub_rn(pz, g.z_lo), g.sz);
  const float fc = __fmul_rn(__fadd_rn(az, 1.f), g.sc);
  const float fx = __fmul_rn(__fadd_rn(xs, g.r_max), g.sxy);
  const float fy = __fmul_rn(__fadd_rn(ys, g.r_max), g.sxy);
  // the comparisons are false for NaN
  if (!(fz >= 0.f && fz < (float)g.nz && fx >= 0.f && fx < (float)g.nxy && fy >= 0.f && fy < (float)g.nxy &&
        fc >= 0.f))
    return -1;
  const int iz = (int)fz, ix = (int)fx, iy = (int)fy;  // truncation is floor here (f >= 0)
  const int ic = fc < (float)g.nc ? (int)fc : g.nc - 1;
  return ((iz * g.nc + ic) * g.nxy + ix) * g.nxy + iy;
}

// floor(65535 * reachable / labels) of a cell; 65535 for a cell without
// labels (no evidence, so no rejection); 0 outside the grid, which is meant
// to cover the arm's workspace.
__device__ __forceinline__ unsigned int rmap_score(const uint2* counts, int cell) {
  if (cell < 0) return 0u;
  const uint2 c = counts[cell];
  return c.y ? (unsigned int)(((unsigned long long)c.x * 65535ull) / c.y) : 65535u;
}

// counts[cell] = (reachable labels, labels), accumulated over n targets
// ([n][12]: R row-major, then p; base frame) with labels u8 [n].
cudaError_t rmap_build(const RmapGrid& g, uint2* counts, const float* targets, const uint8_t* labels, int n,
                       int num_sms, cudaStream_t s);

// score[i] = floor(65535 * reachable / labels) of target i's cell; 65535
// for a cell without labels, 0 for a target outside the grid.
cudaError_t rmap_query(const RmapGrid& g, const uint2* counts, const float* targets, int n, uint16_t* score,
                       int num_sms, cudaStream_t s);

}  // namespace sc
