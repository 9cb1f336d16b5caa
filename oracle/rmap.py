"""Oracle of the 4D reachability map (TEST INFRASTRUCTURE ONLY; see the
package docstring for who may use it).

The paper's reachability check queries an RM4D map (Sec. IV-E). This is the
plain definition of the map the library builds from labelled IK outcomes:
every target gets a cell of a 4D grid (height, cosine of the approach tilt,
and the position turned about the base z axis to the approach azimuth), each
cell counts (reachable labels, labels), a query reads its cell's counts.

The cell index is an integer decided by floating point, so it is computed in
FP32, one IEEE-rounded numpy operation per step in the order the library
states (numpy never fuses a multiply and an add); counts and scores are
integers.
"""
from __future__ import annotations

import numpy as np

F = np.float32


def grid(params):
    """(nz, nc, nxy, z_lo, sz, sc, r_max, sxy): the FP32 scale factors of the
    bins, each one FP32 division."""
    nz, nc, nxy, z_lo, z_hi, r_max = params
    span = F(z_hi) - F(z_lo)
    return (int(nz), int(nc), int(nxy), F(z_lo), F(nz) / span, F(nc) / F(2), F(r_max), F(nxy) / (F(2) * F(r_max)))


def cells(params, targets) -> np.ndarray:
    """Cell of every target ([n][12] float32: R row-major, p), -1 outside the grid."""
    nz, nc, nxy, z_lo, sz, sc, r_max, sxy = grid(params)
    t = np.asarray(targets, dtype=F).reshape(-1, 12)
    ax, ay, az = t[:, 2], t[:, 5], t[:, 8]  # approach axis: third column of R
    bx, by = t[:, 0], t[:, 3]  # tool x axis: first column of R
    with np.errstate(all="ignore"):
        tilted = (ax * ax + ay * ay) > F(1e-6)
        ux = np.where(tilted, ax, bx)
        uy = np.where(tilted, ay, by)
        n2 = ux * ux + uy * uy
        inv = F(1) / np.sqrt(n2)
        hx, hy = ux * inv, uy * inv
        px, py, pz = t[:, 9], t[:, 10], t[:, 11]
        xs = px * hx + py * hy  # position turned about z by minus the azimuth of h
        ys = py * hx - px * hy
        fz = (pz - z_lo) * sz
        fc = (az + F(1)) * sc
        fx = (xs + r_max) * sxy
        fy = (ys + r_max) * sxy
        ok = (n2 > 0) & (fz >= 0) & (fz < F(nz)) & (fx >= 0) & (fx < F(nxy)) & (fy >= 0) & (fy < F(nxy)) & (fc >= 0)
        iz = np.floor(np.where(ok, fz, 0)).astype(np.int64)
        ix = np.floor(np.where(ok, fx, 0)).astype(np.int64)
        iy = np.floor(np.where(ok, fy, 0)).astype(np.int64)
        ic = np.where(ok & (fc < F(nc)), np.floor(np.where(ok, fc, 0)), nc - 1).astype(np.int64)
    cell = ((iz * nc + ic) * nxy + ix) * nxy + iy
    return np.where(ok, cell, -1)


def n_cells(params) -> int:
    nz, nc, nxy = int(params[0]), int(params[1]), int(params[2])
    return nz * nc * nxy * nxy


def build(params, targets, labels) -> np.ndarray:
    """uint32 [cells][2] = (reachable labels, labels) per cell."""
    c = cells(params, targets)
    y = np.asarray(labels).astype(bool)
    keep = c >= 0
    counts = np.zeros((n_cells(params), 2), np.uint64)
    np.add.at(counts[:, 1], c[keep], 1)
    np.add.at(counts[:, 0], c[keep & y], 1)
    return counts.astype(np.uint32)


def score(params, counts, targets) -> np.ndarray:
    """uint16 floor(65535 * reachable / labels) of each target's cell; 65535
    for a cell without labels, 0 for a target without a cell."""
    c = cells(params, targets)
    pos = np.where(c >= 0, counts[np.maximum(c, 0), 0], 0).astype(np.uint64)
    tot = np.where(c >= 0, counts[np.maximum(c, 0), 1], 0).astype(np.uint64)
    s = np.where(tot > 0, (pos * 65535) // np.maximum(tot, 1), 65535)
    return np.where(c >= 0, s, 0).astype(np.uint16)


def tune(scores, labels, min_recall: float):
    """Largest tau with recall >= min_recall when passing score >= tau; (tau,
    recall, pass rate)."""
    s = np.asarray(scores).astype(np.int64)
    y = np.asarray(labels).astype(bool)
    pos = np.sort(s[y])[::-1]
    need = int(np.ceil(float(F(min_recall)) * len(pos)))  # the library takes min_recall as an FP32 value
    tau = int(pos[min(len(pos), max(need, 1)) - 1])
    passed = s >= tau
    return tau, float((passed & y).sum()) / len(pos), float(passed.mean())
