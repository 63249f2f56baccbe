"""Explicit 3-D system matrix of a multi-ring scanner by Siddon ray tracing (FP64).

The paper's torso experiment (§5.3) reconstructs fully 3-D data from a
scanner with 2 rings; the paper fixes no discretisation, so this module states
one (parity unpinned as a convention; the geometry itself is pinned below):

* image: nx x ny x nz voxels; voxel (ix, iy, iz) is the half-open box
  [x_min + ix d, x_min + (ix+1) d) x [y_min + iy d, ...) x
  [z_min + iz dz, z_min + (iz+1) dz) with x_min = -nx d/2, y_min = -ny d/2,
  z_min = -nz dz/2; index n = (iy nx + ix) nz + iz (axial index innermost);
* rings r = 0..n_rings-1 at axial positions z_r = (r - (n_rings-1)/2) ring_mm
  on a detector cylinder of radius R (mm);
* line of response (i, j, r1, r2): transaxially the parallel-beam ray
  x cos(theta_i) + y sin(theta_i) = s_j of the 2-D geometry, parametrised
  p(t) = s_j (cos, sin) + t (-sin, cos); it meets the cylinder at t = -T and
  t = +T, T = sqrt(R^2 - s_j^2), where it lies on ring r1 and ring r2:
  z(t) = z_r1 + (t + T) (z_r2 - z_r1) / (2T);
* sinogram index m = (i n_bins + j) n_pairs + p with p = r1 n_rings + r2
  (every ordered ring pair, n_pairs = n_rings^2; r1 = r2 are the direct planes);
* a_mn = length (mm) of line m inside voxel n: dt sqrt(1 + kappa^2) with
  kappa = dz/dt = (z_r2 - z_r1) / (2T).

``system_matrix3d`` is the classical Siddon construction (merge the line's
crossings with the x, y and z grid planes, charge each piece to the voxel of
its midpoint); ``voxel_length_bruteforce`` clips the line against one voxel box
at a time (Liang-Barsky in 3-D) with the same half-open rule, and pins it.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .geometry import bin_offsets, image_bounds, view_trig


def ring_positions(n_rings: int, ring_mm: float) -> np.ndarray:
    """Axial centres z_r of the rings (mm)."""
    return (np.arange(n_rings, dtype=np.float64) - 0.5 * (n_rings - 1)) * ring_mm


def axial_bounds(nz: int, dz: float):
    return -0.5 * nz * dz, 0.5 * nz * dz


def lor_line(c, s, sj, z1, z2, R):
    """(px, py, ux, uy, z0, kappa, T): p(t) = (px + t ux, py + t uy, z0 + kappa t)."""
    T = np.sqrt(R * R - sj * sj)
    kappa = (z2 - z1) / (2.0 * T)
    z0 = 0.5 * (z1 + z2)              # z(0): the line is linear in t
    return sj * c, sj * s, -s, c, z0, kappa, T


def _clip(p, u, lo, hi, t_lo, t_hi):
    """Intersect [t_lo, t_hi] with {t : lo <= p + t u <= hi}; None if empty."""
    if u == 0.0:
        if p < lo or p > hi:
            return None
        return t_lo, t_hi
    t1, t2 = (lo - p) / u, (hi - p) / u
    return max(t_lo, min(t1, t2)), min(t_hi, max(t1, t2))


def siddon_lor3d(c, s, sj, z1, z2, geom):
    """Voxel indices ((iy nx + ix) nz + iz) and lengths of one line of response."""
    nx, ny, nz, d, dz = geom.nx, geom.ny, geom.nz, geom.pixel_mm, geom.slice_mm
    x_min, x_max, y_min, y_max = image_bounds(nx, ny, d)
    z_min, z_max = axial_bounds(nz, dz)
    px, py, ux, uy, z0, kappa, T = lor_line(c, s, sj, z1, z2, geom.radius_mm)
    span = (-T, T)
    for p, u, lo, hi in ((px, ux, x_min, x_max), (py, uy, y_min, y_max), (z0, kappa, z_min, z_max)):
        span = _clip(p, u, lo, hi, *span)
        if span is None:
            return np.zeros(0, np.int64), np.zeros(0)
    t_lo, t_hi = span
    if not t_hi > t_lo:
        return np.zeros(0, np.int64), np.zeros(0)
    ts = [np.array([t_lo, t_hi])]
    for p, u, lo, step, n in ((px, ux, x_min, d, nx), (py, uy, y_min, d, ny), (z0, kappa, z_min, dz, nz)):
        if u != 0.0:
            tc = (lo + step * np.arange(n + 1) - p) / u
            ts.append(tc[(tc > t_lo) & (tc < t_hi)])
    t = np.unique(np.concatenate(ts))
    length = np.diff(t) * np.sqrt(1.0 + kappa * kappa)
    tm = 0.5 * (t[1:] + t[:-1])
    ix = np.floor((px + tm * ux - x_min) / d).astype(np.int64)
    iy = np.floor((py + tm * uy - y_min) / d).astype(np.int64)
    iz = np.floor((z0 + tm * kappa - z_min) / dz).astype(np.int64)
    keep = (length > 0.0) & (ix >= 0) & (ix < nx) & (iy >= 0) & (iy < ny) & (iz >= 0) & (iz < nz)
    return (iy[keep] * nx + ix[keep]) * nz + iz[keep], length[keep]


def lors(geom):
    """Yield (row, c, s, sj, z1, z2) for every line of response, in row order."""
    c, s = view_trig(geom.n_angles)
    sj = bin_offsets(geom.n_bins, geom.ds)
    zr = ring_positions(geom.n_rings, geom.ring_mm)
    npairs = geom.n_rings * geom.n_rings
    for i in range(geom.n_angles):
        for j in range(geom.n_bins):
            for r1 in range(geom.n_rings):
                for r2 in range(geom.n_rings):
                    row = (i * geom.n_bins + j) * npairs + r1 * geom.n_rings + r2
                    yield row, c[i], s[i], sj[j], zr[r1], zr[r2]


def system_matrix3d(geom) -> sp.csr_matrix:
    """CSR matrix A (M x N, float64): M = n_angles n_bins n_rings^2 lines of
    response, N = nx ny nz voxels, in the index orders stated above."""
    rows, cols, vals = [], [], []
    for row, c, s, sj, z1, z2 in lors(geom):
        idx, ln = siddon_lor3d(c, s, sj, z1, z2, geom)
        rows.append(np.full(idx.size, row, np.int64))
        cols.append(idx)
        vals.append(ln)
    M = geom.n_angles * geom.n_bins * geom.n_rings ** 2
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(M, geom.nx * geom.ny * geom.nz)).tocsr()
    A.sum_duplicates()
    return A


def line_length_in_box(px, py, ux, uy, z0, kappa, T, box):
    """Length of the segment t in [-T, T] of the line inside the closed box
    (x0, x1, y0, y1, z0, z1), by Liang-Barsky clipping."""
    x0, x1, y0, y1, zlo, zhi = box
    span = (-T, T)
    for p, u, lo, hi in ((px, ux, x0, x1), (py, uy, y0, y1), (z0, kappa, zlo, zhi)):
        span = _clip(p, u, lo, hi, *span)
        if span is None:
            return 0.0
    return max(0.0, span[1] - span[0]) * np.sqrt(1.0 + kappa * kappa)


def voxel_length_bruteforce(c, s, sj, z1, z2, ix, iy, iz, geom) -> float:
    """Length of one line of response inside the half-open voxel (ix, iy, iz)."""
    d, dz = geom.pixel_mm, geom.slice_mm
    x_min, _, y_min, _ = image_bounds(geom.nx, geom.ny, d)
    z_min, _ = axial_bounds(geom.nz, dz)
    box = (x_min + ix * d, x_min + (ix + 1) * d, y_min + iy * d, y_min + (iy + 1) * d,
           z_min + iz * dz, z_min + (iz + 1) * dz)
    px, py, ux, uy, z0, kappa, T = lor_line(c, s, sj, z1, z2, geom.radius_mm)
    # half-open boxes: a line lying in a +x, +y or +z face belongs to the neighbour
    if ux == 0.0 and px == box[1]:
        return 0.0
    if uy == 0.0 and py == box[3]:
        return 0.0
    if kappa == 0.0 and z0 == box[5]:
        return 0.0
    return line_length_in_box(px, py, ux, uy, z0, kappa, T, box)


def system_matrix3d_bruteforce(geom) -> np.ndarray:
    """Dense A by clipping every line of response against every voxel (tiny geometries only)."""
    M = geom.n_angles * geom.n_bins * geom.n_rings ** 2
    A = np.zeros((M, geom.nx * geom.ny * geom.nz))
    for row, c, s, sj, z1, z2 in lors(geom):
        for iy in range(geom.ny):
            for ix in range(geom.nx):
                for iz in range(geom.nz):
                    A[row, (iy * geom.nx + ix) * geom.nz + iz] = voxel_length_bruteforce(
                        c, s, sj, z1, z2, ix, iy, iz, geom)
    return A
