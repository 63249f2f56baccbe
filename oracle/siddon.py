"""Explicit system matrix by classical Siddon ray tracing (FP64).

The paper takes A as a nonnegative M x N matrix (§2.1, Eq. (voxel_td)) and
computes it with a Radon transform; here a_mn is the exact length (mm) of ray
m inside pixel n, built the classical Siddon way (Siddon, Med. Phys. 12, 1985):

  1. parametrise the ray as p(t) = s_j (cos, sin) + t (-sin, cos), t in mm;
  2. clip t to the closed image square;
  3. collect the parameters of all crossings with the x- and y-grid lines
     inside the clipped interval and merge them with its two ends;
  4. each piece between consecutive parameters lies in one pixel: the one
     containing its midpoint (pixels are half-open squares, so a ray lying
     exactly on a grid line is charged to the pixel on its +x / +y side and a
     ray on the far edge x = +nx*d/2 or y = +ny*d/2 contributes nothing;
     parity unpinned: a tie-break convention the paper does not fix).

``pixel_length_bruteforce`` is an independent route to the same numbers:
Liang-Barsky clipping of the line against one pixel square at a time with the
same half-open rule.  It is used by the tests to pin ``system_matrix``.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .geometry import bin_offsets, image_bounds, view_trig


def siddon_ray(c: float, s: float, sj: float, nx: int, ny: int, d: float):
    """Pixel indices (row-major iy*nx+ix) and intersection lengths of one ray."""
    x_min, x_max, y_min, y_max = image_bounds(nx, ny, d)
    px, py = sj * c, sj * s          # foot of the perpendicular from the origin
    ux, uy = -s, c                   # unit direction
    t_lo, t_hi = -np.inf, np.inf
    for p, u, lo, hi in ((px, ux, x_min, x_max), (py, uy, y_min, y_max)):
        if u == 0.0:
            if p < lo or p > hi:
                return np.zeros(0, np.int64), np.zeros(0)
        else:
            t1, t2 = (lo - p) / u, (hi - p) / u
            t_lo, t_hi = max(t_lo, min(t1, t2)), min(t_hi, max(t1, t2))
    if not t_hi > t_lo:
        return np.zeros(0, np.int64), np.zeros(0)
    ts = [np.array([t_lo, t_hi])]
    if ux != 0.0:
        tx = (x_min + d * np.arange(nx + 1) - px) / ux
        ts.append(tx[(tx > t_lo) & (tx < t_hi)])
    if uy != 0.0:
        ty = (y_min + d * np.arange(ny + 1) - py) / uy
        ts.append(ty[(ty > t_lo) & (ty < t_hi)])
    t = np.unique(np.concatenate(ts))
    length = np.diff(t)
    tm = 0.5 * (t[1:] + t[:-1])
    ix = np.floor((px + tm * ux - x_min) / d).astype(np.int64)
    iy = np.floor((py + tm * uy - y_min) / d).astype(np.int64)
    keep = (length > 0.0) & (ix >= 0) & (ix < nx) & (iy >= 0) & (iy < ny)
    return iy[keep] * nx + ix[keep], length[keep]


def system_matrix(geom) -> sp.csr_matrix:
    """CSR matrix A (M x N, float64), row m = view*n_bins + bin, column
    n = iy*nx + ix."""
    c, s = view_trig(geom.n_angles)
    sj = bin_offsets(geom.n_bins, geom.ds)
    rows, cols, vals = [], [], []
    for i in range(geom.n_angles):
        for j in range(geom.n_bins):
            idx, ln = siddon_ray(c[i], s[i], sj[j], geom.nx, geom.ny, geom.pixel_mm)
            rows.append(np.full(idx.size, i * geom.n_bins + j, np.int64))
            cols.append(idx)
            vals.append(ln)
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(geom.n_rays, geom.n_pixels))
    A = A.tocsr()
    A.sum_duplicates()
    return A


def _liang_barsky(px, py, ux, uy, x0, x1, y0, y1):
    """Length of the infinite line p + t u inside the closed box (Liang-Barsky)."""
    t_lo, t_hi = -np.inf, np.inf
    for p, u, lo, hi in ((px, ux, x0, x1), (py, uy, y0, y1)):
        if u == 0.0:
            if p < lo or p > hi:
                return 0.0
        else:
            t1, t2 = (lo - p) / u, (hi - p) / u
            t_lo, t_hi = max(t_lo, min(t1, t2)), min(t_hi, max(t1, t2))
    return max(0.0, t_hi - t_lo)


def pixel_length_bruteforce(c: float, s: float, sj: float, ix: int, iy: int,
                            nx: int, ny: int, d: float) -> float:
    """Length of ray (c, s, sj) inside the half-open pixel (ix, iy)."""
    x_min, _, y_min, _ = image_bounds(nx, ny, d)
    x0, x1 = x_min + ix * d, x_min + (ix + 1) * d
    y0, y1 = y_min + iy * d, y_min + (iy + 1) * d
    px, py, ux, uy = sj * c, sj * s, -s, c
    # half-open squares: a line lying on the +x or +y edge belongs to the neighbour
    if ux == 0.0 and px == x1:
        return 0.0
    if uy == 0.0 and py == y1:
        return 0.0
    return _liang_barsky(px, py, ux, uy, x0, x1, y0, y1)


def system_matrix_bruteforce(geom) -> np.ndarray:
    """Dense A by clipping every ray against every pixel (tiny geometries only)."""
    c, s = view_trig(geom.n_angles)
    sj = bin_offsets(geom.n_bins, geom.ds)
    A = np.zeros((geom.n_rays, geom.n_pixels))
    for i in range(geom.n_angles):
        for j in range(geom.n_bins):
            for iy in range(geom.ny):
                for ix in range(geom.nx):
                    A[i * geom.n_bins + j, iy * geom.nx + ix] = pixel_length_bruteforce(
                        c[i], s[i], sj[j], ix, iy, geom.nx, geom.ny, geom.pixel_mm)
    return A
