"""Parallel-beam geometry of the oracle (FP64).

The paper's forward model is "the Radon transform" over evenly spaced views
(§5.1: 180 views at 1 degree); the discretisation below is the one the GPU
library also uses, derived independently here:

* pixel (ix, iy) is the square [x_min + ix*d, x_min + (ix+1)*d) x
  [y_min + iy*d, y_min + (iy+1)*d) with x_min = -nx*d/2, y_min = -ny*d/2;
* view i has angle theta_i = i*pi/n_angles;
* bin j has signed offset s_j = (j - (n_bins-1)/2) * ds;
* ray (i, j) is the line x cos(theta_i) + y sin(theta_i) = s_j.

cos/sin are evaluated in FP64 and values within 1e-12 of 0 or +-1 are snapped
to exactly 0 / +-1, so that axis-aligned views are exactly axis-aligned
(parity unpinned: a convention the paper does not fix).
"""
from __future__ import annotations

import numpy as np


def view_trig(n_angles: int):
    """Snapped (cos theta_i, sin theta_i), i = 0..n_angles-1, float64."""
    th = np.arange(n_angles, dtype=np.float64) * (np.pi / n_angles)
    c, s = np.cos(th), np.sin(th)
    for v in (c, s):
        v[np.abs(v) < 1e-12] = 0.0
        v[np.abs(v - 1.0) < 1e-12] = 1.0
        v[np.abs(v + 1.0) < 1e-12] = -1.0
    return c, s


def bin_offsets(n_bins: int, ds: float):
    """Signed radial offsets s_j of the bin centres (mm), float64."""
    return (np.arange(n_bins, dtype=np.float64) - 0.5 * (n_bins - 1)) * ds


def image_bounds(nx: int, ny: int, d: float):
    """(x_min, x_max, y_min, y_max) of the image square (mm)."""
    return -0.5 * nx * d, 0.5 * nx * d, -0.5 * ny * d, 0.5 * ny * d
