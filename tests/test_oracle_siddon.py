"""Pins for the oracle's system matrix (CPU only).

The Siddon matrix is pinned against things other than itself: a brute-force
per-pixel Liang-Barsky clipper, the closed-form chord of the image square, the
bound sqrt(2)*d on one pixel's chord, and the chord 2 sqrt(R^2 - s^2) of a
disk, approached at first order as the pixel size shrinks.
"""
import math

import numpy as np
import pytest

from oracle.geometry import bin_offsets, view_trig
from oracle.siddon import siddon_ray, system_matrix, system_matrix_bruteforce
from paper_2106_03172_gb300.phantoms import Geometry


@pytest.mark.parametrize("geom", [
    Geometry(8, 8, 12, 13),                       # views at 0/45/90/135 deg, rays on grid lines
    Geometry(7, 5, 10, 11, pixel_mm=1.5, bin_mm=1.1),   # non-square, odd sizes
    Geometry(6, 6, 8, 9, pixel_mm=2.0, bin_mm=1.0),     # rays through pixel corners at 45 deg
])
def test_siddon_equals_bruteforce(geom):
    A = system_matrix(geom).toarray()
    B = system_matrix_bruteforce(geom)
    assert A.shape == B.shape
    np.testing.assert_allclose(A, B, rtol=0, atol=1e-12)


def _square_chord(c, s, off, half):
    """Closed-form chord of the square [-half, half]^2 cut by x c + y s = off
    (trapezoidal projection of a square)."""
    a, b = sorted((abs(c), abs(s)), reverse=True)      # a >= b
    if abs(off) <= half * (a - b):
        return 2.0 * half / a
    if abs(off) < half * (a + b):
        return (half * (a + b) - abs(off)) / (a * b)
    return 0.0


def test_row_sums_are_square_chords():
    geom = Geometry(32, 32, 36, 47, pixel_mm=2.0, bin_mm=1.7)
    A = system_matrix(geom)
    rows = np.asarray(A.sum(axis=1)).ravel()
    c, s = view_trig(geom.n_angles)
    sj = bin_offsets(geom.n_bins, geom.ds)
    half = 0.5 * geom.nx * geom.pixel_mm
    for i in range(geom.n_angles):
        for j in range(geom.n_bins):
            exp = _square_chord(c[i], s[i], sj[j], half)
            assert rows[i * geom.n_bins + j] == pytest.approx(exp, abs=1e-10)


def test_half_open_edge_rule():
    """Axis-aligned rays on the left/bottom edge see the whole image, on the
    right/top edge see nothing (the half-open pixel convention)."""
    nx, d = 4, 2.0
    # theta = 0: line x = s
    idx, ln = siddon_ray(1.0, 0.0, -4.0, nx, nx, d)
    assert set(idx % nx) == {0} and ln.sum() == pytest.approx(8.0)
    idx, ln = siddon_ray(1.0, 0.0, 4.0, nx, nx, d)
    assert idx.size == 0
    # a ray on an interior grid line goes to the +x column
    idx, ln = siddon_ray(1.0, 0.0, 0.0, nx, nx, d)
    assert set(idx % nx) == {2} and ln.sum() == pytest.approx(8.0)
    # theta = 90 deg: line y = s
    idx, ln = siddon_ray(0.0, 1.0, 2.0, nx, nx, d)
    assert set(idx // nx) == {3} and ln.sum() == pytest.approx(8.0)


def test_entries_bounded():
    geom = Geometry(24, 24, 30, 35, bin_mm=1.3)
    A = system_matrix(geom)
    assert A.data.min() > 0.0
    assert A.data.max() <= math.sqrt(2.0) * geom.pixel_mm + 1e-12


def _disk_error(n, radius_mm, fov_mm):
    d = fov_mm / n
    geom = Geometry(n, n, 16, 2 * n + 1, pixel_mm=d, bin_mm=d / 2)
    A = system_matrix(geom)
    xs = (np.arange(n) - 0.5 * (n - 1)) * d
    X, Y = np.meshgrid(xs, xs)
    disk = ((X ** 2 + Y ** 2) <= radius_mm ** 2).astype(float).ravel()
    proj = (A @ disk).reshape(geom.n_angles, geom.n_bins)
    s = bin_offsets(geom.n_bins, geom.ds)
    sel = np.abs(s) <= 0.9 * radius_mm
    exact = 2.0 * np.sqrt(radius_mm ** 2 - s[sel] ** 2)
    return float(np.mean(np.abs(proj[:, sel] - exact[None, :]))), d


def test_disk_chord_first_order():
    e1, d1 = _disk_error(32, 20.0, 64.0)
    e2, d2 = _disk_error(64, 20.0, 64.0)
    e3, d3 = _disk_error(128, 20.0, 64.0)
    assert e1 < 1.5 * d1 and e2 < 1.5 * d2 and e3 < 1.5 * d3
    assert e2 < 0.75 * e1 and e3 < 0.75 * e2
