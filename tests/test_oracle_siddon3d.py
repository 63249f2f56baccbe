"""Pins for the oracle's multi-ring (fully 3-D) system matrix (CPU only).

The 3-D Siddon matrix is pinned against things other than itself: a
brute-force per-voxel Liang-Barsky clipper in 3-D, the 2-D matrix (direct
planes through voxel centres are the 2-D rays in one layer), and the axial
stretch sqrt(1 + kappa^2) of an oblique line's transaxial chord.
"""
import math

import numpy as np
import pytest

from oracle.siddon import system_matrix
from oracle.siddon3d import (axial_bounds, lor_line, ring_positions, system_matrix3d,
                             system_matrix3d_bruteforce)
from paper_2106_03172_gb300.phantoms import Geometry

# rings at voxel centres (slice = ring/2, nz = 2 rings - 1), as scanners bin direct and cross planes
TWO_RINGS = Geometry(8, 8, 6, 9, nz=3, n_rings=2, ring_mm=4.0, radius_mm=40.0, slice_mm=2.0)
THREE_RINGS = Geometry(7, 6, 8, 11, pixel_mm=1.5, bin_mm=1.2, nz=5, n_rings=3, ring_mm=3.0,
                       radius_mm=30.0, slice_mm=1.5)
# steep lines (small radius, wide ring spacing): pieces cross several z planes
STEEP = Geometry(6, 6, 6, 7, nz=5, n_rings=3, ring_mm=6.0, radius_mm=9.0, slice_mm=3.0)
# rings on voxel faces z = -4, 0, +4: direct planes lie in z planes (half-open rule)
ON_FACES = Geometry(6, 6, 4, 7, nz=2, n_rings=3, ring_mm=4.0, radius_mm=30.0, slice_mm=4.0)


@pytest.mark.parametrize("geom", [TWO_RINGS, THREE_RINGS, STEEP, ON_FACES])
def test_siddon3d_equals_bruteforce(geom):
    A = system_matrix3d(geom).toarray()
    B = system_matrix3d_bruteforce(geom)
    assert A.shape == B.shape == (geom.n_angles * geom.n_bins * geom.n_rings ** 2,
                                  geom.nx * geom.ny * geom.nz)
    np.testing.assert_allclose(A, B, rtol=0, atol=1e-12)
    assert np.count_nonzero(A) > 0


@pytest.mark.parametrize("geom", [TWO_RINGS, THREE_RINGS])
def test_direct_planes_are_the_2d_rays(geom):
    """A line of response between a ring and itself runs at constant z = z_r;
    with z_r inside layer iz(r) it is the 2-D ray of its view and bin, in
    that layer only."""
    A3 = system_matrix3d(geom).toarray()
    A2 = system_matrix(geom).toarray()
    npairs, nz = geom.n_rings ** 2, geom.nz
    z_min, _ = axial_bounds(nz, geom.slice_mm)
    for r, z in enumerate(ring_positions(geom.n_rings, geom.ring_mm)):
        iz = int(math.floor((z - z_min) / geom.slice_mm))
        rows = np.arange(geom.n_rays) * npairs + r * geom.n_rings + r
        block = A3[rows].reshape(geom.n_rays, geom.nx * geom.ny, nz)
        np.testing.assert_allclose(block[:, :, iz], A2, rtol=0, atol=1e-12)
        assert not np.delete(block, iz, axis=2).any()


def test_direct_planes_on_voxel_faces_go_to_the_upper_layer():
    """Voxels are half-open in z too: a direct plane on the face between two
    layers belongs to the upper one, on the image's bottom face to layer 0,
    and on its top face to no voxel."""
    g = ON_FACES
    A3 = system_matrix3d(g).toarray()
    A2 = system_matrix(g).toarray()

    def direct(r):
        return A3[np.arange(g.n_rays) * 9 + 4 * r].reshape(g.n_rays, g.nx * g.ny, 2)

    for r, layer in ((0, 0), (1, 1)):                 # z = -4 (bottom face), z = 0 (layers 0|1)
        np.testing.assert_allclose(direct(r)[:, :, layer], A2, atol=1e-12)
        assert not direct(r)[:, :, 1 - layer].any()
    assert not direct(2).any()                        # z = +4 (top face)


@pytest.mark.parametrize("geom", [TWO_RINGS, THREE_RINGS, STEEP])
def test_row_sums_are_stretched_2d_chords(geom):
    """While the line stays inside the image's axial extent over its
    transaxial chord (true here: the rings lie inside it), its 3-D length is
    the 2-D chord times sqrt(1 + kappa^2), kappa = (z_r2 - z_r1) / (2T)."""
    z_min, z_max = axial_bounds(geom.nz, geom.slice_mm)
    zr = ring_positions(geom.n_rings, geom.ring_mm)
    assert zr.min() >= z_min and zr.max() < z_max
    A3 = system_matrix3d(geom)
    chord2 = np.asarray(system_matrix(geom).sum(axis=1)).ravel()
    got = np.asarray(A3.sum(axis=1)).ravel().reshape(geom.n_rays, geom.n_rings, geom.n_rings)
    s = (np.arange(geom.n_bins) - 0.5 * (geom.n_bins - 1)) * geom.ds
    T = np.sqrt(geom.radius_mm ** 2 - s ** 2)
    for r1 in range(geom.n_rings):
        for r2 in range(geom.n_rings):
            kappa = (zr[r2] - zr[r1]) / (2.0 * np.tile(T, geom.n_angles))
            np.testing.assert_allclose(got[:, r1, r2], chord2 * np.sqrt(1.0 + kappa ** 2), rtol=1e-12, atol=1e-12)


def test_oblique_line_parametrisation():
    """The line of response runs from ring r1 at t = -T to ring r2 at t = +T
    on the detector cylinder."""
    R, s = 40.0, 7.0
    px, py, ux, uy, z0, kappa, T = lor_line(0.6, 0.8, s, -2.0, 6.0, R)
    for t, z in ((-T, -2.0), (T, 6.0)):
        x, y = px + t * ux, py + t * uy
        assert math.hypot(x, y) == pytest.approx(R, rel=1e-14)
        assert z0 + kappa * t == pytest.approx(z, abs=1e-13)
