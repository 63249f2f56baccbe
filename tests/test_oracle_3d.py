"""Pins for the oracle's multi-ring (fully 3-D) problem (CPU only): the
6-neighbourhood penalty against its closed form and finite differences, the
closed-form ellipsoid line integrals against quadrature, and the EM
properties (§2.2) on a 3-D system matrix."""
import math

import numpy as np
import pytest

from oracle import em
from oracle.penalty import POTENTIALS, Penalty
from oracle.siddon3d import ring_positions
from paper_2106_03172_gb300.phantoms import (Geometry, Workload, analytic_lor_sinogram, ellipsoid_solids,
                                             make_data)

GEOM = Geometry(10, 10, 12, 15, nz=3, n_rings=2, ring_mm=4.0, radius_mm=40.0, slice_mm=2.0)
WORK = Workload("t10r2", GEOM, n_subsets=3, counts=2e4, bg_frac=0.1, beta=0.02, n_ellipses=3)


@pytest.fixture(scope="module")
def prob3():
    data = make_data(WORK, 4)
    return em.build_problem(GEOM, data["g"], data["w"], WORK.n_subsets, WORK.beta), data


def test_quadratic_6_neighbourhood_closed_form():
    """R(f) = 1/2 sum over neighbouring voxel pairs (f_n - f_j)^2 for the
    quadratic potential: the sums of squared differences along x, y and z."""
    nx, ny, nz = 5, 4, 3
    vol = np.random.default_rng(1).uniform(0.0, 3.0, (ny, nx, nz))
    pen = Penalty(nx, ny, "quadratic", axial=nz)
    want = 0.5 * sum((np.diff(vol, axis=a) ** 2).sum() for a in range(3))
    assert pen.value(vol.reshape(-1, 1))[0] == pytest.approx(want, rel=1e-13)


@pytest.mark.parametrize("potential", POTENTIALS)
def test_6_neighbourhood_gradient_finite_difference(potential):
    nx, ny, nz = 4, 3, 3
    rng = np.random.default_rng(2)
    f = rng.uniform(0.2, 2.0, (nx * ny * nz, 1))
    v = rng.standard_normal(f.shape)
    pen = Penalty(nx, ny, potential, delta=0.7, axial=nz)
    h = 1e-6
    fd = (pen.value(f + h * v)[0] - pen.value(f - h * v)[0]) / (2 * h)
    assert float((pen.grad(f) * v).sum()) == pytest.approx(fd, rel=1e-6)


def test_analytic_lor_integrals_match_quadrature():
    """The closed-form chord of each ellipsoid along an oblique line of
    response equals a midpoint-rule integral of the phantom along it."""
    solids = ellipsoid_solids(GEOM, 7, 3, 0.5 * GEOM.nz * GEOM.slice_mm, body_c=0.9)
    sino = analytic_lor_sinogram(solids, GEOM)
    zr = ring_positions(GEOM.n_rings, GEOM.ring_mm)
    n = 200000
    for (i, j, r1, r2) in ((0, 7, 0, 1), (5, 3, 1, 0), (9, 11, 1, 1), (3, 7, 0, 0)):
        th = i * math.pi / GEOM.n_angles
        s = (j - 0.5 * (GEOM.n_bins - 1)) * GEOM.ds
        T = math.sqrt(GEOM.radius_mm ** 2 - s * s)
        t = -T + (np.arange(n) + 0.5) * (2 * T / n)
        x, y = s * math.cos(th) - t * math.sin(th), s * math.sin(th) + t * math.cos(th)
        z = zr[r1] + (t + T) * (zr[r2] - zr[r1]) / (2 * T)
        val = np.zeros(n)
        for (cx, cy, cz, a, b, c, phi, v) in solids:
            cp, sp = math.cos(phi), math.sin(phi)
            xr, yr = (x - cx) * cp + (y - cy) * sp, -(x - cx) * sp + (y - cy) * cp
            val += v * (((xr / a) ** 2 + (yr / b) ** 2 + ((z - cz) / c) ** 2) <= 1.0)
        stretch = math.sqrt(1.0 + ((zr[r2] - zr[r1]) / (2 * T)) ** 2)
        numeric = val.sum() * (2 * T / n) * stretch
        assert sino[i, j, r1 * GEOM.n_rings + r2] == pytest.approx(numeric, rel=2e-3, abs=1e-3)


def test_osem_one_subset_is_mlem_in_3d():
    p1 = em.build_problem(GEOM, make_data(WORK, 5)["g"], 0.5, 1, 0.0)
    f = p1.uniform_image()
    for _ in range(3):
        np.testing.assert_allclose(em.osem_step(p1, f, 0), em.mlem_step(p1, f), rtol=1e-13)
        f = em.mlem_step(p1, f)


def test_mlem_monotone_and_counts_conserved_in_3d(prob3):
    """MM property (§2.2) and count conservation on the 3-D system matrix:
    L increases, f stays >= 0, and after an MLEM step sum_n (A^T 1)_n f'_n
    equals sum_m g_m (A f)_m / (A f + w)_m."""
    prob, _ = prob3
    p1 = em.Problem(prob.A, prob.g, prob.w, [np.arange(prob.M)], 0.0, GEOM.nx, GEOM.ny, 1, axial=GEOM.nz)
    f = p1.uniform_image()
    L = p1.loglik(f)[0]
    for _ in range(5):
        yh = p1.yhat(f)
        want = float((p1.g * (p1.A @ f) / yh).sum())
        f = em.mlem_step(p1, f)
        assert float((p1.sens * f).sum()) == pytest.approx(want, rel=1e-12)
        L2 = p1.loglik(f)[0]
        assert L2 >= L - 1e-9 * abs(L) and f.min() >= 0.0
        L = L2


def test_map_em_objective_monotone_in_3d(prob3):
    """The penalised M-step with the 6-neighbourhood surrogate (§3) never
    decreases Phi (SVREM with one subset and alpha = 1 is MAP-EM)."""
    prob, _ = prob3
    p1 = em.Problem(prob.A, prob.g, prob.w, [np.arange(prob.M)], prob.beta, GEOM.nx, GEOM.ny, 1,
                    axial=GEOM.nz)
    f = p1.initial_image()
    phi = p1.objective(f)
    alg = em.SVREM(p1, f, alpha=1.0, eta=1)
    for _ in range(6):
        f = alg.step(0)
        phi2 = p1.objective(f)
        assert phi2 >= phi - 1e-10 * abs(phi)
        phi = phi2


def test_3d_problem_shapes_and_subsets(prob3):
    prob, data = prob3
    npairs = GEOM.n_rings ** 2
    assert prob.A.shape == (GEOM.n_rays * npairs, GEOM.nx * GEOM.ny * GEOM.nz)
    assert data["g"].shape == (GEOM.n_angles, GEOM.n_bins, npairs)
    rows = np.sort(np.concatenate(prob.subsets))
    np.testing.assert_array_equal(rows, np.arange(prob.M))
    for t, r in enumerate(prob.subsets):
        views = np.unique(r // (GEOM.n_bins * npairs))
        np.testing.assert_array_equal(views, np.arange(t, GEOM.n_angles, WORK.n_subsets))
