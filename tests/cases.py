"""Seeded parity cases shared by the GPU tests (inputs only; the oracle side is
built here from ``oracle`` and the GPU side from the binding)."""
from __future__ import annotations

import functools
from dataclasses import replace

import numpy as np

from paper_2106_03172_gb300.phantoms import WORKLOADS, Geometry, Workload, make_data

CASES = {
    # 64x64, 60 views x 91 bins, 6 subsets (the small benchmark configuration)
    "c64": WORKLOADS["c64"],
    # odd, non-square image, ragged subsets (23 views / 5 subsets), bins != pixels
    "ragged": Workload("ragged", Geometry(37, 29, 23, 41, pixel_mm=1.7, bin_mm=1.3), n_subsets=5,
                       counts=3e5, bg_frac=0.1, beta=0.02, n_ellipses=5),
    # slice stack, slice index innermost
    "stack": replace(WORKLOADS["c128x47"], name="stack",
                     geometry=Geometry(24, 24, 18, 35, bin_mm=1.4, nz=5), n_subsets=3, counts=2e5),
    # deeper stacks: 20 slices (4 per z-lane), 70 slices (two slice windows of a warp, the second ragged)
    "stack20": replace(WORKLOADS["c128x47"], name="stack20",
                       geometry=Geometry(20, 16, 14, 27, bin_mm=1.5, nz=20), n_subsets=3, counts=2e5),
    "stack70": replace(WORKLOADS["c128x47"], name="stack70",
                       geometry=Geometry(12, 10, 11, 19, bin_mm=1.3, nz=70), n_subsets=4, counts=3e5),
}

# edge cases of the method
EDGE_CASES = {
    # no background (w = 0) and bins wider than the image: 324 of 1704 rays miss
    # the image, so yhat = 0 there (ratio 0, §2.3 remedy) and their counts are 0;
    # low counts leave most rays with g = 0
    "nobg": Workload("nobg", Geometry(40, 28, 24, 71, pixel_mm=2.0, bin_mm=1.5), n_subsets=4, counts=4e3,
                     bg_frac=0.0, beta=0.02, n_ellipses=4),
    # four views and nine narrow bins: 4 pixels no ray reaches (sens_n = 0) and
    # 225 / 120 pixels outside one subset's rays (sens_t,n = 0), so the M-step's
    # S_n = 0 branch (f_n = 0) and zero preconditioner entries are taken
    "sparse": Workload("sparse", Geometry(24, 24, 4, 9, pixel_mm=2.0, bin_mm=2.0), n_subsets=2, counts=2e4,
                       bg_frac=0.1, beta=0.02, n_ellipses=4),
}
CASES.update(EDGE_CASES)

# multi-ring volumes (fully 3-D lines of response)
RING_CASES = {
    # two rings on a clinical-size cylinder (kappa <= ~0.007), rings at layer centres
    "ring2": Workload("ring2", Geometry(32, 32, 30, 47, nz=3, n_rings=2, ring_mm=4.0, radius_mm=300.0,
                                       slice_mm=2.0), n_subsets=5, counts=3e5, bg_frac=0.1, beta=0.02, n_ellipses=5),
    # three rings on a narrow cylinder: steep lines whose pieces cross layer faces
    "ring3steep": Workload("ring3steep", Geometry(24, 20, 18, 33, bin_mm=1.6, nz=6, n_rings=3, ring_mm=7.0,
                                                  radius_mm=36.0, slice_mm=3.0),
                           n_subsets=3, counts=2e5, bg_frac=0.1, beta=0.02, n_ellipses=4),
    # four rings (16 lines per ray) through a 10-layer volume: the per-voxel back projection for tall volumes
    "ring4tall": Workload("ring4tall", Geometry(12, 12, 8, 17, nz=10, n_rings=4, ring_mm=3.0, radius_mm=30.0,
                                                slice_mm=1.5), n_subsets=2, counts=1e5, bg_frac=0.1, beta=0.02,
                          n_ellipses=3),
    # rings on layer faces (z = -4, 0, +4): half-open layers decide the direct planes
    "ringfaces": Workload("ringfaces", Geometry(16, 16, 12, 23, nz=2, n_rings=3, ring_mm=4.0, radius_mm=40.0,
                                                slice_mm=4.0), n_subsets=4, counts=1e5, bg_frac=0.1, beta=0.02,
                          n_ellipses=3),
}
CASES.update(RING_CASES)


@functools.lru_cache(maxsize=None)
def oracle_problem(name: str, seed: int = 0):
    """(oracle Problem, data dict) for a named case or workload."""
    from oracle.em import build_problem
    work = CASES.get(name) or WORKLOADS[name]
    data = make_data(work, seed)
    prob = build_problem(work.geometry, data["g"], data["w"], work.n_subsets, work.beta, work.potential, work.delta)
    return prob, data, work


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
