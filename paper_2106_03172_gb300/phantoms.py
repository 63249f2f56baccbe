"""Seeded synthetic inputs for penalised PET reconstruction.

This module is the only code that both the CUDA path and the FP64 oracle
consume.  It holds none of the reconstruction arithmetic: no system matrix,
no projector, no likelihood, no update rule.  It produces

* the scanner/image geometry of each named workload (parallel-beam 2-D
  sinograms, §5 of the paper uses the same kind of data with a Radon
  transform forward model);
* random-ellipse (and ellipsoid-stack) activity phantoms;
* Poisson count data ``g ~ Poisson(p + w)`` (§2.1, Eq. (voxel_td)/(pdf)),
  where ``p`` is the *analytic* line integral of the continuous ellipse
  phantom (the closed-form Radon transform of an ellipse), so that the data
  model never goes through the discrete projector under test;
* the subset index sequences ``t_k`` that the stochastic methods draw
  (§2.3: indices drawn uniformly at random), from SplitMix64 (Steele, Lea and
  Flood, OOPSLA 2014) so that both sides consume the identical sequence.

Units: lengths in mm, activity per pixel in arbitrary units scaled so that the
expected trues sum to the requested total counts.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Geometry", "Workload", "WORKLOADS", "Ellipse", "random_ellipse_phantom",
    "ellipsoid_stack_phantom", "ellipsoid_solids", "rasterise", "analytic_sinogram",
    "analytic_lor_sinogram", "rasterise_volume", "make_data",
    "splitmix64", "subset_sequence", "batched_workloads", "serving_workloads", "serving_pool",
    "serving_requests", "subset_sequences",
]


@dataclass(frozen=True)
class Geometry:
    """2-D parallel-beam geometry, optionally with ``nz`` independent slices,
    or (``n_rings`` > 0) a multi-ring scanner with fully 3-D lines of response.

    Image: ``nx`` x ``ny`` square pixels of side ``pixel_mm`` centred on the
    origin, stored row-major ``[iy][ix]`` (slice / axial index innermost when
    nz > 1).  Sinogram: ``n_angles`` views at ``theta_i = i*pi/n_angles`` and
    ``n_bins`` radial bins centred on the origin with spacing ``bin_mm``,
    stored ``[view][bin]`` (slice index innermost when nz > 1).

    Multi-ring mode: the nz image layers are ``slice_mm`` thick and centred
    on z = 0; ``n_rings`` rings ``ring_mm`` apart (centred on z = 0) sit on a
    cylinder of radius ``radius_mm``; the sinogram is ``[view][bin][pair]``
    with one line of response per ordered ring pair, pair = r1 n_rings + r2.
    """

    nx: int
    ny: int
    n_angles: int
    n_bins: int
    pixel_mm: float = 2.0
    bin_mm: float | None = None
    nz: int = 1
    n_rings: int = 0
    ring_mm: float = 0.0
    radius_mm: float = 0.0
    slice_mm: float = 0.0

    @property
    def multiring(self) -> bool:
        return self.n_rings > 0

    @property
    def n_pairs(self) -> int:
        """Sinogram entries per (view, bin): ring pairs, or slices of a stack."""
        return self.n_rings * self.n_rings if self.multiring else self.nz

    @property
    def ds(self) -> float:
        return self.pixel_mm if self.bin_mm is None else self.bin_mm

    @property
    def n_pixels(self) -> int:
        return self.nx * self.ny

    @property
    def n_rays(self) -> int:
        return self.n_angles * self.n_bins


@dataclass(frozen=True)
class Workload:
    """A named reconstruction workload: geometry, phantom recipe and method knobs."""

    name: str
    geometry: Geometry
    n_subsets: int
    counts: float
    bg_frac: float
    beta: float
    n_ellipses: int
    n_lesions: int = 0
    epochs: int = 10
    methods: tuple = ("osem", "svrem")
    eta_svrg: int = 2
    eta_svrem: int = 1
    alpha_svrem: float = 0.7
    alpha_saga: float = 1.0
    alpha_svrg: float = 2.0
    stack: bool = False
    potential: str = "quadratic"
    delta: float = 1.0
    extra: dict = field(default_factory=dict)


# Named workloads (sizes, counts, penalties and subset numbers of the
# benchmark configurations).  Step sizes start from the paper's brain-phantom
# values (§5.1: alpha=2 for SAGA/SVRG with eta=2, alpha=0.7 and eta=1 for
# SVREM); SAGA uses alpha=1 because alpha=2 diverges on these phantoms in the
# FP64 oracle (the paper reports SAGA's sensitivity to large steps, §5.2).
WORKLOADS = {
    "c64": Workload(
        "c64", Geometry(64, 64, 60, 91), n_subsets=6, counts=1e5, bg_frac=0.10,
        beta=0.01, n_ellipses=8, epochs=10, methods=("osem", "svrem")),
    "c256": Workload(
        "c256", Geometry(256, 256, 180, 367), n_subsets=21, counts=1e7, bg_frac=0.10,
        beta=0.005, n_ellipses=20, n_lesions=6, epochs=50,
        methods=("osem", "svrem", "saga", "svrg")),
    "c128x47": Workload(
        "c128x47", Geometry(128, 128, 252, 344, bin_mm=math.sqrt(2.0) * 128 * 2.0 / 344, nz=47),
        n_subsets=14, counts=5e8, bg_frac=0.15, beta=0.002, n_ellipses=10, epochs=10,
        methods=("svrg",), eta_svrg=2, stack=True),
    # fully 3-D data of a 2-ring scanner, shaped after the torso experiment of §5.3 (280 views,
    # 20 subsets of 14 views, log-cosh penalty with delta = 1, SVRG anchor every 5 epochs and
    # SVREM every 3): 128 x 128 x 3 volume (direct and cross planes, slice = ring/2)
    "ring2_128": Workload(
        "ring2_128", Geometry(128, 128, 280, 183, nz=3, n_rings=2, ring_mm=4.0, radius_mm=400.0, slice_mm=2.0),
        n_subsets=20, counts=1e7, bg_frac=0.10, beta=0.005, n_ellipses=12, epochs=10,
        methods=("osem", "svrem", "saga", "svrg"), eta_svrg=5, eta_svrem=3, potential="logcosh", delta=1.0),
}


@dataclass(frozen=True)
class Ellipse:
    cx: float
    cy: float
    a: float          # semi-axis along the rotated x' axis (mm)
    b: float          # semi-axis along the rotated y' axis (mm)
    phi: float        # rotation of x' from x (rad)
    value: float      # activity added inside the ellipse


def _contains(e: Ellipse, x, y):
    c, s = math.cos(e.phi), math.sin(e.phi)
    xr = (x - e.cx) * c + (y - e.cy) * s
    yr = -(x - e.cx) * s + (y - e.cy) * c
    return (xr / e.a) ** 2 + (yr / e.b) ** 2 <= 1.0


def _value_at(ellipses, x, y) -> float:
    return float(sum(e.value for e in ellipses if _contains(e, x, y)))


def random_ellipse_phantom(geom: Geometry, seed: int, n_ellipses: int,
                           n_lesions: int = 0) -> list:
    """Body ellipse of activity 1 plus ``n_ellipses`` inner ellipses whose added
    activity is U[0.5, 4], plus ``n_lesions`` hot disks of radius 3-6 pixels
    at 4x the local activity (the lesion adds 3x the value at its centre)."""
    rng = np.random.default_rng(seed)
    half = 0.5 * min(geom.nx, geom.ny) * geom.pixel_mm
    body = Ellipse(rng.uniform(-0.03, 0.03) * half, rng.uniform(-0.03, 0.03) * half,
                   half * rng.uniform(0.80, 0.88), half * rng.uniform(0.62, 0.72),
                   rng.uniform(-0.2, 0.2), 1.0)
    out = [body]
    for _ in range(n_ellipses):
        for _try in range(100):
            r = math.sqrt(rng.uniform(0.0, 1.0)) * 0.7
            ang = rng.uniform(0.0, 2.0 * math.pi)
            cx = body.cx + r * body.a * math.cos(ang)
            cy = body.cy + r * body.b * math.sin(ang)
            a = half * rng.uniform(0.04, 0.22)
            b = half * rng.uniform(0.04, 0.22)
            e = Ellipse(cx, cy, a, b, rng.uniform(0.0, math.pi), rng.uniform(0.5, 4.0))
            # keep the inner ellipse inside the body: test its 8 extreme points
            pts = [(cx + a * math.cos(u) * math.cos(e.phi) - b * math.sin(u) * math.sin(e.phi),
                    cy + a * math.cos(u) * math.sin(e.phi) + b * math.sin(u) * math.cos(e.phi))
                   for u in np.linspace(0.0, 2.0 * math.pi, 8, endpoint=False)]
            if all(_contains(body, px, py) for px, py in pts):
                out.append(e)
                break
    for _ in range(n_lesions):
        rad = rng.uniform(3.0, 6.0) * geom.pixel_mm
        r = math.sqrt(rng.uniform(0.0, 1.0)) * 0.6
        ang = rng.uniform(0.0, 2.0 * math.pi)
        cx = body.cx + r * body.a * math.cos(ang)
        cy = body.cy + r * body.b * math.sin(ang)
        local = _value_at(out, cx, cy)
        out.append(Ellipse(cx, cy, rad, rad, 0.0, 3.0 * local))
    return out


def ellipsoid_solids(geom: Geometry, seed: int, n_ellipsoids: int, zhalf: float, body_c: float = 1.05) -> list:
    """Random ellipsoids (cx, cy, cz, a, b, c, phi, value), rotated by phi about
    z: a body of activity 1 with axial semi-axis ``body_c * zhalf`` plus
    ``n_ellipsoids`` inner ones adding U[0.5, 4]."""
    rng = np.random.default_rng(seed)
    half = 0.5 * min(geom.nx, geom.ny) * geom.pixel_mm
    solids = [(0.0, 0.0, 0.0, 0.85 * half, 0.66 * half, body_c * zhalf, 0.0, 1.0)]
    for _ in range(n_ellipsoids):
        r = math.sqrt(rng.uniform(0.0, 1.0)) * 0.55
        ang = rng.uniform(0.0, 2.0 * math.pi)
        solids.append((r * 0.85 * half * math.cos(ang), r * 0.66 * half * math.sin(ang),
                       rng.uniform(-0.5, 0.5) * zhalf, half * rng.uniform(0.05, 0.2),
                       half * rng.uniform(0.05, 0.2), zhalf * rng.uniform(0.2, 0.6),
                       rng.uniform(0.0, math.pi), rng.uniform(0.5, 4.0)))
    return solids


def ellipsoid_stack_phantom(geom: Geometry, seed: int, n_ellipsoids: int) -> list:
    """Per-slice ellipse lists of a random ellipsoid phantom sampled at the
    ``nz`` slice centres (slice thickness = pixel size).  Each slice of an
    ellipsoid with semi-axes (a, b, c) at height dz from its centre is the
    ellipse with semi-axes scaled by sqrt(1 - (dz/c)^2)."""
    solids = ellipsoid_solids(geom, seed, n_ellipsoids, 0.5 * geom.nz * geom.pixel_mm)
    slices = []
    for k in range(geom.nz):
        z = (k - 0.5 * (geom.nz - 1)) * geom.pixel_mm
        cur = []
        for (cx, cy, cz, a, b, c, phi, val) in solids:
            t = 1.0 - ((z - cz) / c) ** 2
            if t > 0.0:
                sc = math.sqrt(t)
                cur.append(Ellipse(cx, cy, a * sc, b * sc, phi, val))
        slices.append(cur)
    return slices


def rasterise(ellipses, geom: Geometry) -> np.ndarray:
    """Sample the phantom at pixel centres, ``[iy][ix]`` float64 (reference image only)."""
    xs = (np.arange(geom.nx) - 0.5 * (geom.nx - 1)) * geom.pixel_mm
    ys = (np.arange(geom.ny) - 0.5 * (geom.ny - 1)) * geom.pixel_mm
    X, Y = np.meshgrid(xs, ys)
    img = np.zeros((geom.ny, geom.nx))
    for e in ellipses:
        c, s = math.cos(e.phi), math.sin(e.phi)
        xr = (X - e.cx) * c + (Y - e.cy) * s
        yr = -(X - e.cx) * s + (Y - e.cy) * c
        img += e.value * (((xr / e.a) ** 2 + (yr / e.b) ** 2) <= 1.0)
    return img


def analytic_sinogram(ellipses, geom: Geometry) -> np.ndarray:
    """Closed-form line integrals of the continuous ellipse phantom,
    ``[view][bin]`` float64, for the lines ``x cos(th) + y sin(th) = s``.

    For an ellipse with semi-axes (a, b) rotated by phi and centred at c, the
    chord of that line is ``2ab sqrt(q - s'^2) / q`` with
    ``q = a^2 cos^2(th-phi) + b^2 sin^2(th-phi)`` and
    ``s' = s - (cx cos th + cy sin th)`` (zero when ``s'^2 >= q``)."""
    th = np.arange(geom.n_angles) * (math.pi / geom.n_angles)
    s = (np.arange(geom.n_bins) - 0.5 * (geom.n_bins - 1)) * geom.ds
    out = np.zeros((geom.n_angles, geom.n_bins))
    for e in ellipses:
        tp = th - e.phi
        q = (e.a * np.cos(tp)) ** 2 + (e.b * np.sin(tp)) ** 2
        sp = s[None, :] - (e.cx * np.cos(th) + e.cy * np.sin(th))[:, None]
        rad = q[:, None] - sp * sp
        chord = np.where(rad > 0.0, 2.0 * e.a * e.b * np.sqrt(np.maximum(rad, 0.0)) / q[:, None], 0.0)
        out += e.value * chord
    return out


def _ring_positions(geom: Geometry) -> np.ndarray:
    return (np.arange(geom.n_rings) - 0.5 * (geom.n_rings - 1)) * geom.ring_mm


def analytic_lor_sinogram(solids, geom: Geometry) -> np.ndarray:
    """Closed-form line integrals of the continuous ellipsoid phantom along
    the multi-ring lines of response, ``[view][bin][pair]`` float64.

    Line (i, j, r1, r2): p(t) = (s_j cos th_i, s_j sin th_i, zm) + t (-sin th_i,
    cos th_i, kappa), zm = (z_r1 + z_r2)/2, kappa = (z_r2 - z_r1) / (2T),
    T = sqrt(R^2 - s_j^2) (ring r1 at t = -T, ring r2 at t = +T on the
    cylinder of radius R).  For an ellipsoid x'^T D x' <= 1 (x' the point
    relative to the centre, rotated by -phi about z) the chord in t solves
    A t^2 + 2 B t + C = 0; its length is 2 sqrt(B^2 - A C) / A times
    sqrt(1 + kappa^2)."""
    th = np.arange(geom.n_angles) * (math.pi / geom.n_angles)
    s = (np.arange(geom.n_bins) - 0.5 * (geom.n_bins - 1)) * geom.ds
    zr = _ring_positions(geom)
    T = np.sqrt(geom.radius_mm ** 2 - s ** 2)
    out = np.zeros((geom.n_angles, geom.n_bins, geom.n_rings, geom.n_rings))
    c, sn = np.cos(th)[:, None], np.sin(th)[:, None]
    for r1 in range(geom.n_rings):
        for r2 in range(geom.n_rings):
            kappa = ((zr[r2] - zr[r1]) / (2.0 * T))[None, :]
            zm = 0.5 * (zr[r1] + zr[r2])
            stretch = np.sqrt(1.0 + kappa * kappa)
            for (cx, cy, cz, a, b, cc, phi, val) in solids:
                cp, sp = math.cos(phi), math.sin(phi)
                px, py, pz = s[None, :] * c - cx, s[None, :] * sn - cy, zm - cz
                ux, uy = -sn, c
                # rotate into the ellipsoid's frame
                qx, qy = px * cp + py * sp, -px * sp + py * cp
                vx, vy = ux * cp + uy * sp, -ux * sp + uy * cp
                A = (vx / a) ** 2 + (vy / b) ** 2 + (kappa / cc) ** 2
                B = qx * vx / a ** 2 + qy * vy / b ** 2 + pz * kappa / cc ** 2
                C = (qx / a) ** 2 + (qy / b) ** 2 + (pz / cc) ** 2 - 1.0
                disc = B * B - A * C
                chord = np.where(disc > 0.0, 2.0 * np.sqrt(np.maximum(disc, 0.0)) / A, 0.0)
                out[:, :, r1, r2] += val * chord * stretch
    return out.reshape(geom.n_angles, geom.n_bins, geom.n_rings * geom.n_rings)


def rasterise_volume(solids, geom: Geometry) -> np.ndarray:
    """Sample the ellipsoid phantom at voxel centres, ``[iy][ix][iz]`` float64."""
    xs = (np.arange(geom.nx) - 0.5 * (geom.nx - 1)) * geom.pixel_mm
    ys = (np.arange(geom.ny) - 0.5 * (geom.ny - 1)) * geom.pixel_mm
    zs = (np.arange(geom.nz) - 0.5 * (geom.nz - 1)) * geom.slice_mm
    Y, X, Z = np.meshgrid(ys, xs, zs, indexing="ij")
    vol = np.zeros((geom.ny, geom.nx, geom.nz))
    for (cx, cy, cz, a, b, cc, phi, val) in solids:
        cp, sp = math.cos(phi), math.sin(phi)
        xr = (X - cx) * cp + (Y - cy) * sp
        yr = -(X - cx) * sp + (Y - cy) * cp
        vol += val * (((xr / a) ** 2 + (yr / b) ** 2 + ((Z - cz) / cc) ** 2) <= 1.0)
    return vol


def make_data(work: Workload, seed: int):
    """Phantom ``seed`` and Poisson data with noise seed ``seed + 1000``.

    Returns a dict with
      ``g``      float32 counts, ``[view][bin]`` (``[view][bin][z]`` for stacks,
                 ``[view][bin][ring pair]`` for multi-ring scanners);
      ``w``      float background per bin (uniform: ``bg_frac`` x mean trues);
      ``x_true`` float64 scaled reference image ``[iy][ix]`` (``[iy][ix][z]``);
      ``scale``  the activity scale that makes the expected trues sum to ``counts``.
    """
    geom = work.geometry
    if geom.multiring:
        # the body stays inside the axial field of view (no activity the image cannot hold)
        solids = ellipsoid_solids(geom, seed, work.n_ellipses, 0.5 * geom.nz * geom.slice_mm, body_c=0.9)
        sino = analytic_lor_sinogram(solids, geom)
        img = rasterise_volume(solids, geom)
    elif work.stack:
        per_slice = ellipsoid_stack_phantom(geom, seed, work.n_ellipses)
        sino = np.stack([analytic_sinogram(e, geom) for e in per_slice], axis=-1)
        img = np.stack([rasterise(e, geom) for e in per_slice], axis=-1)
    else:
        ell = random_ellipse_phantom(geom, seed, work.n_ellipses, work.n_lesions)
        sino = analytic_sinogram(ell, geom)
        img = rasterise(ell, geom)
    scale = work.counts / float(sino.sum())
    trues = scale * sino
    w = work.bg_frac * float(trues.mean())
    rng = np.random.default_rng(seed + 1000)
    g = rng.poisson(trues + w).astype(np.float32)
    return {"g": g, "w": float(w), "x_true": scale * img, "scale": scale}


_M64 = (1 << 64) - 1


def splitmix64(seed: int, n: int) -> list:
    """First ``n`` outputs of SplitMix64 started from ``seed`` (published
    definition: add the golden gamma 0x9E3779B97F4A7C15, then two xor-shift
    multiply rounds and a final xor-shift)."""
    state = seed & _M64
    out = []
    for _ in range(n):
        state = (state + 0x9E3779B97F4A7C15) & _M64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        out.append(z ^ (z >> 31))
    return out


def subset_sequence(seed: int, n_subsets: int, length: int) -> np.ndarray:
    """i.i.d. uniform subset indices in ``[0, n_subsets)`` (with replacement),
    ``floor(u * n_subsets)`` with ``u`` the top 53 bits of SplitMix64."""
    if n_subsets <= 0 or length < 0:
        raise ValueError("n_subsets must be positive and length nonnegative")
    vals = splitmix64(seed, length)
    return np.array([int(((v >> 11) * n_subsets) >> 53) for v in vals], dtype=np.int32)


def subset_sequences(seeds, n_subsets: int, length: int) -> np.ndarray:
    """``subset_sequence(seed, n_subsets, length)`` for every seed at once, as
    rows of an int32 array: the same SplitMix64 steps in unsigned 64-bit
    array arithmetic (products wrap modulo 2^64 as the definition has them)."""
    if n_subsets <= 0 or length < 0:
        raise ValueError("n_subsets must be positive and length nonnegative")
    seeds = np.asarray(seeds, dtype=np.uint64).reshape(-1, 1)
    steps = np.arange(1, length + 1, dtype=np.uint64).reshape(1, -1)
    with np.errstate(over="ignore"):
        z = seeds + steps * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (((z >> np.uint64(11)) * np.uint64(n_subsets)) >> np.uint64(53)).astype(np.int32)


def serving_workloads(seed: int, count: int, sizes=(128, 256), prefix: str = "serve") -> list:
    """Request templates of the serving stream: image N uniform in ``sizes``,
    views round(1.4 N) (720 for N = 512), bins the odd integer nearest 1.43 N,
    counts log-uniform in [1e6, 1e8], subsets uniform in {6, 12, 21}, method
    SVREM or SAGA.  The method is stored in ``methods[0]``; template i is
    named ``f"{prefix}{i}"``."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(list(sizes)))
        views = 720 if n == 512 else int(round(1.4 * n))
        nb = int(round(1.43 * n))
        if nb % 2 == 0:
            nb += 1 if (1.43 * n) >= nb else -1
        geom = Geometry(n, n, views, nb)
        cnt = float(10.0 ** rng.uniform(6.0, 8.0))
        algo = str(rng.choice(["svrem", "saga"]))
        out.append(Workload(f"{prefix}{i}", geom, n_subsets=int(rng.choice([6, 12, 21])), counts=cnt,
                            bg_frac=0.10, beta=0.005, n_ellipses=12, n_lesions=2, methods=(algo,)))
    return out


def serving_pool() -> list:
    """The request templates the serving stream draws from: eight at 128^2 and
    256^2 (seed 0), two at 384^2 with 538 views x 549 bins (seed 5: SVREM
    with 21 subsets, SAGA with 6) and two at 512^2 with 720 views x 733 bins
    (seed 3: SVREM with 6 subsets, SAGA with 12)."""
    return (serving_workloads(0, 8) + serving_workloads(5, 2, sizes=(384,), prefix="serve384_")
            + serving_workloads(3, 2, sizes=(512,), prefix="serve512_"))


def serving_requests(count: int) -> list:
    """A stream of distinct requests, each with its own phantom and counts:
    request i is ``(workload req<i>, data seed 20000 + i)``, the workload drawn
    as in ``serving_workloads`` (seed 11) with N uniform in {128, 256, 384,
    512} and counts log-uniform in [1e6, 1e8].  Requests of one size and
    subset number share a geometry (and so a plan), nothing else."""
    works = serving_workloads(11, count, sizes=(128, 256, 384, 512), prefix="req")
    return [(w, 20000 + i) for i, w in enumerate(works)]


def batched_workloads(seed: int, count: int) -> list:
    """Uneven batch of reconstruction geometries: N uniform in {64,128,192,256},
    views round(1.4 N), bins the odd integer nearest 1.43 N, counts
    log-uniform in [1e5, 1e7], subsets uniform in {6, 12, 21}."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice([64, 128, 192, 256]))
        nb = int(round(1.43 * n))
        if nb % 2 == 0:
            nb += 1 if (1.43 * n) >= nb else -1
        geom = Geometry(n, n, int(round(1.4 * n)), nb)
        cnt = float(10.0 ** rng.uniform(5.0, 7.0))
        out.append(Workload(f"batch{i}", geom, n_subsets=int(rng.choice([6, 12, 21])),
                            counts=cnt, bg_frac=0.10, beta=0.005, n_ellipses=8,
                            methods=("saga",)))
    return out
