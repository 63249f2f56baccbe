"""Pairwise penalty, its parabolic surrogate and the closed-form M-step (§3).

R(f) = 1/2 sum_n sum_{j in N_n} w_nj rho(f_n - f_j)            (§3, penalty)
with N_n the 4-neighbourhood of pixel n inside the image (out-of-image
neighbours are dropped, slices of a stack are not coupled) and w_nj = 1; a
multi-ring volume uses the 6-neighbourhood (its axial neighbours added, also
with w_nj = 1).

Potentials rho, rho' and the curvature gamma = rho'(t)/t follow Table 1
(quadratic, Huber, log cosh, hyperbola); the hyperbola's printed rho lacks a
factor delta (reading noted at ``rho``).

The parabolic surrogate of rho around f^k (§3, following De Pierro-style
separable surrogates) makes the penalised M-step separable; setting the
derivative (§3, Eq. (svrsurder)) to zero gives, per pixel, a/f - 2 b f + c = 0
with
    a = s_hat_n,
    b = beta * sum_j d_nj,
    c = beta * (f^k_n sum_j d_nj + sum_j d_nj f^k_j) - S_n,
    d_nj = w_nj gamma(f^k_n - f^k_j),
where S_n is the sensitivity sum_m a_mn of the data term.

Readings of the printed root (each is a place where the printed text is
garbled or silent):
  * b > 0: f = (c + sqrt(c^2 + 8ab)) / (4b), as printed;
  * the printed b = 0 case "f = -c/a" is a typo: the linear equation
    a/f + c = 0 gives f = -a/c = a/S;
  * when c <= 0 the equivalent form f = 2a / (sqrt(c^2 + 8ab) - c) is used,
    which is free of cancellation and covers b = 0;
  * S_n = 0 or a <= 0 (the statistic of a variance-reduced update can go
    nonpositive) gives f_n = 0, the paper's zero-denominator remedy (§2.3).
"""
from __future__ import annotations

import numpy as np

POTENTIALS = ("quadratic", "huber", "logcosh", "hyperbola")


def rho(t, potential="quadratic", delta=1.0):
    """Potential rho(t) of Table 1."""
    t = np.asarray(t, dtype=np.float64)
    if potential == "quadratic":
        return 0.5 * t * t
    if potential == "huber":
        a = np.abs(t)
        return np.where(a <= delta, 0.5 * t * t, delta * a - 0.5 * delta * delta)
    if potential == "logcosh":
        # delta^2 log cosh(t/delta), written overflow-free:
        # log cosh(u) = |u| + log1p(exp(-2|u|)) - log 2
        u = np.abs(t / delta)
        return delta * delta * (u + np.log1p(np.exp(-2.0 * u)) - np.log(2.0))
    if potential == "hyperbola":
        # Table 1 prints delta*(sqrt(1+(t/delta)^2) - 1), whose derivative is
        # 1/delta times the printed rho'; the printed rho' and gamma (and the
        # quadratic limit delta -> inf shared by the other rows) fix the
        # factor delta^2 used here.
        return delta * delta * (np.sqrt(1.0 + (t / delta) ** 2) - 1.0)
    raise ValueError(potential)


def drho(t, potential="quadratic", delta=1.0):
    """Derivative rho'(t) of Table 1."""
    t = np.asarray(t, dtype=np.float64)
    if potential == "quadratic":
        return t.copy()
    if potential == "huber":
        return np.clip(t, -delta, delta)
    if potential == "logcosh":
        return delta * np.tanh(t / delta)
    if potential == "hyperbola":
        return t / np.sqrt(1.0 + (t / delta) ** 2)
    raise ValueError(potential)


def gamma(t, potential="quadratic", delta=1.0):
    """Curvature gamma(t) = rho'(t)/t of Table 1, with its finite limit at 0."""
    t = np.asarray(t, dtype=np.float64)
    if potential == "quadratic":
        return np.ones_like(t)
    if potential == "huber":
        a = np.abs(t)
        return np.where(a <= delta, 1.0, delta / np.maximum(a, delta))
    if potential == "logcosh":
        small = np.abs(t) < 1e-8 * delta
        safe = np.where(small, 1.0, t)
        return np.where(small, 1.0, delta * np.tanh(safe / delta) / safe)
    if potential == "hyperbola":
        return 1.0 / np.sqrt(1.0 + (t / delta) ** 2)
    raise ValueError(potential)


def neighbour_pairs(nx: int, ny: int, axial: int = 1):
    """Ordered pairs (n, j), j in the in-image 4-neighbourhood of n; with
    axial > 1 the image is a volume of `axial` layers (index
    (iy nx + ix) axial + iz) and the neighbourhood its in-volume
    6-neighbourhood (the two axial neighbours added, weight 1)."""
    iy, ix, iz = np.meshgrid(np.arange(ny), np.arange(nx), np.arange(axial), indexing="ij")
    n = ((iy * nx + ix) * axial + iz).ravel()
    iy, ix, iz = iy.ravel(), ix.ravel(), iz.ravel()
    steps = [(0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)]
    if axial > 1:
        steps += [(0, 0, -1), (0, 0, 1)]
    src, dst = [], []
    for dy, dx, dz in steps:
        jy, jx, jz = iy + dy, ix + dx, iz + dz
        ok = (jy >= 0) & (jy < ny) & (jx >= 0) & (jx < nx) & (jz >= 0) & (jz < axial)
        src.append(n[ok])
        dst.append(((jy * nx + jx) * axial + jz)[ok])
    return np.concatenate(src), np.concatenate(dst)


class Penalty:
    """R, its gradient and surrogate weights on images of shape (N, nz)
    (nz independent slices), or with axial > 1 on volumes of shape
    (N * axial, 1) coupled along z as well."""

    def __init__(self, nx: int, ny: int, potential="quadratic", delta=1.0, axial: int = 1):
        if potential not in POTENTIALS:
            raise ValueError(potential)
        self.nx, self.ny, self.axial = nx, ny, axial
        self.potential, self.delta = potential, delta
        self.src, self.dst = neighbour_pairs(nx, ny, axial)

    def value(self, f):
        """R(f) per slice, shape (nz,)."""
        diff = f[self.src] - f[self.dst]
        return 0.5 * rho(diff, self.potential, self.delta).sum(axis=0)

    def grad(self, f):
        """dR/df_n = sum_{j in N_n} rho'(f_n - f_j) (both ordered pairs of a
        symmetric neighbourhood contribute, and rho' is odd)."""
        g = np.zeros_like(f)
        np.add.at(g, self.src, drho(f[self.src] - f[self.dst], self.potential, self.delta))
        return g

    def surrogate_weights(self, fk):
        """(sum_j d_nj, sum_j d_nj f^k_j) with d_nj = gamma(f^k_n - f^k_j)."""
        d = gamma(fk[self.src] - fk[self.dst], self.potential, self.delta)
        sd = np.zeros_like(fk)
        sdf = np.zeros_like(fk)
        np.add.at(sd, self.src, d)
        np.add.at(sdf, self.src, d * fk[self.dst])
        return sd, sdf

    def surrogate_value(self, f, fk):
        """Surrogate R_hat(f; f^k) of §3 (up to an f-independent constant):
        1/2 sum_n sum_j d_nj ((f_n - mu)^2 + (f_j - mu)^2), mu = (f^k_n + f^k_j)/2,
        plus the constant that makes R_hat(f^k; f^k) = R(f^k)."""
        fs, fd = f[self.src], f[self.dst]
        ks, kd = fk[self.src], fk[self.dst]
        d = gamma(ks - kd, self.potential, self.delta)
        mu = 0.5 * (ks + kd)
        quad = 0.5 * (d * ((fs - mu) ** 2 + (fd - mu) ** 2)).sum(axis=0)
        quad_k = 0.5 * (d * ((ks - mu) ** 2 + (kd - mu) ** 2)).sum(axis=0)
        return quad - quad_k + self.value(fk)


def m_step_root(a, fk, S, beta, penalty: Penalty):
    """Nonnegative root of a/f - 2 b f + c = 0 per pixel (§3, readings above)."""
    sd, sdf = penalty.surrogate_weights(fk)
    b = beta * sd
    c = beta * (fk * sd + sdf) - S
    live = (S > 0.0) & (a > 0.0)
    disc = np.sqrt(np.where(live, c * c + 8.0 * a * b, 0.0))
    out = np.zeros_like(fk)
    neg = live & (c <= 0.0)
    pos = live & (c > 0.0)
    out[neg] = 2.0 * a[neg] / (disc[neg] - c[neg])
    out[pos] = (c[pos] + disc[pos]) / (4.0 * b[pos])
    return out
