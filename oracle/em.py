"""Likelihood, subset statistics and the stochastic EM family in FP64.

Notation follows the paper: A (M x N) the system matrix, g the counts, w the
background, subsets S_1..S_Ns of the rows, A_t / g_t / w_t their restrictions,
beta the penalty weight, R the penalty (``penalty.py``).

Readings (the places where the printed text is garbled or silent):
  C1  the log-likelihood is L(f) = sum_m g_m log(a_m^T f + w_m) - (a_m^T f + w_m)
      (§2.1, Eq. (log_likelihood) prints the sign of w garbled; log g! dropped).
  C3  every ratio g/(A f) of §2.2/§4 carries the background: g/(A f + w), as
      Eq. (tau_t) does; a zero denominator gives ratio 0 (§2.3 remedy).
  C5  penalised OSEM maximises the subset surrogate with the subset
      sensitivity A_t^T 1 and penalty weight beta/N_s (§2.2, Eq. (Mstep) with
      the penalty of §3 split evenly over subsets as in §4, Phi_t);
      parity unpinned.
  C6  SAGA's direction uses the mean of the table *before* the write of the
      current subset (§4, Eq. (saga_update)).
  C9  SVREM refreshes the anchor before the update at k = 0 mod eta*N_s,
      and starts from s_hat^(0) = s(f^(0)).
  C10 SAGA and SVRG project every iterate with P_{>=0} (§4).
  C12 the warm start is one unpenalised OSEM epoch, cyclic subset order, from
      the constant image f_u = sum_m max(g_m - w_m, 0) / sum_n (A^T 1)_n.
  C13 the constant preconditioner is d = N_s f^(0) / A^T 1 (global, OSEM
      scale; §4 freezes d = d(f^(0))); parity unpinned.
  C17 SVREM/SVRG keep the anchor's subset quantities for all t (computed once
      per anchor), matching the paper's epoch count (§5.1).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .penalty import Penalty, m_step_root


def as_image(x, nz=1):
    """Flat or shaped image -> float64 array (N, nz)."""
    x = np.asarray(x, dtype=np.float64)
    return x.reshape(-1, nz)


def bf16_round(x):
    """Round float64 values to bfloat16 (round to nearest even on the float32
    value, i.e. keep the top 16 bits of the IEEE-754 single), returned as float64."""
    f = np.asarray(x, dtype=np.float32).copy()
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


class Problem:
    """The penalised Poisson problem max_{f>=0} Phi(f) = L(f) - beta R(f) (§3,
    Eq. (PET-MAP)) with its subset split (§2.1, Eq. (subobjective))."""

    def __init__(self, A: sp.csr_matrix, g, w, subsets, beta: float, nx: int, ny: int,
                 nz: int = 1, potential="quadratic", delta=1.0, axial: int = 1):
        self.A = A.tocsr()
        self.M, self.N = A.shape
        self.nz = nz
        self.g = np.asarray(g, dtype=np.float64).reshape(self.M, nz)
        w = np.asarray(w, dtype=np.float64)
        self.w = np.broadcast_to(w.reshape(-1, nz) if w.size > 1 else w, (self.M, nz)).copy()
        self.subsets = [np.asarray(r) for r in subsets]
        self.Ns = len(self.subsets)
        self.beta = float(beta)
        self.pen = Penalty(nx, ny, potential, delta, axial)
        self.At = [self.A[r] for r in self.subsets]
        self.gt = [self.g[r] for r in self.subsets]
        self.wt = [self.w[r] for r in self.subsets]
        ones = np.ones((self.M, 1))
        self.sens = np.asarray(self.A.T @ ones)                       # A^T 1
        self.sens_t = [np.asarray(At.T @ np.ones((At.shape[0], 1))) for At in self.At]

    # ---- data term -------------------------------------------------------
    def yhat(self, f, t=None):
        """Expected counts A f + w (§2.1, Eq. (voxel_td)), all rows or subset t."""
        if t is None:
            return self.A @ f + self.w
        return self.At[t] @ f + self.wt[t]

    @staticmethod
    def _ratio(g, yh):
        out = np.zeros_like(yh)
        nz = yh != 0.0
        out[nz] = g[nz] / yh[nz]
        return out

    def loglik(self, f):
        """L(f) = sum_m g_m log yhat_m - yhat_m (reading C1), per slice (nz,)."""
        yh = self.yhat(f)
        glog = np.where(self.g > 0.0, self.g * np.log(np.where(yh > 0, yh, 1.0)), 0.0)
        return (glog - yh).sum(axis=0)

    def objective(self, f):
        """Phi(f) = L(f) - beta R(f) (§3, Eq. (PET-MAP)), summed over slices."""
        return float((self.loglik(f) - self.beta * self.pen.value(f)).sum())

    def backproj_ratio(self, f, t=None):
        """e^t(f) = A_t^T (g_t / (A_t f + w_t)) (§2.2, Eq. (EMsurrogate), reading C3)."""
        if t is None:
            return self.A.T @ self._ratio(self.g, self.yhat(f))
        return self.At[t].T @ self._ratio(self.gt[t], self.yhat(f, t))

    def grad_L_t(self, f, t):
        """grad L_t(f) = A_t^T (g_t / (A_t f + w_t) - 1) (§4, Eq. (osem_additive))."""
        return self.backproj_ratio(f, t) - self.sens_t[t]

    def grad_L(self, f):
        return self.backproj_ratio(f) - self.sens

    def grad_Phi_t(self, f, t):
        """grad Phi_t = grad L_t - (beta/N_s) grad R (§4, Phi_t)."""
        return self.grad_L_t(f, t) - (self.beta / self.Ns) * self.pen.grad(f)

    def grad_Phi(self, f):
        return self.grad_L(f) - self.beta * self.pen.grad(f)

    def tau_t(self, f, t):
        """Subset statistic tau_t(f) = N_s f . A_t^T(g_t / (A_t f + w_t)) (§2.3, Eq. (tau_t))."""
        return self.Ns * f * self.backproj_ratio(f, t)

    def tau_t_from_gradient(self, f, t):
        """The same statistic written as N_s f . (grad L_t + A_t^T 1) (§2.3, Eq. (subsetstat))."""
        return self.Ns * f * (self.grad_L_t(f, t) + self.sens_t[t])

    def statistic(self, f):
        """Full expected statistic s(f) = f . A^T(g / (A f + w)) = mean_t tau_t(f)."""
        return f * self.backproj_ratio(f)

    # ---- warm start --------------------------------------------------------
    def uniform_image(self):
        """f_u = sum_m max(g_m - w_m, 0) / sum_n (A^T 1)_n, per slice (reading C12)."""
        tot = np.maximum(self.g - self.w, 0.0).sum(axis=0)
        return np.ones((self.N, self.nz)) * (tot / self.sens.sum())

    def initial_image(self):
        """f^(0): one unpenalised OSEM epoch in cyclic order from f_u (reading C12)."""
        f = self.uniform_image()
        for t in range(self.Ns):
            f = osem_step(self, f, t, beta=0.0)
        return f


# ---- EM family (§2.2, §2.3, §3) -------------------------------------------

def mlem_step(prob: Problem, f):
    """Unpenalised MLEM, f_n e_n(f) / sum_m a_mn (§2.2, the N_s = 1 update)."""
    live = np.broadcast_to(prob.sens > 0, f.shape)
    return np.divide(f * prob.backproj_ratio(f), prob.sens, out=np.zeros_like(f), where=live)


def osem_step(prob: Problem, f, t, beta=None):
    """Penalised OSEM on subset t: the M-step (§2.2, Eq. (Mstep)) of the
    surrogate with statistic a = f . e^t(f), sensitivity A_t^T 1 and penalty
    weight beta/N_s solved in closed form (§3; reading C5).  At beta = 0 this is
    exactly f e^t / A_t^T 1."""
    b = prob.beta if beta is None else beta
    a = f * prob.backproj_ratio(f, t)
    return m_step_root(a, f, prob.sens_t[t], b / prob.Ns, prob.pen)


def osem_epoch(prob: Problem, f, seq):
    for t in seq:
        f = osem_step(prob, f, int(t))
    return f


def map_em_step(prob: Problem, f):
    """Full-batch penalised EM: M-step with the full statistic s(f), full
    sensitivity and weight beta (§3, Eq. (vrsemreg) with s_hat = s(f^k))."""
    return m_step_root(prob.statistic(f), f, prob.sens, prob.beta, prob.pen)


def map_em(prob: Problem, f, max_iter=100000, tol=1e-10):
    """Run MAP-EM until the relative change of Phi per iteration is <= tol.
    Returns (f, Phi history)."""
    hist = [prob.objective(f)]
    for _ in range(max_iter):
        f = map_em_step(prob, f)
        hist.append(prob.objective(f))
        if abs(hist[-1] - hist[-2]) <= tol * abs(hist[-1]):
            break
    return f, hist


def map_reference(prob: Problem, f0=None, maxiter=20000):
    """Maximiser f* and Phi* of max_{f>=0} Phi by bounded L-BFGS-B, the kind of
    reference solver the paper uses for its error curves (§5.1).  Returns
    (f*, Phi*, KKT residual)."""
    import scipy.optimize
    x0 = (prob.initial_image() if f0 is None else f0).ravel()
    shape = (prob.N, prob.nz)
    res = scipy.optimize.minimize(
        lambda x: -prob.objective(x.reshape(shape)), x0,
        jac=lambda x: -prob.grad_Phi(x.reshape(shape)).ravel(), method="L-BFGS-B",
        bounds=[(0.0, None)] * x0.size,
        options={"maxiter": maxiter, "ftol": 1e-16, "gtol": 1e-10, "maxcor": 30})
    fs = res.x.reshape(shape)
    return fs, prob.objective(fs), kkt_residual(prob, fs)


def kkt_residual(prob: Problem, f):
    """|| f - P_{>=0}(f + D grad Phi(f)) || / ||f|| with the EM scaling
    D = f / A^T 1: zero exactly at a KKT point of max_{f>=0} Phi."""
    D = np.where(prob.sens > 0, f / np.where(prob.sens > 0, prob.sens, 1.0), 0.0)
    step = np.maximum(f + D * prob.grad_Phi(f), 0.0) - f
    return float(np.linalg.norm(step) / np.linalg.norm(f))


def bsrem_schedule(k):
    """Decaying step (0.001 k + 1)^{-1} used for SEM and BSREM in §5.1."""
    return 1.0 / (0.001 * k + 1.0)


class SGA:
    """Preconditioned stochastic gradient ascent (§4, Eq. (sga)) with the
    subset preconditioner d_t(f) = f / A_t^T 1 (§4, Eq. (preconditioners)) and
    the projection P_{>=0}:
        f^{k+1} = P_{>=0}(f^k + alpha_k d_t(f^k) . (grad L_t(f^k) - (beta/N_s) grad R(f^k))).
    alpha_k = 1 is SGA; alpha_k = (0.001 k + 1)^{-1} is the subset-dependent
    BSREM variant of §5.1."""

    def __init__(self, prob: Problem, f0, schedule=lambda k: 1.0):
        self.p, self.f, self.k, self.alpha = prob, f0.copy(), 0, schedule

    def step(self, t):
        S = self.p.sens_t[t]
        d = np.where(S > 0, self.f / np.where(S > 0, S, 1.0), 0.0)
        self.f = np.maximum(self.f + self.alpha(self.k) * d * self.p.grad_Phi_t(self.f, t), 0.0)
        self.k += 1
        return self.f


class SEM:
    """Stochastic EM (§2.3, Eq. (tempsem)): s_hat <- (1-alpha_k) s_hat + alpha_k tau_t(f)."""

    def __init__(self, prob: Problem, f0, schedule=lambda k: 1.0 / (0.001 * k + 1.0)):
        self.p, self.f, self.k, self.alpha = prob, f0.copy(), 0, schedule
        self.s_hat = prob.statistic(self.f)

    def step(self, t):
        a = self.alpha(self.k)
        self.s_hat = (1.0 - a) * self.s_hat + a * self.p.tau_t(self.f, t)
        self.f = m_step_root(self.s_hat, self.f, self.p.sens, self.p.beta, self.p.pen)
        self.k += 1
        return self.f


class SVREM:
    """Stochastic variance reduced EM (§2.3, Eq. (tempsvrem); penalised M-step §3):

        if k mod eta*N_s == 0:  f_anc = f^k,  s_anc = s(f_anc)   (before the update, C9)
        s_hat <- (1-alpha) s_hat + alpha (tau_t(f^k) - tau_t(f_anc) + s_anc)
        f^{k+1} = argmax_f  zeta(f)^T s_hat - U(f) - beta R_hat(f; f^k)
    """

    def __init__(self, prob: Problem, f0, alpha: float, eta: int):
        self.p, self.f, self.alpha, self.eta, self.k = prob, f0.copy(), alpha, eta, 0
        self.s_hat = None

    def refresh_anchor(self):
        self.f_anc = self.f.copy()
        self.tau_anc = [self.p.tau_t(self.f_anc, t) for t in range(self.p.Ns)]
        self.s_anc = self.p.statistic(self.f_anc)
        if self.s_hat is None:
            self.s_hat = self.s_anc.copy()

    def step(self, t):
        if self.k % (self.eta * self.p.Ns) == 0:
            self.refresh_anchor()
        a = self.alpha
        self.s_hat = (1.0 - a) * self.s_hat + a * (
            self.p.tau_t(self.f, t) - self.tau_anc[t] + self.s_anc)
        self.f = m_step_root(self.s_hat, self.f, self.p.sens, self.p.beta, self.p.pen)
        self.k += 1
        return self.f


class SAGAEM:
    """SAGA applied to the EM statistic (§2.3, the remark after
    Eq. (tempsvrem)), with the surrogate M-step of §3:
        s_hat <- (1-alpha) s_hat + alpha (tau_t(f^k) - T_t + (1/N_s) sum_t' T_t')
        f^{k+1} = argmax zeta(f)^T s_hat - U(f) - beta R_hat(f; f^k);  T_t <- tau_t(f^k)
    The table starts at T_t = tau_t(f^(0)) and s_hat at their mean s(f^(0)).
    Reading: the remark refreshes the entry of an independently drawn index;
    here the refreshed entry is the subset just used (as SAGA of §4 does),
    so an update costs one subset pass."""

    def __init__(self, prob: Problem, f0, alpha: float):
        self.p, self.f, self.alpha = prob, f0.copy(), alpha
        self.T = [prob.tau_t(self.f, t) for t in range(prob.Ns)]
        self.s_hat = sum(self.T) / prob.Ns

    def step(self, t):
        tau = self.p.tau_t(self.f, t)
        mean_old = sum(self.T) / self.p.Ns
        self.s_hat = (1.0 - self.alpha) * self.s_hat + self.alpha * (tau - self.T[t] + mean_old)
        self.f = m_step_root(self.s_hat, self.f, self.p.sens, self.p.beta, self.p.pen)
        self.T[t] = tau
        return self.f


def preconditioner(prob: Problem, f0):
    """Constant d = N_s f^(0) / A^T 1 (0 where A^T 1 = 0) (§4, reading C13)."""
    pos = prob.sens > 0
    return np.where(pos, prob.Ns * f0 / np.where(pos, prob.sens, 1.0), 0.0)


def subset_preconditioner(prob: Problem, f, t):
    """Iteration- and subset-dependent d_t(f) = f / A_t^T 1 (0 where
    A_t^T 1 = 0) (§4, Eq. (preconditioners)), the form Eqs. (saga_update) and
    (svrg_update) print before the constant one is adopted."""
    S = prob.sens_t[t]
    pos = S > 0
    return np.where(pos, f / np.where(pos, S, 1.0), 0.0)


class SAGA:
    """Preconditioned proximal SAGA (§4, Eq. (saga_update), readings C6, C10):

        q_new = grad Phi_t(f^k)
        f^{k+1} = P_{>=0}(f^k + alpha d . (q_new - q_t + (1/N_s) sum_t' q_t'))
        q_t <- q_new
    The table starts at q_t = grad Phi_t(f^(0)) for every t.  With
    ``table="bf16"`` every stored table entry is rounded to bfloat16 (the mean
    is taken over the rounded entries).  ``precond="constant"`` takes
    d = d(f^(0)) (reading C13); ``precond="iterate"`` takes d_t(f^k) of
    Eq. (preconditioners) at every update."""

    def __init__(self, prob: Problem, f0, alpha: float, d=None, table="fp32", precond="constant"):
        if precond not in ("constant", "iterate"):
            raise ValueError(precond)
        self.p, self.f, self.alpha, self.precond = prob, f0.copy(), alpha, precond
        self.d = preconditioner(prob, f0) if d is None else d
        self.rnd = bf16_round if table == "bf16" else (lambda x: x)
        self.q = [self.rnd(prob.grad_Phi_t(self.f, t)) for t in range(prob.Ns)]

    def step(self, t):
        q_new = self.rnd(self.p.grad_Phi_t(self.f, t))
        mean_old = sum(self.q) / self.p.Ns
        d = self.d if self.precond == "constant" else subset_preconditioner(self.p, self.f, t)
        self.f = np.maximum(self.f + self.alpha * d * (q_new - self.q[t] + mean_old), 0.0)
        self.q[t] = q_new
        return self.f


class SVRG:
    """Preconditioned proximal SVRG (§4, Eq. (svrg_update), reading C10):

        if k mod eta*N_s == 0:  f_anc = f^k,  q_tilde = grad Phi(f_anc) / N_s
        f^{k+1} = P_{>=0}(f^k + alpha d . (grad Phi_t(f^k) - grad Phi_t(f_anc) + q_tilde))
    ``precond`` as for SAGA: d(f^(0)) or d_t(f^k) at every update."""

    def __init__(self, prob: Problem, f0, alpha: float, eta: int, d=None, precond="constant"):
        if precond not in ("constant", "iterate"):
            raise ValueError(precond)
        self.p, self.f, self.alpha, self.eta, self.k = prob, f0.copy(), alpha, eta, 0
        self.precond = precond
        self.d = preconditioner(prob, f0) if d is None else d

    def refresh_anchor(self):
        self.f_anc = self.f.copy()
        self.g_anc = [self.p.grad_Phi_t(self.f_anc, t) for t in range(self.p.Ns)]
        self.q_tilde = self.p.grad_Phi(self.f_anc) / self.p.Ns

    def step(self, t):
        if self.k % (self.eta * self.p.Ns) == 0:
            self.refresh_anchor()
        direction = self.p.grad_Phi_t(self.f, t) - self.g_anc[t] + self.q_tilde
        d = self.d if self.precond == "constant" else subset_preconditioner(self.p, self.f, t)
        self.f = np.maximum(self.f + self.alpha * d * direction, 0.0)
        self.k += 1
        return self.f


def svrem_direction_appendix_b(prob: Problem, f, f_anc, t):
    """Closed-form SVREM search direction at beta = 0 (Appendix B): with
    s_hat^k = A^T 1 . f^k and d(f) = f / A^T 1, one SVREM update is
    f^k + alpha h with
      h/N_s = d(f) grad L_t(f) - d(f_anc) grad L_t(f_anc) + d(f_anc) grad L(f_anc)/N_s
              + (f - f_anc) . (A_t^T 1 / A^T 1 - 1/N_s)."""
    sens = prob.sens
    d = f / sens
    da = f_anc / sens
    h = (d * prob.grad_L_t(f, t) - da * prob.grad_L_t(f_anc, t)
         + da * prob.grad_L(f_anc) / prob.Ns
         + (f - f_anc) * (prob.sens_t[t] / sens - 1.0 / prob.Ns))
    return prob.Ns * h


def build_problem(geom, g, w, n_subsets, beta, potential="quadratic", delta=1.0, A=None):
    """Problem for a geometry object with fields nx, ny, nz, n_angles, n_bins,
    pixel_mm and ds (A is built by Siddon unless given).  A multi-ring
    geometry (n_rings > 0) gives one volume problem: A from the 3-D Siddon
    matrix, the image a column of nx ny nz voxels (axial index innermost),
    the sinogram a column in [view][bin][ring pair] order, subsets by view
    (every bin and ring pair of a view) and the 6-neighbourhood penalty."""
    from .subsets import subset_rows
    rows = subset_rows(geom.n_angles, geom.n_bins, n_subsets)
    if getattr(geom, "n_rings", 0) > 0:
        from .siddon3d import system_matrix3d
        if A is None:
            A = system_matrix3d(geom)
        npairs = geom.n_rings ** 2
        rows = [(r[:, None] * npairs + np.arange(npairs)[None, :]).ravel() for r in rows]
        return Problem(A, np.asarray(g).reshape(-1, 1), w, rows, beta, geom.nx, geom.ny, 1,
                       potential, delta, axial=geom.nz)
    from .siddon import system_matrix
    if A is None:
        A = system_matrix(geom)
    return Problem(A, np.asarray(g).reshape(geom.n_rays, geom.nz), w, rows, beta,
                   geom.nx, geom.ny, geom.nz, potential, delta)


def relative_gap(phi, phi_star):
    """Relative objective gap (Phi* - Phi) / |Phi*| (reading C1)."""
    return (phi_star - phi) / abs(phi_star)
