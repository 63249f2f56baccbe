"""Pins for the oracle's likelihood, penalty and algorithms (CPU only).

Each test checks the oracle against something the paper or the mathematics
fixes independently of the oracle's own code: the Poisson pmf, finite
differences, the majorisation property of the surrogate, a 1-D numerical
maximiser, the MM monotonicity of EM, count conservation, the Appendix B closed
form of the SVREM direction, an L-BFGS-B solution of the MAP problem, and
library bfloat16 rounding.
"""
import numpy as np
import pytest
import scipy.optimize
import scipy.stats
import torch

from oracle import em
from oracle.penalty import POTENTIALS, Penalty, drho, gamma, m_step_root, rho
from oracle.subsets import subset_rows, subset_views
from paper_2106_03172_gb300.phantoms import Geometry

from conftest import tiny_problem


@pytest.fixture(scope="module")
def prob_and_data():
    return tiny_problem(Geometry(16, 16, 24, 23), seed=3)


def _rand_image(prob, seed, lo=0.5, hi=3.0):
    return np.random.default_rng(seed).uniform(lo, hi, size=(prob.N, prob.nz))


def test_loglik_is_poisson_log_pmf(prob_and_data):
    """L(f) + sum_m (-log g_m!) equals the Poisson log-likelihood of §2.1,
    Eq. (pdf), with mean A f + w (pins the sign of w, reading C1)."""
    prob, _ = prob_and_data
    f = _rand_image(prob, 1)
    mean = prob.A @ f + prob.w
    ref = scipy.stats.poisson.logpmf(prob.g, mean).sum()
    got = prob.loglik(f).sum() - scipy.special.gammaln(prob.g + 1.0).sum()
    assert got == pytest.approx(ref, rel=1e-12)


def test_grad_L_finite_difference(prob_and_data):
    prob, _ = prob_and_data
    f = _rand_image(prob, 2)
    v = np.random.default_rng(5).standard_normal(f.shape)
    h = 1e-5
    fd = (prob.loglik(f + h * v).sum() - prob.loglik(f - h * v).sum()) / (2 * h)
    assert float((prob.grad_L(f) * v).sum()) == pytest.approx(fd, rel=1e-6)
    for t in range(prob.Ns):
        rows = prob.subsets[t]
        def Lt(x):
            yh = prob.A[rows] @ x + prob.w[rows]
            return float((prob.g[rows] * np.log(yh) - yh).sum())
        fd_t = (Lt(f + h * v) - Lt(f - h * v)) / (2 * h)
        assert float((prob.grad_L_t(f, t) * v).sum()) == pytest.approx(fd_t, rel=1e-6)


@pytest.mark.parametrize("potential", POTENTIALS)
def test_potential_table(potential):
    """Table 1: rho' is the derivative of rho, gamma = rho'/t, rho even and
    convex, gamma nonincreasing on t >= 0 with a finite nonzero limit at 0."""
    delta = 0.7
    t = np.linspace(-5, 5, 2001)
    h = 1e-6
    fd = (rho(t + h, potential, delta) - rho(t - h, potential, delta)) / (2 * h)
    np.testing.assert_allclose(drho(t, potential, delta), fd, atol=1e-6)  # O(h) at the Huber kink
    nz = np.abs(t) > 1e-3
    np.testing.assert_allclose(gamma(t[nz], potential, delta), drho(t[nz], potential, delta) / t[nz], rtol=1e-12)
    np.testing.assert_allclose(rho(t, potential, delta), rho(-t, potential, delta), rtol=1e-14)
    g = gamma(t[t >= 0], potential, delta)
    assert np.all(np.diff(g) <= 1e-15) and 0 < gamma(np.array([0.0]), potential, delta)[0] < np.inf
    assert np.all(np.diff(drho(t, potential, delta)) >= -1e-15)


@pytest.mark.parametrize("potential", POTENTIALS)
def test_penalty_grad_finite_difference(potential):
    pen = Penalty(7, 5, potential, 0.8)
    rng = np.random.default_rng(0)
    f = rng.uniform(0, 3, (35, 2))
    v = rng.standard_normal(f.shape)
    h = 1e-6
    fd = (pen.value(f + h * v).sum() - pen.value(f - h * v).sum()) / (2 * h)
    assert float((pen.grad(f) * v).sum()) == pytest.approx(fd, rel=1e-6)


def test_quadratic_penalty_closed_form():
    """Quadratic R = 1/2 sum_n sum_{j in N4} (f_n - f_j)^2 / 2 = sum over
    unordered neighbour pairs of (f_n - f_j)^2 / 2."""
    rng = np.random.default_rng(1)
    img = rng.uniform(0, 2, (5, 6))
    pairs = ((img[:, 1:] - img[:, :-1]) ** 2).sum() + ((img[1:, :] - img[:-1, :]) ** 2).sum()
    pen = Penalty(6, 5)
    assert pen.value(img.reshape(-1, 1))[0] == pytest.approx(0.5 * pairs, rel=1e-14)


@pytest.mark.parametrize("potential", POTENTIALS)
def test_surrogate_majorises_penalty(potential):
    """§3: R_hat(.; f^k) >= R, with equality and equal gradient at f^k."""
    pen = Penalty(6, 6, potential, 0.5)
    rng = np.random.default_rng(2)
    fk = rng.uniform(0, 3, (36, 1))
    for _ in range(20):
        f = rng.uniform(0, 3, (36, 1))
        assert pen.surrogate_value(f, fk)[0] >= pen.value(f)[0] - 1e-12
    assert pen.surrogate_value(fk, fk)[0] == pytest.approx(pen.value(fk)[0], rel=1e-14)
    v = rng.standard_normal(fk.shape)
    h = 1e-6
    fd = (pen.surrogate_value(fk + h * v, fk)[0] - pen.surrogate_value(fk - h * v, fk)[0]) / (2 * h)
    assert float((pen.grad(fk) * v).sum()) == pytest.approx(fd, rel=1e-6)


@pytest.mark.parametrize("potential", ["quadratic", "huber", "logcosh"])
def test_root_maximises_separable_surrogate(potential):
    """The M-step root maximises, per pixel, a log f - S f - beta sum_j d_nj (f - mu_nj)^2
    (the separable surrogate objective of §3); checked with a bounded 1-D
    numerical maximiser, plus the residual of a/f - 2bf + c = 0."""
    nx = ny = 5
    pen = Penalty(nx, ny, potential, 0.6)
    rng = np.random.default_rng(4)
    fk = rng.uniform(0.1, 3, (nx * ny, 1))
    a = rng.uniform(0.05, 5, fk.shape)
    S = rng.uniform(0.5, 2, fk.shape)
    beta = 0.7
    root = m_step_root(a, fk, S, beta, pen)
    d = gamma(fk[pen.src] - fk[pen.dst], potential, 0.6)[:, 0]
    mu = 0.5 * (fk[pen.src] + fk[pen.dst])[:, 0]
    for n in range(nx * ny):
        sel = pen.src == n
        def negh(x):
            return -(a[n, 0] * np.log(x) - S[n, 0] * x - beta * np.sum(d[sel] * (x - mu[sel]) ** 2))
        res = scipy.optimize.minimize_scalar(negh, bounds=(1e-9, 50.0), method="bounded",
                                             options={"xatol": 1e-12})
        assert root[n, 0] == pytest.approx(res.x, rel=1e-6)
    sd, sdf = pen.surrogate_weights(fk)
    b, c = beta * sd, beta * (fk * sd + sdf) - S
    np.testing.assert_allclose(a / root - 2 * b * root + c, 0.0, atol=1e-12)
    # beta = 0: the plain EM M-step a / S (the printed "-c/a" is a typo for -a/c)
    np.testing.assert_allclose(m_step_root(a, fk, S, 0.0, pen), a / S, rtol=1e-15)
    # nonpositive statistic -> 0 (zero-denominator remedy)
    a2 = a.copy()
    a2[:3] = -1.0
    assert np.all(m_step_root(a2, fk, S, beta, pen)[:3] == 0.0)


def test_subsets_partition():
    views = subset_views(180, 21)
    assert sorted(np.concatenate(views).tolist()) == list(range(180))
    assert [len(v) for v in views].count(9) == 12 and [len(v) for v in views].count(8) == 9
    rows = subset_rows(6, 5, 4)
    assert sorted(np.concatenate(rows).tolist()) == list(range(30))
    with pytest.raises(ValueError):
        subset_views(5, 6)


def test_osem_one_subset_is_mlem():
    """§2.2: OSEM with N_s = 1 is MLEM."""
    geom = Geometry(12, 12, 18, 17)
    p1, _ = tiny_problem(geom, seed=5, n_subsets=1, beta=0.0)
    f = p1.uniform_image()
    for _ in range(3):
        np.testing.assert_allclose(em.osem_step(p1, f, 0), em.mlem_step(p1, f), rtol=1e-13)
        f = em.mlem_step(p1, f)


def test_mlem_likelihood_monotone_and_nonnegative():
    """MM property (§2.2): every MLEM iterate increases L and stays >= 0."""
    geom = Geometry(12, 12, 18, 17)
    p, _ = tiny_problem(geom, seed=6, n_subsets=1, beta=0.0)
    f = p.uniform_image()
    last = p.loglik(f).sum()
    for _ in range(25):
        f = em.mlem_step(p, f)
        cur = p.loglik(f).sum()
        assert cur >= last - 1e-9 * abs(last) and f.min() >= 0.0
        last = cur


def test_map_em_objective_monotone(prob_and_data):
    """MM property with the parabolic surrogate (§3): MAP-EM increases Phi."""
    prob, _ = prob_and_data
    f = prob.uniform_image()
    last = prob.objective(f)
    for _ in range(25):
        f = em.map_em_step(prob, f)
        cur = prob.objective(f)
        assert cur >= last - 1e-10 * abs(last) and f.min() >= 0.0
        last = cur


def test_count_conservation():
    """w = 0, beta = 0: one OSEM step gives sum_n (A_t^T 1)_n f_n = sum g_m over
    the rays of S_t that meet the image (textbook EM count conservation)."""
    geom = Geometry(12, 12, 18, 17)
    p, _ = tiny_problem(geom, seed=7, n_subsets=3, beta=0.0, w_zero=True)
    f = p.uniform_image() + 0.1
    for t in range(p.Ns):
        f1 = em.osem_step(p, f, t)
        hit = np.asarray(p.At[t].sum(axis=1)).ravel() > 0
        assert (~hit).any()
        assert float((p.sens_t[t] * f1).sum()) == pytest.approx(float(p.gt[t][hit].sum()), rel=1e-12)


def test_statistic_identities(prob_and_data):
    """Eq. (subsetstat) and Eq. (tau_t) agree, and s(f) = mean_t tau_t(f) (§2.3)."""
    prob, _ = prob_and_data
    f = _rand_image(prob, 8)
    for t in range(prob.Ns):
        np.testing.assert_allclose(prob.tau_t(f, t), prob.tau_t_from_gradient(f, t), rtol=1e-12, atol=1e-12)
    mean = sum(prob.tau_t(f, t) for t in range(prob.Ns)) / prob.Ns
    np.testing.assert_allclose(mean, prob.statistic(f), rtol=1e-12)


def test_svrem_step_matches_appendix_b():
    """Appendix B: at beta = 0 with s_hat^k = A^T 1 . f^k, one SVREM update
    equals f^k + alpha h with the printed closed-form direction h."""
    geom = Geometry(12, 12, 18, 17)
    p, _ = tiny_problem(geom, seed=9, n_subsets=3, beta=0.0)
    rng = np.random.default_rng(3)
    fk = rng.uniform(0.5, 2.0, (p.N, 1))
    f_anc = rng.uniform(0.5, 2.0, (p.N, 1))
    alg = em.SVREM(p, f_anc, alpha=0.7, eta=1)
    alg.refresh_anchor()
    alg.f, alg.s_hat, alg.k = fk.copy(), p.sens * fk, 1
    for t in range(p.Ns):
        alg.f, alg.s_hat, alg.k = fk.copy(), p.sens * fk, 1
        got = alg.step(t)
        want = fk + 0.7 * em.svrem_direction_appendix_b(p, fk, f_anc, t)
        np.testing.assert_allclose(got, np.maximum(want, 0.0), rtol=1e-11, atol=1e-12)


def test_svrg_anchor_step_is_full_gradient_step(prob_and_data):
    """§4: at an anchor iteration the SVRG direction is grad Phi(f)/N_s."""
    prob, _ = prob_and_data
    f0 = _rand_image(prob, 10)
    alg = em.SVRG(prob, f0, alpha=1.5, eta=2)
    f1 = alg.step(2)
    want = np.maximum(f0 + 1.5 * alg.d * prob.grad_Phi(f0) / prob.Ns, 0.0)
    np.testing.assert_allclose(f1, want, rtol=1e-12, atol=1e-14)


def test_svrem_single_subset_alpha_one_is_map_em():
    geom = Geometry(12, 12, 18, 17)
    p, _ = tiny_problem(geom, seed=11, n_subsets=1, beta=0.05)
    f = p.uniform_image()
    alg = em.SVREM(p, f, alpha=1.0, eta=1)
    for _ in range(4):
        want = em.map_em_step(p, f)
        f = alg.step(0)
        np.testing.assert_allclose(f, want, rtol=1e-12)


@pytest.fixture(scope="module")
def map_solution(prob_and_data):
    """f* of max_{f>=0} Phi by L-BFGS-B (the paper's reference solver, §5.1)."""
    prob, _ = prob_and_data
    x0 = prob.initial_image().ravel()
    res = scipy.optimize.minimize(
        lambda x: -prob.objective(x.reshape(-1, 1)),
        x0, jac=lambda x: -prob.grad_Phi(x.reshape(-1, 1)).ravel(),
        method="L-BFGS-B", bounds=[(0, None)] * x0.size,
        options={"maxiter": 20000, "ftol": 1e-16, "gtol": 1e-11, "maxcor": 30})
    return res.x.reshape(-1, 1)


def test_map_em_reaches_lbfgsb_maximiser(prob_and_data, map_solution):
    """MAP-EM with the parabolic surrogate converges to the L-BFGS-B maximiser."""
    prob, _ = prob_and_data
    f, hist = em.map_em(prob, prob.initial_image(), max_iter=4000, tol=1e-15)
    assert prob.objective(f) == pytest.approx(prob.objective(map_solution), rel=1e-9)
    assert np.linalg.norm(f - map_solution) / np.linalg.norm(map_solution) < 2e-3
    assert em.kkt_residual(prob, map_solution) < 1e-6


def test_kkt_point_is_fixed_point_of_vr_methods(prob_and_data, map_solution):
    """§4 stationarity: at the maximiser one SAGA step (table built there), one
    SVRG step and one SVREM step leave f* unchanged; plain OSEM does not (the
    limit cycle motivating variance reduction, §1)."""
    prob, _ = prob_and_data
    fs = map_solution
    f0 = prob.initial_image()
    d = em.preconditioner(prob, f0)
    scale = np.linalg.norm(fs)
    for t in range(prob.Ns):
        saga = em.SAGA(prob, fs, alpha=2.0, d=d)
        assert np.linalg.norm(saga.step(t) - fs) / scale < 1e-6
        svrg = em.SVRG(prob, fs, alpha=2.0, eta=2, d=d)
        assert np.linalg.norm(svrg.step(t) - fs) / scale < 1e-6
        for pre in (em.SAGA(prob, fs, alpha=1.0, precond="iterate"),
                    em.SVRG(prob, fs, alpha=1.0, eta=2, precond="iterate")):
            assert np.linalg.norm(pre.step(t) - fs) / scale < 1e-6
        svrem = em.SVREM(prob, fs, alpha=0.7, eta=1)
        assert np.linalg.norm(svrem.step(t) - fs) / scale < 1e-6
    assert np.linalg.norm(em.osem_step(prob, fs, 0) - fs) / scale > 1e-4


def test_bf16_round_matches_torch():
    x = np.random.default_rng(0).standard_normal(10000) * np.logspace(-20, 20, 10000)
    x = np.concatenate([x, [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 65504.0]])
    want = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(em.bf16_round(x), want)


def test_vr_methods_converge_towards_map(prob_and_data, map_solution):
    """SVREM, SAGA and SVRG approach Phi* from the OSEM warm start (§5)."""
    prob, _ = prob_and_data
    phi_star = prob.objective(map_solution)
    f0 = prob.initial_image()
    gap0 = em.relative_gap(prob.objective(f0), phi_star)
    from paper_2106_03172_gb300.phantoms import subset_sequence
    seq = subset_sequence(2000, prob.Ns, 40 * prob.Ns)
    for alg in (em.SVREM(prob, f0, 0.7, 1), em.SAGA(prob, f0, 1.0), em.SVRG(prob, f0, 1.0, 2)):
        for t in seq:
            f = alg.step(int(t))
        gap = em.relative_gap(prob.objective(f), phi_star)
        assert -1e-12 <= gap < 1e-3 * gap0


def test_sga_at_beta_zero_is_osem():
    """§4, Eq. (osem_additive): with beta = 0 and alpha = 1, the preconditioned
    gradient step f + (f / A_t^T 1) grad L_t(f) is the OSEM M-step."""
    geom = Geometry(12, 12, 18, 17)
    p, _ = tiny_problem(geom, seed=13, n_subsets=3, beta=0.0)
    f = p.uniform_image()
    alg = em.SGA(p, f)
    for t in (0, 2, 1, 1):
        want = em.osem_step(p, alg.f, t)
        np.testing.assert_allclose(alg.step(t), want, rtol=1e-12, atol=1e-14)


def test_iterate_preconditioned_vr_single_subset_is_mlem():
    """§4, Eqs. (saga_update), (svrg_update) with d_t(f^k) of Eq.
    (preconditioners): with one subset, beta = 0 and alpha = 1 the table
    correction (SAGA) and the anchor correction (SVRG) cancel, and the step is
    f + (f / A^T 1) grad L(f), which is MLEM (§2.2).  The constant
    preconditioner d(f^(0)) gives a different step."""
    geom = Geometry(12, 12, 18, 17)
    p1, _ = tiny_problem(geom, seed=21, n_subsets=1, beta=0.0)
    f = p1.uniform_image()
    saga = em.SAGA(p1, f, alpha=1.0, precond="iterate")
    svrg = em.SVRG(p1, f, alpha=1.0, eta=1, precond="iterate")
    for _ in range(4):
        want = em.mlem_step(p1, f)
        np.testing.assert_allclose(saga.step(0), want, rtol=1e-11, atol=1e-13)
        np.testing.assert_allclose(svrg.step(0), want, rtol=1e-11, atol=1e-13)
        f = want
    const = em.SAGA(p1, p1.uniform_image(), alpha=1.0)
    const.step(0)
    const.step(0)
    assert np.abs(const.step(0) - saga.f).max() > 1e-6 * np.abs(saga.f).max()


def test_sem_full_step_single_subset_is_map_em():
    """SEM with alpha_k = 1 and one subset replaces s_hat by s(f): MAP-EM."""
    geom = Geometry(12, 12, 18, 17)
    p, _ = tiny_problem(geom, seed=14, n_subsets=1, beta=0.05)
    f = p.uniform_image()
    alg = em.SEM(p, f, schedule=lambda k: 1.0)
    for _ in range(3):
        want = em.map_em_step(p, alg.f)
        np.testing.assert_allclose(alg.step(0), want, rtol=1e-12)


def test_bsrem_schedule_and_monotone_decay():
    assert em.bsrem_schedule(0) == 1.0
    assert em.bsrem_schedule(1000) == pytest.approx(0.5)


def test_sagaem_single_subset_alpha_one_is_map_em():
    """SAGA-EM with one subset and alpha = 1 replaces s_hat by s(f^k): MAP-EM."""
    geom = Geometry(12, 12, 18, 17)
    p, _ = tiny_problem(geom, seed=15, n_subsets=1, beta=0.05)
    f = p.uniform_image()
    alg = em.SAGAEM(p, f, alpha=1.0)
    for _ in range(3):
        want = em.map_em_step(p, alg.f)
        np.testing.assert_allclose(alg.step(0), want, rtol=1e-12)


def test_sagaem_statistic_starts_at_full_statistic(prob_and_data):
    prob, _ = prob_and_data
    f = _rand_image(prob, 16)
    alg = em.SAGAEM(prob, f, alpha=0.5)
    np.testing.assert_allclose(alg.s_hat, prob.statistic(f), rtol=1e-12)


# ---- unbiasedness of the stochastic directions (§2.3, §4) -------------------
#
# The variance-reduced estimators are unbiased: averaged over a uniformly drawn
# subset t, the SAGA and SVRG directions equal grad Phi(f) / N_s (§4,
# Eqs. (saga_update) and (svrg_update)) and the SAGA-EM statistic equals the
# full statistic s(f) (§2.3, the remark after Eq. (tempsvrem)), for ANY table
# or anchor, not only at a fixed point.  The identities hold only when the
# table mean is taken before the current entry is overwritten (reading C6), so
# they pin the table bookkeeping of the oracle.  grad Phi and s(f) themselves
# are pinned by finite differences and the Poisson pmf above.

def _unclipped_steps(alg, prob, f, t_list, make_state):
    """Run one step of `alg` from the same state for every t and return the
    direction of each step: the update is f + alpha d . dir with d = eps f,
    alpha = 1 and eps small enough that P_{>=0} never clips, so that
    dir = (f' - f) / (eps f) exactly up to rounding."""
    dirs = []
    for t in t_list:
        make_state(alg)
        f_new = alg.step(t)
        dirs.append((f_new - f) / alg.d)
    return dirs


@pytest.mark.parametrize("table", ["fp32", "bf16"])
def test_saga_direction_is_unbiased_for_any_table(prob_and_data, table):
    """mean_t (q_new,t - q_t + mean_t' q_t') = mean_t q_new,t = grad Phi(f) / N_s
    (FP32 table), with a random table far from f; the post-write mean would
    add (mean_t q_new,t - mean q) / N_s."""
    prob, _ = prob_and_data
    rng = np.random.default_rng(31)
    f = _rand_image(prob, 30)
    grads = [prob.grad_Phi_t(f, t) for t in range(prob.Ns)]
    scale = max(np.abs(g).max() for g in grads)
    table0 = [rng.standard_normal(f.shape) * scale for _ in range(prob.Ns)]
    rnd = em.bf16_round if table == "bf16" else (lambda x: x)
    eps = 1e-3 / (5.0 * scale)
    alg = em.SAGA(prob, f, alpha=1.0, d=eps * f, table=table)

    def reset(a):
        a.f = f.copy()
        a.q = [rnd(q) for q in table0]

    dirs = _unclipped_steps(alg, prob, f, range(prob.Ns), reset)
    mean_dir = sum(dirs) / prob.Ns
    want = sum(rnd(g) for g in grads) / prob.Ns          # = grad Phi(f) / N_s for the FP32 table
    np.testing.assert_allclose(mean_dir, want, rtol=0, atol=1e-9 * scale)
    if table == "fp32":
        np.testing.assert_allclose(mean_dir, prob.grad_Phi(f) / prob.Ns, rtol=0, atol=1e-9 * scale)
    # the table is far from f, so the pre- and post-write means differ by far more than the tolerance
    assert np.abs(sum(grads) / prob.Ns - sum(table0) / prob.Ns).max() > 1e3 * 1e-9 * scale * prob.Ns


def test_svrg_direction_is_unbiased_for_any_anchor(prob_and_data):
    """mean_t (grad Phi_t(f) - grad Phi_t(f_anc) + grad Phi(f_anc) / N_s) = grad Phi(f) / N_s
    with the anchor away from f (§4, Eq. (svrg_update))."""
    prob, _ = prob_and_data
    f = _rand_image(prob, 32)
    f_anc = _rand_image(prob, 33)
    scale = max(np.abs(prob.grad_Phi_t(x, t)).max() for x in (f, f_anc) for t in range(prob.Ns))
    eps = 1e-3 / (5.0 * scale)
    alg = em.SVRG(prob, f_anc, alpha=1.0, eta=3, d=eps * f)
    alg.refresh_anchor()

    def reset(a):
        a.f, a.k = f.copy(), 1                             # inside the epoch: no anchor refresh

    dirs = _unclipped_steps(alg, prob, f, range(prob.Ns), reset)
    np.testing.assert_allclose(sum(dirs) / prob.Ns, prob.grad_Phi(f) / prob.Ns, rtol=0, atol=1e-9 * scale)
    # each single direction is not the full gradient (the anchor correction is live)
    assert max(np.abs(d - prob.grad_Phi(f) / prob.Ns).max() for d in dirs) > 1e-3 * scale


def test_sagaem_statistic_is_unbiased_for_any_table():
    """With alpha = 1 the SAGA-EM statistic is tau_t(f) - T_t + mean T; its mean
    over t is mean_t tau_t(f) = s(f) = f . A^T(g / (A f + w)) for any table T
    (§2.3), N_s = 4 and a table not built at f."""
    geom = Geometry(12, 12, 18, 17)
    p, _ = tiny_problem(geom, seed=34, n_subsets=4, beta=0.05)
    rng = np.random.default_rng(35)
    f = rng.uniform(0.5, 3.0, (p.N, 1))
    s_full = f * (p.A.T @ (p.g / (p.A @ f + p.w)))       # the statistic from its definition
    table0 = [rng.uniform(0.0, 2.0, f.shape) * s_full.max() for _ in range(p.Ns)]
    alg = em.SAGAEM(p, f, alpha=1.0)
    stats = []
    for t in range(p.Ns):
        alg.f, alg.T = f.copy(), [x.copy() for x in table0]
        alg.step(t)
        stats.append(alg.s_hat.copy())
    np.testing.assert_allclose(sum(stats) / p.Ns, s_full, rtol=1e-12, atol=1e-12 * s_full.max())
    assert np.abs(sum(table0) / p.Ns - s_full).max() > 1e-2 * s_full.max()


def test_saga_three_steps_by_hand():
    """Three SAGA steps (N_s = 3, subsets 1, 1, 2) written out from §4,
    Eq. (saga_update) with the table mean taken before each write (C6):
      f1 = P(f0 + a d (g1(f0) - g1(f0) + (g0(f0) + g1(f0) + g2(f0)) / 3))
      f2 = P(f1 + a d (g1(f1) - g1(f0) + (g0(f0) + g1(f0) + g2(f0)) / 3))
      f3 = P(f2 + a d (g2(f2) - g2(f0) + (g0(f0) + g1(f1) + g2(f0)) / 3))
    with g_t = grad Phi_t and d = d(f0).  The post-write mean would change
    the second and third steps."""
    geom = Geometry(12, 12, 18, 17)
    p, _ = tiny_problem(geom, seed=36, n_subsets=3, beta=0.05)
    f0 = p.initial_image()
    a = 0.8
    d = em.preconditioner(p, f0)
    g = p.grad_Phi_t
    P = lambda x: np.maximum(x, 0.0)
    f1 = P(f0 + a * d * (g(f0, 0) + g(f0, 1) + g(f0, 2)) / 3)
    f2 = P(f1 + a * d * (g(f1, 1) - g(f0, 1) + (g(f0, 0) + g(f0, 1) + g(f0, 2)) / 3))
    f3 = P(f2 + a * d * (g(f2, 2) - g(f0, 2) + (g(f0, 0) + g(f1, 1) + g(f0, 2)) / 3))
    alg = em.SAGA(p, f0, alpha=a)
    for t, want in zip((1, 1, 2), (f1, f2, f3)):
        np.testing.assert_allclose(alg.step(t), want, rtol=1e-12, atol=1e-14 * np.abs(want).max())
    # the readings differ here: the post-write mean moves f2 by a d (g1(f1) - g1(f0)) / 3
    assert np.abs(a * d * (g(f1, 1) - g(f0, 1)) / 3).max() > 1e-6 * np.abs(f2).max()


def test_sagaem_three_steps_by_hand():
    """Three SAGA-EM steps (N_s = 3, subsets 0, 2, 0, alpha = 0.6) written out
    from §2.3 (the remark after Eq. (tempsvrem)) with the M-step of §3:
      s1 = (1-a) s0 + a (tau0(f0) - tau0(f0) + Tbar0),           Tbar0 = mean_t tau_t(f0)
      s2 = (1-a) s1 + a (tau2(f1) - tau2(f0) + Tbar0)
      s3 = (1-a) s2 + a (tau0(f2) - tau0(f0) + (tau0(f0) + tau1(f0) + tau2(f1)) / 3)
    where f_{k+1} is the M-step root with s_{k+1}, s0 = Tbar0 = s(f0)."""
    from oracle.penalty import m_step_root as root
    geom = Geometry(12, 12, 18, 17)
    p, _ = tiny_problem(geom, seed=37, n_subsets=3, beta=0.05)
    f0 = p.initial_image()
    a = 0.6
    tau = p.tau_t
    M = lambda s, fk: root(s, fk, p.sens, p.beta, p.pen)
    Tbar0 = (tau(f0, 0) + tau(f0, 1) + tau(f0, 2)) / 3
    s1 = (1 - a) * Tbar0 + a * Tbar0
    f1 = M(s1, f0)
    s2 = (1 - a) * s1 + a * (tau(f1, 2) - tau(f0, 2) + Tbar0)
    f2 = M(s2, f1)
    s3 = (1 - a) * s2 + a * (tau(f2, 0) - tau(f0, 0) + (tau(f0, 0) + tau(f0, 1) + tau(f1, 2)) / 3)
    f3 = M(s3, f2)
    alg = em.SAGAEM(p, f0, alpha=a)
    for t, want in zip((0, 2, 0), (f1, f2, f3)):
        np.testing.assert_allclose(alg.step(t), want, rtol=1e-11, atol=1e-13 * np.abs(want).max())


def test_svrg_three_steps_by_hand():
    """Three SVRG steps (N_s = 3, eta = 1, subsets 2, 0, 2) from §4,
    Eq. (svrg_update): the anchor is f0 for the whole epoch,
      f_{k+1} = P(f_k + a d (g_t(f_k) - g_t(f0) + grad Phi(f0) / 3))."""
    geom = Geometry(12, 12, 18, 17)
    p, _ = tiny_problem(geom, seed=38, n_subsets=3, beta=0.05)
    f0 = p.initial_image()
    a = 1.3
    d = em.preconditioner(p, f0)
    g = p.grad_Phi_t
    P = lambda x: np.maximum(x, 0.0)
    G0 = p.grad_Phi(f0) / 3
    f1 = P(f0 + a * d * (g(f0, 2) - g(f0, 2) + G0))
    f2 = P(f1 + a * d * (g(f1, 0) - g(f0, 0) + G0))
    f3 = P(f2 + a * d * (g(f2, 2) - g(f0, 2) + G0))
    alg = em.SVRG(p, f0, alpha=a, eta=1)
    for t, want in zip((2, 0, 2), (f1, f2, f3)):
        np.testing.assert_allclose(alg.step(t), want, rtol=1e-12, atol=1e-14 * np.abs(want).max())
    # the fourth step (k = N_s) takes a new anchor: the direction is grad Phi(f3) / 3
    want = P(f3 + a * d * p.grad_Phi(f3) / 3)
    np.testing.assert_allclose(alg.step(1), want, rtol=1e-12, atol=1e-14 * np.abs(want).max())
