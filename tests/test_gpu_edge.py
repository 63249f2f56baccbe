"""GPU parity on the method's edge cases, against the FP64 oracle.

* a zero expected count (no background, rays that miss the image): the ratio
  g / yhat is 0 there (§2.3 remedy), so the updates stay finite;
* pixels no ray of a subset (or of any subset) reaches: S_n = 0 gives f_n = 0
  in the M-step (§2.3 remedy; §3, Eq. (svrsurder)), and the preconditioner is
  0 there (§4);
* a variance-reduced statistic s_hat_n <= 0 (SVREM with a large step, §2.3,
  Eq. (tempsvrem)): the M-step root is then f_n = 0 (reading C7);
* projections P_{>=0} that clip (SAGA and SVRG with a large step, §4);
* the numeric latch: a nonpositive mean with positive data makes the
  objective -inf and is reported as PET_ERR_NUMERIC by the next synchronising
  call, after which the problem is usable again.

Where the oracle's value is exactly zero through one of these branches (and
is not a borderline decision within rounding), the GPU value must be exactly
zero too.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from cases import oracle_problem, rel_l2
from oracle import em
from paper_2106_03172_gb300.phantoms import Geometry, Workload, subset_sequence

pytestmark = pytest.mark.gpu

# every FP32 iterate within 1e-5 relative L2 of the oracle's (the per-iterate
# tolerance of the parity tests)
ITERATE_RTOL = 1e-5


def _pv():
    from paper_2106_03172_gb300 import petvr
    petvr.lib()
    return petvr


def _cuda(x):
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def _setup(name):
    pv = _pv()
    prob, data, work = oracle_problem(name)
    plan = pv.Plan(work.geometry, work.n_subsets)
    gp = pv.Problem(plan, _cuda(data["g"]), None, data["w"], work.beta)
    f0 = prob.initial_image().astype(np.float32).astype(np.float64)
    return pv, prob, data, work, plan, gp, f0


@pytest.mark.parametrize("method", ["osem", "svrem", "saga", "svrg"])
def test_zero_expected_counts(method, record_error):
    """w = 0 and rays that miss the image: yhat = 0 on 19% of the rays."""
    pv, prob, data, work, plan, gp, f0 = _setup("nobg")
    assert data["w"] == 0.0
    yhat0 = prob.A @ f0
    assert (yhat0 == 0).sum() > 100 and np.all(prob.g[yhat0[:, 0] == 0] == 0)
    img = _cuda(f0)
    state = pv.State(gp, method, img)
    alg = {"osem": None, "svrem": em.SVREM(prob, f0, 0.7, 1), "saga": em.SAGA(prob, f0, 1.0),
           "svrg": em.SVRG(prob, f0, 2.0, 2)}[method]
    f, errs = f0, []
    for k, t in enumerate(subset_sequence(6100, work.n_subsets, 2 * work.n_subsets)):
        state.epoch([int(t)], alpha={"svrem": 0.7, "saga": 1.0, "svrg": 2.0}.get(method, 1.0),
                    eta={"svrg": 2}.get(method, 1))
        f = em.osem_step(prob, f, int(t)) if alg is None else alg.step(int(t))
        got = _host(img)
        assert np.all(np.isfinite(got))
        errs.append(rel_l2(got, f))
        assert errs[-1] <= ITERATE_RTOL, f"step {k}: {errs[-1]:.3e}"
    phi_gpu, phi_ora = pv.pet_objective(gp.handle, img), prob.objective(f)
    record_error(test="edge_zero_expected_counts", case="nobg", method=method, table="fp32", epochs=2,
                 one_step=errs[0], trajectory=errs[-1], trajectory_max=max(errs),
                 phi_rel=abs(phi_gpu - phi_ora) / abs(phi_ora))
    assert phi_gpu == pytest.approx(phi_ora, rel=1e-7)


@pytest.mark.parametrize("method", ["osem", "svrem", "saga", "svrg", "sga", "sem"])
def test_unseen_pixels(method, record_error):
    """Pixels with sens_t,n = 0 (or sens_n = 0): the GPU gives exactly 0 where
    the M-step's S_n = 0 branch gives 0, and leaves the pixel unchanged where
    the preconditioner is 0, as the oracle does."""
    pv, prob, data, work, plan, gp, f0 = _setup("sparse")
    assert (prob.sens == 0).sum() > 0 and all((s == 0).sum() > 0 for s in prob.sens_t)
    img = _cuda(f0)
    state = pv.State(gp, method, img)
    alg = {"osem": None, "svrem": em.SVREM(prob, f0, 0.7, 1), "saga": em.SAGA(prob, f0, 1.0),
           "svrg": em.SVRG(prob, f0, 2.0, 2), "sga": em.SGA(prob, f0),
           "sem": em.SEM(prob, f0, schedule=lambda k: 1.0)}[method]
    f, errs = f0, []
    for k, t in enumerate(subset_sequence(6200, work.n_subsets, 3 * work.n_subsets)):
        if method in ("sga", "sem"):
            state.epoch([int(t)], alpha=1.0, decay=0.0)
        else:
            state.epoch([int(t)], alpha={"svrem": 0.7, "saga": 1.0, "svrg": 2.0}.get(method, 1.0),
                        eta={"svrg": 2}.get(method, 1))
        f = em.osem_step(prob, f, int(t)) if alg is None else alg.step(int(t))
        got = _host(img)
        errs.append(rel_l2(got, f))
        assert errs[-1] <= ITERATE_RTOL, f"step {k}: {errs[-1]:.3e}"
        S = prob.sens_t[int(t)] if method == "osem" else prob.sens
        if method in ("osem", "svrem", "sem"):
            dead = S[:, 0] == 0
            assert dead.any() and np.all(got[dead] == 0.0) and np.all(f[dead, 0] == 0.0)
    record_error(test="edge_unseen_pixels", case="sparse", method=method, table="fp32", epochs=3,
                 one_step=errs[0], trajectory=errs[-1], trajectory_max=max(errs))


def test_svrem_nonpositive_statistic(record_error):
    """SVREM with alpha = 2 drives s_hat_n <= 0 on up to 130 pixels per step
    (32x32, 5 subsets): those pixels are exactly 0 on both sides."""
    pv = _pv()
    work = Workload("svremneg", Geometry(32, 32, 30, 47), n_subsets=5, counts=2e5, bg_frac=0.1, beta=0.02,
                    n_ellipses=4)
    from oracle.em import build_problem
    from paper_2106_03172_gb300.phantoms import make_data
    data = make_data(work, 0)
    prob = build_problem(work.geometry, data["g"], data["w"], work.n_subsets, work.beta)
    plan = pv.Plan(work.geometry, work.n_subsets)
    gp = pv.Problem(plan, _cuda(data["g"]), None, data["w"], work.beta)
    f0 = prob.initial_image().astype(np.float32).astype(np.float64)
    img = _cuda(f0)
    state = pv.State(gp, "svrem", img)
    alg = em.SVREM(prob, f0, 2.0, 1)
    zeros_seen, errs = 0, []
    for k, t in enumerate(subset_sequence(5, work.n_subsets, 2 * work.n_subsets)):
        state.epoch([int(t)], alpha=2.0, eta=1)
        f = alg.step(int(t))
        got = _host(img)
        errs.append(rel_l2(got, f))
        assert errs[-1] <= ITERATE_RTOL, f"step {k}: {errs[-1]:.3e}"
        clear = alg.s_hat[:, 0] < -1e-5 * np.abs(alg.s_hat).max()     # not a borderline sign
        assert np.all(f[clear, 0] == 0.0) and np.all(got[clear] == 0.0)
        zeros_seen += int(clear.sum())
    assert zeros_seen > 50
    record_error(test="edge_svrem_nonpositive_statistic", case="32x32 alpha 2", method="svrem", table="fp32",
                 epochs=2, one_step=errs[0], trajectory=errs[-1], trajectory_max=max(errs))


@pytest.mark.parametrize("method,alpha", [("saga", 2.0), ("svrg", 3.0)])
def test_projection_clips(method, alpha, record_error):
    """SAGA / SVRG with steps large enough that P_{>=0} clips many pixels:
    where the oracle's unprojected value is clearly negative, both sides give
    exactly 0."""
    pv, prob, data, work, plan, gp, f0 = _setup("c64")
    img = _cuda(f0)
    state = pv.State(gp, method, img)
    alg = em.SAGA(prob, f0, alpha) if method == "saga" else em.SVRG(prob, f0, alpha, 2)
    clipped, errs = 0, []
    f = f0
    for k, t in enumerate(subset_sequence(6300, work.n_subsets, work.n_subsets)):
        state.epoch([int(t)], alpha=alpha, eta=2)
        f_prev = f.copy()
        if method == "saga":                               # the table before this step's write
            q_t, q_mean = alg.q[int(t)].copy(), sum(alg.q) / prob.Ns
        f = alg.step(int(t))
        got = _host(img)
        errs.append(rel_l2(got, f))
        assert errs[-1] <= ITERATE_RTOL, f"step {k}: {errs[-1]:.3e}"
        # the unprojected step from the same direction (SVRG's anchor is refreshed before its update)
        g_t = prob.grad_Phi_t(f_prev, int(t))
        if method == "saga":
            raw = f_prev + alpha * alg.d * (g_t - q_t + q_mean)
        else:
            raw = f_prev + alpha * alg.d * (g_t - alg.g_anc[int(t)] + alg.q_tilde)
        np.testing.assert_allclose(np.maximum(raw, 0.0), f, rtol=1e-12, atol=1e-12 * np.abs(f).max())
        clear = raw[:, 0] < -1e-5 * np.abs(f_prev).max()
        assert np.all(f[clear, 0] == 0.0) and np.all(got[clear] == 0.0)
        clipped += int(clear.sum())
    assert clipped > 20
    record_error(test="edge_projection_clips", case="c64", method=f"{method} alpha {alpha:g}", table="fp32",
                 epochs=1, one_step=errs[0], trajectory=errs[-1], trajectory_max=max(errs))


def test_numeric_latch_then_recovery():
    """f = 0 with w = 0 and g > 0: pet_objective returns PET_ERR_NUMERIC
    (a latched status word, read when it synchronises) and reports Phi = -inf;
    the status is cleared, and the next objective of a positive image (whose
    only zero means are on rays that miss the image, with zero counts) is the
    oracle's."""
    pv = _pv()
    prob, data, work = oracle_problem("nobg")
    assert data["w"] == 0.0
    plan = pv.Plan(work.geometry, work.n_subsets)
    gp = pv.Problem(plan, _cuda(data["g"]), None, 0.0, work.beta)
    zero = torch.zeros(prob.N, device="cuda")
    phi = torch.zeros(3, dtype=torch.float64, device="cuda")
    pv.pet_objective_async(gp.handle, zero, phi)          # enqueued: latches, returns OK
    torch.cuda.synchronize()
    assert phi[0].item() == -np.inf and phi[1].item() == -np.inf
    with pytest.raises(pv.PetError) as e:
        pv.pet_objective(gp.handle, zero)                 # synchronising: reports the latch
    assert e.value.status == 5
    f = prob.initial_image().astype(np.float32).astype(np.float64)
    assert pv.pet_objective(gp.handle, _cuda(f)) == pytest.approx(prob.objective(f), rel=1e-7)
