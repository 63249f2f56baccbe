"""pet_run_to_gap through the C ABI: many reconstructions run to the
objective gap on several worker states and streams give, job by job, the
epochs and final images of the same warm start, reset, epoch calls and
objective checks run one job at a time on one stream."""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from cases import oracle_problem

pytestmark = pytest.mark.gpu

GAP = 1e-4
MAX_EPOCHS = 30


@functools.lru_cache(maxsize=None)
def _phi_star(name):
    from oracle.em import map_reference
    prob, _, _ = oracle_problem(name)
    return float(map_reference(prob)[1])


def _setup(name):
    from paper_2106_03172_gb300 import petvr as pv
    pv.lib()
    prob, data, work = oracle_problem(name)
    plan = pv.Plan(work.geometry, work.n_subsets)
    gp = pv.Problem(plan, torch.from_numpy(np.ascontiguousarray(data["g"]).ravel()).cuda(), None, data["w"],
                    work.beta)
    return pv, gp, prob.N * prob.nz, work


def _one_at_a_time(pv, gp, n, algo, table, seqs, ns, alpha, eta, decay, phi_star):
    img = torch.empty(n, device="cuda")
    st = pv.State(gp, algo, img, table=table)
    phi = torch.zeros(3, dtype=torch.float64, device="cuda")
    out = []
    for q in seqs:
        pv.pet_warm_start(gp.handle, img)
        st.reset()
        e = 0
        while True:
            st.epoch(q[e * ns:(e + 1) * ns], alpha=alpha, eta=eta, decay=decay)
            st.objective_async(phi)
            e += 1
            g = (phi_star - float(phi[0].cpu())) / abs(phi_star)
            if g <= GAP or e >= MAX_EPOCHS:
                break
        out.append((e, g, img.clone()))
    return out


@pytest.mark.parametrize("name,algo,table,alpha,eta,workers", [
    ("c64", "osem", "fp32", 1.0, 1, 3), ("c64", "svrem", "fp32", 0.7, 1, 3), ("c64", "saga", "bf16", 1.0, 1, 3),
    ("c64", "svrg", "fp32", 2.0, 2, 4), ("ragged", "svrem", "fp32", 0.7, 2, 2), ("ragged", "saga", "fp32", 1.0, 1, 5),
    ("c64", "sga", "fp32", 0.8, 1, 2), ("c64", "sem", "fp32", 0.5, 1, 3), ("c64", "sagaem", "fp32", 0.7, 1, 3),
    ("c64", "svrg", "fp32", 2.0, 1, 1)])
def test_executor_equals_one_job_at_a_time(name, algo, table, alpha, eta, workers):
    pv, gp, n, work = _setup(name)
    ns = work.n_subsets
    phi_star = _phi_star(name)
    decay = 0.01 if algo in ("sga", "sem") else 0.0
    n_jobs = 7
    seqs = np.random.default_rng(len(algo) + workers).integers(0, ns, (n_jobs, MAX_EPOCHS * ns)).astype(np.int32)
    imgs = [torch.empty(n, device="cuda") for _ in range(workers)]
    states = [pv.State(gp, algo, im, table=table) for im in imgs]
    results = torch.zeros(n_jobs, n, device="cuda")
    epochs, gaps, ms = pv.pet_run_to_gap(states, seqs, MAX_EPOCHS, phi_star, GAP, alpha=alpha, decay=decay, eta=eta,
                                         results=results)
    want = _one_at_a_time(pv, gp, n, algo, table, seqs, ns, alpha, eta, decay, phi_star)
    for j, (e, g, im) in enumerate(want):
        assert epochs[j] == e, (j, epochs[j], e)
        assert gaps[j] == g, (j, gaps[j], g)
        assert torch.equal(results[j], im), j
    assert np.all(ms > 0) and np.all(np.isfinite(gaps)) and np.all(epochs >= 1)


def test_executor_refuses_mixed_or_repeated_workers():
    pv, gp, n, work = _setup("c64")
    _, gp2, _, _ = _setup("c64")
    a, b, c = (torch.empty(n, device="cuda") for _ in range(3))
    s1, s2 = pv.State(gp, "osem", a), pv.State(gp, "svrem", b)
    s3 = pv.State(gp2, "osem", c)
    seqs = np.zeros((1, 2 * work.n_subsets), dtype=np.int32)
    for workers in ([s1, s2], [s1, s3], [s1, s1]):
        with pytest.raises(pv.PetError):
            pv.pet_run_to_gap(workers, seqs, 2, 1.0e6)
    with pytest.raises(pv.PetError):                 # a subset index out of range
        pv.pet_run_to_gap([s1], seqs + work.n_subsets, 2, 1.0e6)
    e, g, ms = pv.pet_run_to_gap([s1], np.zeros((0, 2 * work.n_subsets), dtype=np.int32), 2, 1.0e6)
    assert len(e) == 0


def test_jobs_on_their_own_states_equal_one_job_at_a_time():
    """pet_run_jobs_to_gap: jobs of different problems, plans and algorithms,
    each on its own state, up to three at a time; every job gives the epochs,
    gap and final image of the same calls made one job at a time."""
    from paper_2106_03172_gb300 import petvr as pv
    spec = [("c64", "svrem", "fp32", 0.7, 1), ("ragged", "saga", "fp32", 1.0, 1), ("c64", "osem", "fp32", 1.0, 1),
            ("ragged", "svrg", "fp32", 2.0, 2), ("c64", "sagaem", "fp32", 0.7, 1), ("c64", "saga", "bf16", 1.0, 1),
            ("ragged", "svrem", "fp32", 0.7, 1)]
    setups = {name: _setup(name) for name in ("c64", "ragged")}
    states, seqs, want = [], [], []
    for k, (name, algo, table, alpha, eta) in enumerate(spec):
        _, gp, n, work = setups[name]
        ns = work.n_subsets
        q = np.random.default_rng(40 + k).integers(0, ns, MAX_EPOCHS * ns).astype(np.int32)
        seqs.append(q)
        states.append(pv.State(gp, algo, torch.empty(n, device="cuda"), table=table))
        want.append(_one_at_a_time(pv, gp, n, algo, table, [q], ns, alpha, eta, 0.0, _phi_star(name))[0])
    epochs, gaps, ms = pv.pet_run_jobs_to_gap(states, seqs, [s[3] for s in spec], [s[4] for s in spec],
                                              [_phi_star(s[0]) for s in spec], MAX_EPOCHS, GAP, n_streams=3)
    for j, (e, g, im) in enumerate(want):
        assert epochs[j] == e and gaps[j] == g, (j, epochs[j], e, gaps[j], g)
        assert torch.equal(states[j].img, im), j
    assert np.all(ms > 0)
    with pytest.raises(pv.PetError):                 # one state for two jobs
        pv.pet_run_jobs_to_gap([states[0], states[0]], seqs[:1] * 2, [0.7] * 2, [1] * 2, [1.0e6] * 2, MAX_EPOCHS)
