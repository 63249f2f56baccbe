"""Batched updates through the C ABI: each member of a batch gives exactly
the image its own epoch calls give (mixed algorithms, table types, image
sizes and launch shapes in one batch)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from cases import oracle_problem
from paper_2106_03172_gb300.phantoms import subset_sequence

pytestmark = pytest.mark.gpu


def _pv():
    from paper_2106_03172_gb300 import petvr
    petvr.lib()
    return petvr


def _setup(pv, name, run=None):
    prob, data, work = oracle_problem(name)
    plan = pv.Plan(work.geometry, work.n_subsets)
    if run is not None:
        pv.pet_plan_set_tuning(plan.handle, 0, run)
    gp = pv.Problem(plan, torch.from_numpy(data["g"].ravel()).cuda(), None, data["w"], work.beta)
    f0 = torch.empty(prob.N, device="cuda")
    pv.pet_warm_start(gp.handle, f0)
    return plan, gp, f0, work


MEMBERS = [("c64", "osem", "fp32", 1.0, 1), ("c64", "svrem", "fp32", 0.7, 1), ("c64", "saga", "bf16", 1.0, 1),
           ("c64", "svrg", "fp32", 2.0, 2), ("ragged", "svrem", "fp32", 0.7, 1), ("ragged", "saga", "fp32", 1.0, 1),
           ("c256", "svrg", "fp32", 2.0, 1), ("c64", "sga", "fp32", 0.8, 1), ("ragged", "sem", "fp32", 0.5, 1),
           ("c64", "sagaem", "fp32", 0.7, 1)]


@pytest.mark.parametrize("mode", ["phases", "dataflow", "streams"])
def test_batch_equals_individual_epochs(mode):
    """Both batch modes (persistent phases; one dependency-driven launch per
    call) give every member exactly its own epochs' iterates and objectives."""
    pv = _pv()
    setups = {"c64": _setup(pv, "c64"), "ragged": _setup(pv, "ragged", run=4), "c256": _setup(pv, "c256")}
    solo, batched, solo_states, batch_states = [], [], [], []
    for name, algo, table, alpha, eta in MEMBERS:
        plan, gp, f0, work = setups[name]
        a, b = f0.clone(), f0.clone()
        solo.append(a)
        batched.append(b)
        solo_states.append(pv.State(gp, algo, a, table=table))
        batch_states.append(pv.State(gp, algo, b, table=table))
    batch = pv.Batch(batch_states)
    batch.set_mode(mode)
    rng = np.random.default_rng(5)
    for n_iter in (7, 4, 21):
        seqs = [rng.integers(0, setups[m[0]][3].n_subsets, n_iter) for m in MEMBERS]
        batch.epoch(seqs, [m[3] for m in MEMBERS], [m[4] for m in MEMBERS])
        for st, q, m in zip(solo_states, seqs, MEMBERS):
            st.epoch(q, alpha=m[3], eta=m[4])
        batch.sync()
        for a, b, m in zip(solo, batched, MEMBERS):
            assert torch.equal(a, b), (n_iter, m)
    phi_b = torch.empty(len(MEMBERS), 3, dtype=torch.float64, device="cuda")
    phi_s = torch.empty(len(MEMBERS), 3, dtype=torch.float64, device="cuda")
    batch.objective_async(phi_b)
    for j, st in enumerate(solo_states):
        st.objective_async(phi_s[j])
    torch.cuda.synchronize()
    assert torch.equal(phi_b, phi_s)


def test_batch_rejects_bad_input():
    pv = _pv()
    plan, gp, f0, work = _setup(pv, "c64")
    st = pv.State(gp, "osem", f0.clone())
    with pytest.raises(pv.PetError):
        pv.Batch([st, st])
    batch = pv.Batch([st])
    with pytest.raises(pv.PetError):
        batch.epoch([[0, work.n_subsets]], [1.0], [1])
    # batches take single-slice images: a multi-ring volume is refused
    plan3, gp3, f3, _ = _setup(pv, "ring2")
    with pytest.raises(pv.PetError):
        pv.Batch([pv.State(gp3, "saga", f3.clone())])


def test_batch_mixed_potentials_and_many_members():
    """A batch whose members use both the quadratic and an edge-preserving
    potential (two back-projection launches per phase), with 170 members so
    that the work lists outgrow the segment table a block stages in shared
    memory: every member still matches its own epochs bit for bit."""
    pv = _pv()
    from paper_2106_03172_gb300.phantoms import Geometry, Workload, make_data
    geoms = [Geometry(16, 16, 8, 23), Geometry(20, 12, 9, 25, bin_mm=1.5), Geometry(24, 24, 10, 35)]
    algos = ["osem", "saga", "svrg", "svrem", "sga"]
    members = []
    for j in range(170):
        geom = geoms[j % 3]
        pot = "logcosh" if j % 4 == 1 else "quadratic"
        work = Workload(f"m{j}", geom, n_subsets=2 + j % 3, counts=2e4, bg_frac=0.1, beta=0.3 if pot != "quadratic"
                        else 0.02, n_ellipses=3)
        data = make_data(work, 300 + j)
        plan = pv.Plan(geom, work.n_subsets)
        gp = pv.Problem(plan, torch.from_numpy(data["g"].ravel()).cuda(), None, data["w"], work.beta,
                        potential=pot, delta=0.1)
        f0 = torch.empty(geom.n_pixels, device="cuda")
        pv.pet_warm_start(gp.handle, f0)
        a, b = f0.clone(), f0.clone()
        algo = algos[j % len(algos)]
        members.append((work, plan, gp, a, b, pv.State(gp, algo, a), pv.State(gp, algo, b), algo))
    batch = pv.Batch([m[6] for m in members])
    rng = np.random.default_rng(9)
    alphas = [0.7 if m[7] == "svrem" else 1.0 for m in members]
    etas = [1 for _ in members]
    for n_iter in (5, 6):
        seqs = [rng.integers(0, m[0].n_subsets, n_iter) for m in members]
        batch.epoch(seqs, alphas, etas)
        for m, q, al, et in zip(members, seqs, alphas, etas):
            m[5].epoch(q, alpha=al, eta=et)
        torch.cuda.synchronize()
        for m in members:
            assert torch.equal(m[3], m[4]), (n_iter, m[0].name, m[7])
    phi_b = torch.empty(len(members), 3, dtype=torch.float64, device="cuda")
    phi_s = torch.empty(len(members), 3, dtype=torch.float64, device="cuda")
    batch.objective_async(phi_b)
    for j, m in enumerate(members):
        m[5].objective_async(phi_s[j])
    torch.cuda.synchronize()
    assert torch.equal(phi_b, phi_s)


def test_dataflow_wait_that_runs_out_latches_timeout():
    """A dependency wait of the dataflow epoch that runs out latches
    PET_ERR_TIMEOUT, which pet_batch_sync reports; the launch still ends and
    the GPU stays usable.  With a limit of 0 polls, the first back-projection
    items of a 256^2 member (claimed by the grid's first wave while its forward
    items are still running) fail their wait.  A fresh batch with the default
    limit then matches the member's own epochs again."""
    pv = _pv()
    plan, gp, f0, work = _setup(pv, "c256")
    img = f0.clone()
    st = pv.State(gp, "osem", img)
    batch = pv.Batch([st])
    batch.set_mode("dataflow")
    batch.set_wait_limit(0)
    seq = [np.arange(work.n_subsets) % work.n_subsets]
    batch.epoch(seq, [1.0], [1])
    with pytest.raises(pv.PetError) as e:
        batch.sync()
    assert e.value.status == 4
    batch.sync()                                   # the status word was cleared
    # recovery: fresh states, default limit, bit-identical to solo epochs
    a, b = f0.clone(), f0.clone()
    solo, member = pv.State(gp, "svrg", a), pv.State(gp, "svrg", b)
    batch2 = pv.Batch([member])
    batch2.set_mode("dataflow")
    for epoch in range(2):
        q = np.random.default_rng(epoch).integers(0, work.n_subsets, work.n_subsets)
        batch2.epoch([q], [2.0], [2])
        solo.epoch(q, alpha=2.0, eta=2)
    batch2.sync()
    torch.cuda.synchronize()
    assert torch.equal(a, b)
