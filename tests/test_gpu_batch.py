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


def test_batch_equals_individual_epochs():
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
    rng = np.random.default_rng(5)
    for n_iter in (7, 4, 21):
        seqs = [rng.integers(0, setups[m[0]][3].n_subsets, n_iter) for m in MEMBERS]
        batch.epoch(seqs, [m[3] for m in MEMBERS], [m[4] for m in MEMBERS])
        for st, q, m in zip(solo_states, seqs, MEMBERS):
            st.epoch(q, alpha=m[3], eta=m[4])
        torch.cuda.synchronize()
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
