"""pet_state_run through the C ABI: updates with the objective inside give,
bit for bit, the iterates and objectives of the epoch calls with an
objective call after every epoch, including where an objective's forward
projection also serves the next anchor (SVREM, SVRG)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from cases import oracle_problem

pytestmark = pytest.mark.gpu

RUNS = [("c64", "osem", "fp32", 1.0, 1), ("c64", "svrem", "fp32", 0.7, 1), ("c64", "saga", "bf16", 1.0, 1),
        ("c64", "saga", "fp32", 1.0, 1), ("c64", "svrg", "fp32", 2.0, 2), ("ragged", "svrem", "fp32", 0.7, 2),
        ("ragged", "svrg", "fp32", 2.0, 1), ("c64", "sga", "fp32", 0.8, 1), ("c64", "sem", "fp32", 0.5, 1),
        ("c64", "sagaem", "fp32", 0.7, 1), ("stack", "svrem", "fp32", 0.7, 1), ("ring2", "svrg", "fp32", 2.0, 1)]


def _setup(name):
    from paper_2106_03172_gb300 import petvr as pv
    pv.lib()
    prob, data, work = oracle_problem(name)
    plan = pv.Plan(work.geometry, work.n_subsets)
    gp = pv.Problem(plan, torch.from_numpy(np.ascontiguousarray(data["g"]).ravel()).cuda(), None, data["w"],
                    work.beta)
    f0 = torch.empty(prob.N * prob.nz, device="cuda")
    pv.pet_warm_start(gp.handle, f0)
    return pv, plan, gp, f0, work


@pytest.mark.parametrize("name,algo,table,alpha,eta", RUNS)
@pytest.mark.parametrize("every", ["epoch", "4"])
def test_run_equals_epoch_calls_with_objectives(name, algo, table, alpha, eta, every):
    pv, plan, gp, f0, work = _setup(name)
    ns = work.n_subsets
    step = ns if every == "epoch" else 4
    n_iter = 3 * ns + (0 if every == "epoch" else 1)          # a tail after the last objective point
    points = n_iter // step
    seq = np.random.default_rng(ns + len(algo)).integers(0, ns, n_iter)
    decay = 0.01 if algo in ("sga", "sem") else 0.0
    a, b = f0.clone(), f0.clone()
    sa = pv.State(gp, algo, a, table=table)
    sb = pv.State(gp, algo, b, table=table)
    phi_a = torch.zeros(points, 3, dtype=torch.float64, device="cuda")
    phi_b = torch.zeros(points, 3, dtype=torch.float64, device="cuda")
    for rep in range(2):                    # the second call replays the captured graphs
        for j in range(points):
            sa.epoch(seq[j * step:(j + 1) * step], alpha=alpha, eta=eta, decay=decay)
            sa.objective_async(phi_a[j])
        sa.epoch(seq[points * step:], alpha=alpha, eta=eta, decay=decay)
        sb.run(seq, alpha=alpha, eta=eta, objective_every=step, phi=phi_b, decay=decay)
        torch.cuda.synchronize()
        assert torch.equal(a, b), (rep, name, algo)
        assert torch.equal(phi_a, phi_b), (rep, name, algo)
        assert torch.isfinite(phi_b).all()


def test_run_without_objectives_and_bad_arguments():
    pv, plan, gp, f0, work = _setup("c64")
    ns = work.n_subsets
    seq = list(range(ns)) * 2
    a, b = f0.clone(), f0.clone()
    sa, sb = pv.State(gp, "svrem", a), pv.State(gp, "svrem", b)
    sa.epoch(seq, alpha=0.7, eta=1)
    sb.run(seq, alpha=0.7, eta=1)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    with pytest.raises(ValueError):         # too small an output buffer, refused before the call
        sb.run(seq, alpha=0.7, objective_every=ns, phi=torch.zeros(1, 3, dtype=torch.float64, device="cuda"))
    with pytest.raises(pv.PetError):
        sb.run(seq, alpha=0.7, eta=0, objective_every=ns, phi=torch.zeros(2, 3, dtype=torch.float64, device="cuda"))


def test_many_output_buffers_evict_graphs_without_changing_results():
    """Each new output buffer is a new captured graph; past the cache's 64
    graphs the least recently used are destroyed (some still in flight),
    and every call still writes what the epoch calls give."""
    pv, plan, gp, f0, work = _setup("c64")
    ns = work.n_subsets
    a, b = f0.clone(), f0.clone()
    sa, sb = pv.State(gp, "svrg", a), pv.State(gp, "svrg", b)
    want, got = [], []
    for j in range(90):
        seq = np.random.default_rng(300 + j).integers(0, ns, ns)
        pa = torch.zeros(1, 3, dtype=torch.float64, device="cuda")
        pb = torch.zeros(1, 3, dtype=torch.float64, device="cuda")
        sa.epoch(seq, alpha=2.0, eta=2)
        sa.objective_async(pa[0])
        sb.run(seq, alpha=2.0, eta=2, objective_every=ns, phi=pb)
        want.append(pa)
        got.append(pb)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert torch.equal(torch.cat(want), torch.cat(got))
