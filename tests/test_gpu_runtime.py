"""GPU runtime behaviour through the C ABI: graph replay equals direct
launches, state reset equals a fresh state, launch accounting, and the
reconstructions reach the oracle's MAP objective."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from cases import oracle_problem, rel_l2
from oracle import em
from paper_2106_03172_gb300.phantoms import subset_sequence

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ALPHA = {"osem": (1.0, 1), "svrem": (0.7, 1), "saga": (1.0, 1), "svrg": (2.0, 2)}


def _pv():
    from paper_2106_03172_gb300 import petvr
    petvr.lib()
    return petvr


def _run_methods(case: str, epochs: int):
    """Images after `epochs` epochs of each method (as numpy arrays)."""
    pv = _pv()
    prob, data, work = oracle_problem(case)
    plan = pv.Plan(work.geometry, work.n_subsets)
    gp = pv.Problem(plan, torch.from_numpy(data["g"].ravel()).cuda(), None, data["w"], work.beta)
    f0 = torch.empty(prob.N * prob.nz, device="cuda")
    pv.pet_warm_start(gp.handle, f0)
    out = {}
    for m, (alpha, eta) in ALPHA.items():
        img = f0.clone()
        st = pv.State(gp, m, img)
        for e in range(epochs):
            st.epoch(subset_sequence(300 + e, work.n_subsets, work.n_subsets), alpha=alpha, eta=eta)
        torch.cuda.synchronize()
        out[m] = img.cpu().numpy()
    return out


def test_graph_replay_equals_direct_launches(tmp_path):
    """Epochs replayed from captured CUDA graphs give bit-identical images to
    the same launches issued directly (PETVR_NO_GRAPHS=1, in a subprocess)."""
    got = _run_methods("ragged", 3)
    path = tmp_path / "direct.npz"
    code = (f"import sys; sys.path.insert(0, {ROOT!r}); sys.path.insert(0, {os.path.join(ROOT, 'tests')!r});"
            "import numpy as np; from test_gpu_runtime import _run_methods;"
            f"np.savez({str(path)!r}, **_run_methods('ragged', 3))")
    env = dict(os.environ, PETVR_NO_GRAPHS="1")
    subprocess.run([sys.executable, "-c", code], check=True, env=env, cwd=ROOT)
    ref = np.load(path)
    for m in ALPHA:
        np.testing.assert_array_equal(got[m], ref[m], err_msg=m)


def test_state_reset_equals_fresh_state():
    pv = _pv()
    prob, data, work = oracle_problem("c64")
    plan = pv.Plan(work.geometry, work.n_subsets)
    gp = pv.Problem(plan, torch.from_numpy(data["g"].ravel()).cuda(), None, data["w"], work.beta)
    f0 = torch.from_numpy(prob.initial_image().astype(np.float32).ravel()).cuda()
    for m, (alpha, eta) in ALPHA.items():
        a = f0.clone()
        sa = pv.State(gp, m, a)
        for e in range(2):
            sa.epoch(subset_sequence(400 + e, work.n_subsets, work.n_subsets), alpha=alpha, eta=eta)
        b = a.clone()
        sb = pv.State(gp, m, b)                 # fresh state at the same image
        sa.reset()
        seq = subset_sequence(500, work.n_subsets, work.n_subsets)
        sa.epoch(seq, alpha=alpha, eta=eta)
        sb.epoch(seq, alpha=alpha, eta=eta)
        torch.cuda.synchronize()
        assert torch.equal(a, b), m


def test_problem_update_reaches_captured_epochs():
    """After pet_problem_update with new counts and a new scalar background,
    a state whose epochs were captured before (and reset) gives what a state
    of a fresh problem with that data gives: cached graphs do not keep the
    old background."""
    pv = _pv()
    prob, data, work = oracle_problem("c64")
    from paper_2106_03172_gb300.phantoms import make_data
    other = dict(make_data(work, 77))
    other["w"] = 1.5 * data["w"]                       # the generator's w depends only on the total counts
    plan = pv.Plan(work.geometry, work.n_subsets)
    gp = pv.Problem(plan, torch.from_numpy(data["g"].ravel()).cuda(), None, data["w"], work.beta)
    fresh = pv.Problem(plan, torch.from_numpy(other["g"].ravel()).cuda(), None, other["w"], work.beta)
    f0 = torch.from_numpy(prob.initial_image().astype(np.float32).ravel()).cuda()
    seq = subset_sequence(600, work.n_subsets, work.n_subsets)
    for m, (alpha, eta) in ALPHA.items():
        a, b = f0.clone(), f0.clone()
        sa = pv.State(gp, m, a)
        sa.epoch(seq, alpha=alpha, eta=eta)              # captures with the first data
        pv.pet_problem_update(gp.handle, torch.from_numpy(other["g"].ravel()).cuda(), None, other["w"])
        a.copy_(f0)
        sa.reset()
        sb = pv.State(fresh, m, b)
        sa.epoch(seq, alpha=alpha, eta=eta)
        sb.epoch(seq, alpha=alpha, eta=eta)
        phi_a = torch.zeros(3, dtype=torch.float64, device="cuda")
        phi_b = torch.zeros(3, dtype=torch.float64, device="cuda")
        sa.objective_async(phi_a)
        sb.objective_async(phi_b)
        torch.cuda.synchronize()
        assert torch.equal(a, b), m
        assert torch.equal(phi_a, phi_b), m
        pv.pet_problem_update(gp.handle, torch.from_numpy(data["g"].ravel()).cuda(), None, data["w"])


def test_launch_accounting_includes_graph_replays():
    pv = _pv()
    prob, data, work = oracle_problem("c64")
    plan = pv.Plan(work.geometry, work.n_subsets)
    gp = pv.Problem(plan, torch.from_numpy(data["g"].ravel()).cuda(), None, data["w"], work.beta)
    img = torch.from_numpy(prob.initial_image().astype(np.float32).ravel()).cuda()
    st = pv.State(gp, "osem", img)
    seq = subset_sequence(1, work.n_subsets, work.n_subsets)
    st.epoch(seq)                                # first call captures
    n0 = pv.pet_kernel_launches()
    st.epoch(seq)                                # replay
    torch.cuda.synchronize()
    assert pv.pet_kernel_launches() - n0 == 2 * work.n_subsets


def test_methods_reach_map_objective_like_the_oracle():
    """From the OSEM warm start, each variance-reduced method's objective gap
    to the L-BFGS-B optimum Phi* after 12 epochs matches the FP64 oracle's
    (same subset sequences) within 2% of the gap, and SVRG gets below 1e-4."""
    pv = _pv()
    prob, data, work = oracle_problem("c64")
    _, phi_star, _ = em.map_reference(prob)
    plan = pv.Plan(work.geometry, work.n_subsets)
    gp = pv.Problem(plan, torch.from_numpy(data["g"].ravel()).cuda(), None, data["w"], work.beta)
    f0 = prob.initial_image().astype(np.float32).astype(np.float64)
    algs = {"svrem": em.SVREM(prob, f0, *ALPHA["svrem"]), "saga": em.SAGA(prob, f0, ALPHA["saga"][0]),
            "svrg": em.SVRG(prob, f0, *ALPHA["svrg"])}
    for m, alg in algs.items():
        img = torch.from_numpy(f0.astype(np.float32).ravel()).cuda()
        st = pv.State(gp, m, img)
        for e in range(12):
            seq = subset_sequence(600 + e, work.n_subsets, work.n_subsets)
            st.epoch(seq, alpha=ALPHA[m][0], eta=ALPHA[m][1])
            for t in seq:
                alg.step(int(t))
        gap_gpu = em.relative_gap(pv.pet_objective(gp.handle, img), phi_star)
        gap_ora = em.relative_gap(prob.objective(alg.f), phi_star)
        assert gap_gpu == pytest.approx(gap_ora, rel=0.02), m
        if m == "svrg":
            assert gap_gpu <= 1e-4
        assert rel_l2(img.double().cpu().numpy(), alg.f) <= 1e-4
