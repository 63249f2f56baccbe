"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (float32 kernels against float64 oracle):
  * projections: per element |gpu - oracle| <= 2e-5 |oracle| + 2e-6 max|oracle|
    (FP32 accumulation along rays of up to ~2n pixels and FP32 ray geometry);
  * every iterate of a trajectory (the first update from the same iterate and
    every later one, up to three epochs): relative L2 <= 1e-5, the stated
    per-iterate tolerance; objective |dPhi|/|Phi| <= 1e-7;
  * FP64 objective of a given image: relative 1e-7;
  * BF16 SAGA table against the oracle's BF16 emulation: one update within
    1e-5, three epochs within 1e-4.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from cases import CASES, oracle_problem, rel_l2
from oracle import em
from paper_2106_03172_gb300.phantoms import subset_sequence

pytestmark = pytest.mark.gpu

PROJ_RTOL, PROJ_ATOL = 2e-5, 2e-6
# FP32 iterates against the FP64 oracle, relative L2, at EVERY step of a
# trajectory (the stated per-iterate tolerance).  Measured: one update from
# the same iterate 4e-8 to 1.3e-7; after two epochs of the small cases at most
# 5.4e-7; after three epochs at 256^2 at most 2.2e-6 (SVRG).
ITERATE_RTOL = 1e-5
# BF16 SAGA table against the oracle's BF16 rounding: a rounding decision can
# flip where the FP32 inputs differ by an ulp, and such flips accumulate
# (measured up to 6e-5 after three epochs); one update stays within ITERATE_RTOL.
BF16_TRAJ_RTOL = 1e-4
METHOD_SEED = {"osem": 0, "svrem": 1, "saga": 2, "svrg": 3}


def _pv():
    from paper_2106_03172_gb300 import petvr
    petvr.lib()
    return petvr


def _cuda(x):
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def _assert_proj(gpu, ora):
    ora = np.asarray(ora, dtype=np.float64)
    tol = PROJ_RTOL * np.abs(ora) + PROJ_ATOL * np.abs(ora).max()
    err = np.abs(gpu - ora)
    assert np.all(err <= tol), f"max err {err.max():.3e}, worst ratio {(err / tol).max():.2f}"


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    pv = _pv()
    prob, data, work = oracle_problem(request.param)
    plan = pv.Plan(work.geometry, work.n_subsets)
    return pv, prob, data, work, plan


def test_forward_parity(case):
    pv, prob, data, work, plan = case
    geom = work.geometry
    f = np.random.default_rng(1).uniform(0.5, 3.0, (prob.N, prob.nz))
    fd = _cuda(f)
    out = torch.empty(prob.M * prob.nz, device="cuda")
    pv.pet_forward(plan.handle, fd, None, 0.25, -1, out)
    _assert_proj(_host(out).reshape(-1, prob.nz), prob.A @ f + 0.25)
    bg = np.random.default_rng(2).uniform(0.0, 1.0, (prob.M, prob.nz))
    for t in range(work.n_subsets):
        rows = prob.subsets[t]
        sub = torch.empty(len(rows) * prob.nz, device="cuda")
        pv.pet_forward(plan.handle, fd, _cuda(bg[rows]), 0.0, t, sub)
        _assert_proj(_host(sub).reshape(-1, prob.nz), prob.At[t] @ f + bg[rows])


def test_back_parity_and_adjoint(case):
    pv, prob, data, work, plan = case
    geom = work.geometry
    y = np.random.default_rng(3).uniform(0.0, 2.0, (prob.M, prob.nz))
    img = torch.empty(prob.N * prob.nz, device="cuda")
    pv.pet_back(plan.handle, _cuda(y), -1, img)
    _assert_proj(_host(img).reshape(-1, prob.nz), prob.A.T @ y)
    for t in range(work.n_subsets):
        rows = prob.subsets[t]
        pv.pet_back(plan.handle, _cuda(y[rows]), t, img)
        _assert_proj(_host(img).reshape(-1, prob.nz), prob.At[t].T @ y[rows])
    # adjoint identity <A x, y> = <x, A^T y>, both sides on the GPU
    x = np.random.default_rng(4).uniform(0.0, 1.0, (prob.N, prob.nz))
    ax = torch.empty(prob.M * prob.nz, device="cuda")
    pv.pet_forward(plan.handle, _cuda(x), None, 0.0, -1, ax)
    pv.pet_back(plan.handle, _cuda(y), -1, img)
    lhs = float((_host(ax) * y.ravel().astype(np.float32)).sum())
    rhs = float((_host(img) * x.ravel().astype(np.float32)).sum())
    assert lhs == pytest.approx(rhs, rel=2e-6)


def test_nonzero_counts(case):
    """The library's nonzero count of every A_t matches the oracle's CSR up to
    slivers: entries a ray gets from passing within rounding distance of a
    pixel corner (far below 1e-4 mm), which FP32 and FP64 may keep or drop."""
    pv, prob, data, work, plan = case
    for t in list(range(work.n_subsets)) + [-1]:
        A = prob.A if t < 0 else prob.At[t]
        got = pv.pet_plan_nnz(plan.handle, t)
        assert int((A.data > 1e-4).sum()) <= got <= A.nnz + max(10, A.nnz // 1000), (t, got, A.nnz)


@pytest.mark.parametrize("chunks,run", [(8, 4), (8, 8), (16, 4), (16, 8), (32, 4), (32, 8)])
def test_projection_parity_every_launch_shape(chunks, run):
    """Every forward chunk count and back-projection run length the autotuner
    may pick gives the oracle's projections (odd, non-square image)."""
    pv = _pv()
    prob, data, work = oracle_problem("ragged")
    plan = pv.Plan(work.geometry, work.n_subsets)
    pv.pet_plan_set_tuning(plan.handle, chunks, run)
    assert pv.pet_plan_get_tuning(plan.handle) == (chunks, run)
    f = np.random.default_rng(8).uniform(0.5, 3.0, (prob.N, 1))
    y = np.random.default_rng(9).uniform(0.0, 2.0, (prob.M, 1))
    img = torch.empty(prob.N, device="cuda")
    for t in range(work.n_subsets):
        rows = prob.subsets[t]
        sub = torch.empty(len(rows), device="cuda")
        pv.pet_forward(plan.handle, _cuda(f), None, 0.0, t, sub)
        _assert_proj(_host(sub).reshape(-1, 1), prob.At[t] @ f)
        pv.pet_back(plan.handle, _cuda(y[rows]), t, img)
        _assert_proj(_host(img).reshape(-1, 1), prob.At[t].T @ y[rows])
    pv.pet_back(plan.handle, _cuda(y), -1, img)
    _assert_proj(_host(img).reshape(-1, 1), prob.A.T @ y)


def test_autotune_picks_a_valid_shape():
    pv = _pv()
    prob, data, work = oracle_problem("c64")
    plan = pv.Plan(work.geometry, work.n_subsets)
    chunks, run = pv.pet_plan_autotune(plan.handle)
    assert chunks in (8, 16, 32) and run in (4, 8)
    assert pv.pet_plan_get_tuning(plan.handle) == (chunks, run)
    with pytest.raises(pv.PetError):
        pv.pet_plan_set_tuning(plan.handle, 12, 8)


def test_sensitivities(case):
    pv, prob, data, work, plan = case
    out = torch.empty(prob.N, device="cuda")
    pv.pet_plan_sensitivity(plan.handle, -1, out)
    _assert_proj(_host(out), prob.sens[:, 0])
    for t in range(work.n_subsets):
        pv.pet_plan_sensitivity(plan.handle, t, out)
        _assert_proj(_host(out), prob.sens_t[t][:, 0])


def _gpu_problem(pv, plan, data, work):
    return pv.Problem(plan, _cuda(data["g"]), None, data["w"], work.beta)


def test_objective_and_warm_start(case, record_error):
    pv, prob, data, work, plan = case
    gp = _gpu_problem(pv, plan, data, work)
    img = torch.empty(prob.N * prob.nz, device="cuda")
    pv.pet_warm_start(gp.handle, img)
    f0 = prob.initial_image()
    err = rel_l2(_host(img), f0)
    assert err <= ITERATE_RTOL
    f = f0.astype(np.float32).astype(np.float64)
    phi_gpu, phi_ora = pv.pet_objective(gp.handle, _cuda(f)), prob.objective(f)
    record_error(test="objective_and_warm_start", case=work.name, method="warm start", table="-", epochs=1,
                 one_step=err, phi_rel=abs(phi_gpu - phi_ora) / abs(phi_ora))
    assert phi_gpu == pytest.approx(phi_ora, rel=1e-7)


def _oracle_alg(prob, method, f0, work, table="fp32"):
    if method == "osem":
        return None
    if method == "svrem":
        return em.SVREM(prob, f0, work.alpha_svrem, work.eta_svrem)
    if method == "saga":
        return em.SAGA(prob, f0, work.alpha_saga, table=table)
    return em.SVRG(prob, f0, work.alpha_svrg, work.eta_svrg)


def _gpu_step(state, method, t, work):
    state.epoch([t], alpha={"svrem": work.alpha_svrem, "saga": work.alpha_saga,
                            "svrg": work.alpha_svrg}.get(method, 1.0),
                eta={"svrem": work.eta_svrem, "svrg": work.eta_svrg}.get(method, 1))


@pytest.mark.parametrize("method", ["osem", "svrem", "saga", "svrg"])
def test_update_parity(case, method, record_error):
    """Two epochs step by step, every iterate within the per-iterate
    tolerance (the first one is an update from the same iterate), and the
    objective within 1e-7."""
    pv, prob, data, work, plan = case
    gp = _gpu_problem(pv, plan, data, work)
    f0 = prob.initial_image().astype(np.float32).astype(np.float64)
    img = _cuda(f0)
    state = pv.State(gp, method, img)
    alg = _oracle_alg(prob, method, f0, work)
    seq = subset_sequence(2000 + METHOD_SEED[method], work.n_subsets, 2 * work.n_subsets)
    f = f0
    errs = []
    for k, t in enumerate(seq):
        _gpu_step(state, method, int(t), work)
        f = em.osem_step(prob, f, int(t)) if alg is None else alg.step(int(t))
        err = rel_l2(_host(img), f)
        errs.append(err)
        assert err <= ITERATE_RTOL, f"step {k}: {err:.3e}"
    phi_gpu = pv.pet_objective(gp.handle, img)
    phi_ora = prob.objective(f)
    record_error(test="update_parity", case=work.name, method=method, table="fp32", epochs=2,
                 one_step=errs[0], trajectory=errs[-1], trajectory_max=max(errs),
                 phi_rel=abs(phi_gpu - phi_ora) / abs(phi_ora))
    assert phi_gpu == pytest.approx(phi_ora, rel=1e-7)
    assert _host(img).min() >= 0.0


@pytest.mark.parametrize("name", ["c64", "ragged", "stack", "ring2"])
def test_saga_bf16_table(name, record_error):
    """SAGA with the BF16 table (FP32 running mean) against the oracle's BF16
    rounding of every stored entry, three epochs."""
    pv = _pv()
    prob, data, work = oracle_problem(name)
    plan = pv.Plan(work.geometry, work.n_subsets)
    gp = _gpu_problem(pv, plan, data, work)
    f0 = prob.initial_image().astype(np.float32).astype(np.float64)
    img = _cuda(f0)
    state = pv.State(gp, "saga", img, table="bf16")
    alg = em.SAGA(prob, f0, work.alpha_saga, table="bf16")
    errs = []
    for t in subset_sequence(7, work.n_subsets, 3 * work.n_subsets):
        _gpu_step(state, "saga", int(t), work)
        f = alg.step(int(t))
        errs.append(rel_l2(_host(img), f))
    phi_gpu, phi_ora = pv.pet_objective(gp.handle, img), prob.objective(f)
    record_error(test="saga_bf16_table", case=name, method="saga", table="bf16", epochs=3, one_step=errs[0],
                 trajectory=errs[-1], trajectory_max=max(errs), phi_rel=abs(phi_gpu - phi_ora) / abs(phi_ora))
    assert errs[0] <= ITERATE_RTOL
    assert max(errs) <= BF16_TRAJ_RTOL


def test_epoch_calls_equal_step_calls():
    """An epoch call equals the same updates issued one call at a time
    (ping-pong buffering and the anchor counter are invisible to the caller)."""
    pv = _pv()
    prob, data, work = oracle_problem("ragged")
    plan = pv.Plan(work.geometry, work.n_subsets)
    gp = _gpu_problem(pv, plan, data, work)
    f0 = prob.initial_image().astype(np.float32)
    seq = subset_sequence(11, work.n_subsets, 3 * work.n_subsets)
    for method in ("osem", "svrem", "saga", "svrg"):
        a, b = _cuda(f0), _cuda(f0)
        sa, sb = pv.State(gp, method, a), pv.State(gp, method, b)
        sa.epoch(seq, alpha=0.7, eta=1)
        for t in seq:
            sb.epoch([int(t)], alpha=0.7, eta=1)
        torch.cuda.synchronize()
        assert torch.equal(a, b), method


def test_error_handling():
    pv = _pv()
    from paper_2106_03172_gb300.phantoms import Geometry
    with pytest.raises(pv.PetError) as e:
        pv.Plan(Geometry(0, 8, 10, 11), 2)
    assert e.value.status == 1
    with pytest.raises(pv.PetError):
        pv.Plan(Geometry(8, 8, 4, 11), 5)          # more subsets than views
    prob, data, work = oracle_problem("ragged")
    plan = pv.Plan(work.geometry, work.n_subsets)
    out = torch.empty(10, device="cuda")
    with pytest.raises(pv.PetError):
        pv.pet_forward(plan.handle, _cuda(np.ones(prob.N)), None, 0.0, work.n_subsets, out)
    gp = _gpu_problem(pv, plan, data, work)
    img = _cuda(prob.initial_image())
    before = img.clone()
    st = pv.State(gp, "osem", img)
    st.epoch([])                                      # zero updates: a no-op
    torch.cuda.synchronize()
    assert torch.equal(img, before)
    with pytest.raises(pv.PetError) as e:
        pv.pet_svrem_epoch(st.handle, 0.5, 1, [0])   # wrong algorithm for this state
    assert e.value.status == 6
    with pytest.raises(pv.PetError) as e:
        st.epoch([0, 99])                             # out-of-range subset: nothing enqueued
    assert e.value.status == 1
    torch.cuda.synchronize()
    assert torch.equal(img, before)
    assert pv.pet_state_bytes(gp.handle, "saga", "bf16") < pv.pet_state_bytes(gp.handle, "saga", "fp32")


@pytest.fixture(scope="module")
def full256():
    pv = _pv()
    prob, data, work = oracle_problem("c256")
    plan = pv.Plan(work.geometry, work.n_subsets)
    return pv, prob, data, work, plan


def test_full_size_projection_parity(full256):
    """256x256, 180 views x 367 bins, 21 subsets: every subset's forward and
    back projection in the launch configuration the benchmark times."""
    pv, prob, data, work, plan = full256
    f = prob.initial_image()
    fd = _cuda(f)
    y = np.random.default_rng(5).uniform(0.0, 2.0, (prob.M, 1))
    img = torch.empty(prob.N, device="cuda")
    for t in range(work.n_subsets):
        rows = prob.subsets[t]
        sub = torch.empty(len(rows), device="cuda")
        pv.pet_forward(plan.handle, fd, None, data["w"], t, sub)
        _assert_proj(_host(sub).reshape(-1, 1), prob.At[t] @ f + data["w"])
        pv.pet_back(plan.handle, _cuda(y[rows]), t, img)
        _assert_proj(_host(img).reshape(-1, 1), prob.At[t].T @ y[rows])


@pytest.mark.parametrize("method,table", [("osem", "fp32"), ("svrem", "fp32"), ("saga", "fp32"),
                                          ("saga", "bf16"), ("svrg", "fp32")])
def test_full_size_three_epochs(full256, method, table, record_error):
    """256x256, 21 subsets, in the launch configuration the benchmark times
    (captured epochs): the first update, then three epochs, so that SVREM
    and SVRG take new anchors (SVRG every second epoch) and every SAGA table
    entry is rewritten, each epoch end within the per-iterate tolerance
    (BF16 table: its trajectory tolerance), and the objective within 1e-7."""
    pv, prob, data, work, plan = full256
    gp = _gpu_problem(pv, plan, data, work)
    f0 = prob.initial_image().astype(np.float32).astype(np.float64)
    img = _cuda(f0)
    state = pv.State(gp, method, img, table=table)
    alg = (em.SAGA(prob, f0, work.alpha_saga, table=table) if method == "saga"
           else _oracle_alg(prob, method, f0, work))
    alpha = {"svrem": work.alpha_svrem, "saga": work.alpha_saga, "svrg": work.alpha_svrg}.get(method, 1.0)
    eta = {"svrem": work.eta_svrem, "svrg": work.eta_svrg}.get(method, 1)
    seq = subset_sequence(2000, work.n_subsets, 3 * work.n_subsets)
    _gpu_step(state, method, int(seq[0]), work)
    f = em.osem_step(prob, f0, int(seq[0])) if alg is None else alg.step(int(seq[0]))
    one = rel_l2(_host(img), f)
    assert one <= ITERATE_RTOL
    ns = work.n_subsets
    errs = []
    for e in range(3):
        part = seq[max(1, e * ns):(e + 1) * ns]
        state.epoch(part, alpha=alpha, eta=eta)
        for t in part:
            f = em.osem_step(prob, f, int(t)) if alg is None else alg.step(int(t))
        errs.append(rel_l2(_host(img), f))
        assert errs[-1] <= (BF16_TRAJ_RTOL if table == "bf16" else ITERATE_RTOL), f"epoch {e}: {errs[-1]:.3e}"
    phi_gpu, phi_ora = pv.pet_objective(gp.handle, img), prob.objective(f)
    record_error(test="full_size_three_epochs", case=work.name, method=method, table=table, epochs=3,
                 one_step=one, trajectory=errs[-1], trajectory_max=max(errs),
                 phi_rel=abs(phi_gpu - phi_ora) / abs(phi_ora))
    assert phi_gpu == pytest.approx(phi_ora, rel=1e-7)


def test_full_size_stack_projection():
    """128x128 x 47 slices, 252 views x 344 bins: forward and back of every
    slice through one traversal."""
    pv = _pv()
    from oracle.siddon import system_matrix
    from paper_2106_03172_gb300.phantoms import WORKLOADS
    work = WORKLOADS["c128x47"]
    geom = work.geometry
    A = system_matrix(geom)
    plan = pv.Plan(geom, work.n_subsets)
    f = np.random.default_rng(6).uniform(0.0, 2.0, (geom.n_pixels, geom.nz))
    out = torch.empty(geom.n_rays * geom.nz, device="cuda")
    pv.pet_forward(plan.handle, _cuda(f), None, 0.0, -1, out)
    _assert_proj(_host(out).reshape(-1, geom.nz), A @ f)
    y = np.random.default_rng(7).uniform(0.0, 2.0, (geom.n_rays, geom.nz))
    img = torch.empty(geom.n_pixels * geom.nz, device="cuda")
    pv.pet_back(plan.handle, _cuda(y), -1, img)
    _assert_proj(_host(img).reshape(-1, geom.nz), A.T @ y)


def test_max_size_projection_samples():
    """512x512, 720 views x 733 bins (the largest serving size), 6 subsets:
    sampled rays of the all-view forward projection and sampled pixels of the
    all-view back projection against the oracle's Siddon rays computed one by
    one, and the adjoint identity <A x, y> = <x, A^T y> over the whole image."""
    pv = _pv()
    from oracle.geometry import bin_offsets, view_trig
    from oracle.siddon import siddon_ray
    from paper_2106_03172_gb300.phantoms import Geometry
    geom = Geometry(512, 512, 720, 733)
    nx, ny, na, nb, d = geom.nx, geom.ny, geom.n_angles, geom.n_bins, geom.pixel_mm
    plan = pv.Plan(geom, 6)
    rng = np.random.default_rng(11)
    f = rng.uniform(0.0, 2.0, nx * ny)
    y = rng.uniform(0.0, 2.0, na * nb)
    out = torch.empty(na * nb, device="cuda")
    pv.pet_forward(plan.handle, _cuda(f), None, 0.0, -1, out)
    img = torch.empty(nx * ny, device="cuda")
    pv.pet_back(plan.handle, _cuda(y), -1, img)
    fwd, back = _host(out), _host(img)
    c, s = view_trig(na)
    sj = bin_offsets(nb, geom.ds)

    # sampled rays, one by one
    rays = rng.choice(na * nb, 300, replace=False)
    want = []
    for m in rays:
        idx, ln = siddon_ray(c[m // nb], s[m // nb], sj[m % nb], nx, ny, d)
        want.append(float(np.dot(ln, f[idx])))
    want = np.asarray(want)
    _assert_proj(fwd[rays].reshape(-1, 1), want.reshape(-1, 1))

    # sampled pixels: every ray passing within two pixels of the pixel centre
    pix = rng.choice(nx * ny, 24, replace=False)
    got, want = back[pix], []
    for n in pix:
        ix, iy = n % nx, n // nx
        xc, yc = (ix - 0.5 * (nx - 1)) * d, (iy - 0.5 * (ny - 1)) * d
        total = 0.0
        for i in range(na):
            sc = xc * c[i] + yc * s[i]                     # the pixel centre's radial coordinate
            for j in np.nonzero(np.abs(sj - sc) <= 2.0 * d)[0]:
                idx, ln = siddon_ray(c[i], s[i], sj[j], nx, ny, d)
                hit = ln[idx == n]
                if hit.size:
                    total += float(hit.sum()) * y[i * nb + j]
        want.append(total)
    _assert_proj(got.reshape(-1, 1), np.asarray(want).reshape(-1, 1))

    # adjoint over the whole image (FP64 dot products of the FP32 outputs)
    lhs, rhs = float(np.dot(fwd, y)), float(np.dot(f, back))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


@pytest.fixture(scope="module", params=[("huber", 0.05), ("logcosh", 0.05), ("hyperbola", 0.05)])
def potential_case(request):
    """64x64 workload with an edge-preserving potential of Table 1 (the paper's
    experiments use log cosh) and a penalty weight large enough to matter."""
    from oracle.em import build_problem
    from paper_2106_03172_gb300.phantoms import WORKLOADS, make_data
    pv = _pv()
    pot, delta = request.param
    work = WORKLOADS["c64"]
    data = make_data(work, 0)
    beta = 0.5
    prob = build_problem(work.geometry, data["g"], data["w"], work.n_subsets, beta, pot, delta)
    plan = pv.Plan(work.geometry, work.n_subsets)
    gp = pv.Problem(plan, _cuda(data["g"]), None, data["w"], beta, potential=pot, delta=delta)
    return pv, prob, work, plan, gp


@pytest.mark.parametrize("method", ["osem", "svrem", "saga", "svrg"])
def test_edge_preserving_potential_updates(potential_case, method, record_error):
    pv, prob, work, plan, gp = potential_case
    f0 = prob.initial_image().astype(np.float32).astype(np.float64)
    img = _cuda(f0)
    state = pv.State(gp, method, img)
    alg = _oracle_alg(prob, method, f0, work)
    seq = subset_sequence(3000 + METHOD_SEED[method], work.n_subsets, 2 * work.n_subsets)
    f = f0
    errs = []
    for k, t in enumerate(seq):
        _gpu_step(state, method, int(t), work)
        f = em.osem_step(prob, f, int(t)) if alg is None else alg.step(int(t))
        err = rel_l2(_host(img), f)
        errs.append(err)
        assert err <= ITERATE_RTOL, f"step {k}: {err:.3e}"
    phi_gpu, phi_ora = pv.pet_objective(gp.handle, img), prob.objective(f)
    record_error(test="edge_preserving_potential", case=f"c64 {prob.pen.potential}", method=method, table="fp32",
                 epochs=2, one_step=errs[0], trajectory=errs[-1], trajectory_max=max(errs),
                 phi_rel=abs(phi_gpu - phi_ora) / abs(phi_ora))
    assert phi_gpu == pytest.approx(phi_ora, rel=1e-7)


def test_edge_preserving_potential_objective(potential_case):
    pv, prob, work, plan, gp = potential_case
    f = np.random.default_rng(12).uniform(0.05, 0.6, (prob.N, 1)).astype(np.float32).astype(np.float64)
    assert pv.pet_objective(gp.handle, _cuda(f)) == pytest.approx(prob.objective(f), rel=1e-7)
    assert prob.pen.value(f)[0] > 0.0


@pytest.mark.parametrize("method,alpha0,decay", [("sga", 1.0, 0.0), ("sga", 1.0, 0.001), ("sem", 1.0, 0.001)])
def test_non_vr_baseline_updates(case, method, alpha0, decay, record_error):
    """The paper's baselines on the same kernels (§5.1): SGA, the subset
    BSREM (SGA with alpha_k = (0.001 k + 1)^-1) and SEM, against the oracle."""
    pv, prob, data, work, plan = case
    gp = _gpu_problem(pv, plan, data, work)
    f0 = prob.initial_image().astype(np.float32).astype(np.float64)
    img = _cuda(f0)
    state = pv.State(gp, method, img)
    sched = lambda k: alpha0 / (decay * k + 1.0)
    alg = em.SGA(prob, f0, sched) if method == "sga" else em.SEM(prob, f0, sched)
    seq = subset_sequence(4000, work.n_subsets, 2 * work.n_subsets)
    errs = []
    for k, t in enumerate(seq):
        state.epoch([int(t)], alpha=alpha0, decay=decay)
        f = alg.step(int(t))
        err = rel_l2(_host(img), f)
        errs.append(err)
        assert err <= ITERATE_RTOL, f"step {k}: {err:.3e}"
    label = "bsrem" if (method == "sga" and decay > 0) else method
    record_error(test="non_vr_baseline", case=work.name, method=label, table="fp32", epochs=2,
                 one_step=errs[0], trajectory=errs[-1], trajectory_max=max(errs))
    assert _host(img).min() >= 0.0


@pytest.mark.parametrize("method", ["saga", "svrg"])
def test_iterate_preconditioner_updates(case, method):
    """SAGA and SVRG with d_t(f^k) = f^k / A_t^T 1 recomputed at every update
    (§4, Eq. (preconditioners)), against the oracle's same variant; then a
    switch back to the constant d(f^(0)) at an epoch boundary."""
    pv, prob, data, work, plan = case
    gp = _gpu_problem(pv, plan, data, work)
    f0 = prob.initial_image().astype(np.float32).astype(np.float64)
    img = _cuda(f0)
    state = pv.State(gp, method, img)
    state.set_preconditioner("iterate")
    alpha = 1.0
    alg = (em.SAGA(prob, f0, alpha, precond="iterate") if method == "saga"
           else em.SVRG(prob, f0, alpha, work.eta_svrg, precond="iterate"))
    seq = subset_sequence(4200, work.n_subsets, 2 * work.n_subsets)
    for k, t in enumerate(seq):
        state.epoch([int(t)], alpha=alpha, eta=work.eta_svrg)
        f = alg.step(int(t))
        err = rel_l2(_host(img), f)
        assert err <= ITERATE_RTOL, f"step {k}: {err:.3e}"
    # back to the constant preconditioner of the starting image for one epoch
    state.set_preconditioner("constant")
    alg.precond = "constant"
    state.epoch(seq[:work.n_subsets], alpha=alpha, eta=work.eta_svrg)
    for t in seq[:work.n_subsets]:
        f = alg.step(int(t))
    assert rel_l2(_host(img), f) <= ITERATE_RTOL
    assert _host(img).min() >= 0.0
    with pytest.raises(pv.PetError):
        pv.State(gp, "osem", _cuda(f0)).set_preconditioner("iterate")


def test_sagaem_updates(case, record_error):
    """SAGA on the EM statistic (§2.3 remark) against the oracle."""
    pv, prob, data, work, plan = case
    gp = _gpu_problem(pv, plan, data, work)
    f0 = prob.initial_image().astype(np.float32).astype(np.float64)
    img = _cuda(f0)
    state = pv.State(gp, "sagaem", img)
    alg = em.SAGAEM(prob, f0, 0.7)
    errs = []
    for k, t in enumerate(subset_sequence(4100, work.n_subsets, 2 * work.n_subsets)):
        state.epoch([int(t)], alpha=0.7)
        f = alg.step(int(t))
        err = rel_l2(_host(img), f)
        errs.append(err)
        assert err <= ITERATE_RTOL, f"step {k}: {err:.3e}"
    record_error(test="sagaem", case=work.name, method="sagaem", table="fp32", epochs=2,
                 one_step=errs[0], trajectory=errs[-1], trajectory_max=max(errs))
