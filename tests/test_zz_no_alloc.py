"""The allocation-free objective entry point, pet_objective_noalloc.

It exists for callers that cannot call cudaMalloc: code whose device memory
belongs to a framework or serving allocator that must account for every byte,
and code on a latency path that cannot take cudaMalloc's implicit device
synchronisation.  Its reduction scratch is a fixed array inside the library,
shared by all calls.  This file is collected last so that a failure here
cannot hide the result of any other test; it passes alone and after the rest.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from cases import oracle_problem

pytestmark = pytest.mark.gpu


def _pv():
    from paper_2106_03172_gb300 import petvr
    petvr.lib()
    return petvr


# Both entry points run the same full-data forward launch shape, so every
# ray's FP32 expected count and FP64 log-likelihood term are the same; they
# differ only in the order the FP64 block partials add those terms (rays in
# view order here, subset-major order in pet_objective).  That reordering
# moves an FP64 sum of n terms by at most about n * 2^-53 * sum|term|, far
# below 1e-12 of |Phi| at these sizes; the penalty sum is identical.
RTOL = 1e-12


@pytest.mark.parametrize("case", ["c64", "ragged", "stack"])
def test_noalloc_objective_matches_pet_objective(case):
    """Two calls in a row, on two different images, agree with pet_objective
    (the existing entry point) component by component, within RTOL."""
    pv = _pv()
    prob, data, work = oracle_problem(case)
    plan = pv.Plan(work.geometry, work.n_subsets)
    counts = torch.from_numpy(data["g"].ravel()).cuda()
    gp = pv.Problem(plan, counts, None, data["w"], work.beta)
    rng = np.random.default_rng(11)
    f0 = prob.initial_image()
    images = [f0, f0 * rng.uniform(0.5, 1.5, f0.shape)]
    out = torch.empty(2, 3, dtype=torch.float64, device="cuda")
    ref = torch.empty(2, 3, dtype=torch.float64, device="cuda")
    imgs = [torch.from_numpy(f.astype(np.float32).ravel()).cuda() for f in images]
    for i, img in enumerate(imgs):
        pv.pet_objective_noalloc(plan.handle, img, counts, None, data["w"], work.beta, out[i])
        pv.pet_objective_async(gp.handle, img, ref[i])
    torch.cuda.synchronize()
    got, want = out.cpu().numpy(), ref.cpu().numpy()
    assert got[0, 0] != got[1, 0]
    for i, img in enumerate(imgs):
        np.testing.assert_allclose(got[i], want[i], rtol=RTOL)
        assert got[i, 0] == pytest.approx(pv.pet_objective(gp.handle, img), rel=RTOL)


def test_noalloc_calls_leave_device_memory_unchanged():
    """After a first (set-up) call, further calls allocate nothing: the
    device's free memory is the same before and after three more calls, and
    torch's allocator was not asked for memory either."""
    pv = _pv()
    prob, data, work = oracle_problem("c64")
    plan = pv.Plan(work.geometry, work.n_subsets)
    counts = torch.from_numpy(data["g"].ravel()).cuda()
    img = torch.from_numpy(prob.initial_image().astype(np.float32).ravel()).cuda()
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    pv.pet_objective_noalloc(plan.handle, img, counts, None, data["w"], work.beta, out)
    torch.cuda.synchronize()
    free0, torch0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for _ in range(3):
        pv.pet_objective_noalloc(plan.handle, img, counts, None, data["w"], work.beta, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == torch0


def test_noalloc_nonpositive_mean_with_counts_gives_minus_infinity():
    """A zero image with no background gives yhat = 0 on every ray: with
    positive counts the log-likelihood is -inf, and the call says so in Phi
    and L (it has no status word); pet_objective also returns PET_ERR_NUMERIC."""
    pv = _pv()
    prob, data, work = oracle_problem("c64")
    plan = pv.Plan(work.geometry, work.n_subsets)
    counts = torch.from_numpy(data["g"].ravel()).cuda()
    zero = torch.zeros(prob.N, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    pv.pet_objective_noalloc(plan.handle, zero, counts, None, 0.0, work.beta, out)
    torch.cuda.synchronize()
    phi, L, R = out.cpu().numpy()
    assert phi == -np.inf and L == -np.inf and R == 0.0
    gp = pv.Problem(plan, counts, None, 0.0, work.beta)
    with pytest.raises(pv.PetError) as e:
        pv.pet_objective(gp.handle, zero)
    assert e.value.status == 5


def test_noalloc_rejects_sizes_beyond_its_scratch():
    pv = _pv()
    from paper_2106_03172_gb300.phantoms import Geometry
    geom = Geometry(1024, 1024, 1024, 4096)            # 4.2M rays: 262144 block partials at 16 chunks
    plan = pv.Plan(geom, 1)
    img = torch.ones(geom.n_pixels, device="cuda")
    counts = torch.ones(geom.n_rays, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(pv.PetError, match="too large for its fixed scratch") as e:
        pv.pet_objective_noalloc(plan.handle, img, counts, None, 0.1, 0.01, out)
    assert e.value.status == 1
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0


def test_noalloc_rejects_multi_ring_plans():
    pv = _pv()
    prob, data, work = oracle_problem("ring2")
    plan = pv.Plan(work.geometry, work.n_subsets)
    img = torch.ones(prob.N, device="cuda")
    counts = torch.ones(prob.M, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(pv.PetError, match="multi-ring"):
        pv.pet_objective_noalloc(plan.handle, img, counts, None, 0.1, 0.01, out)
