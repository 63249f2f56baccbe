"""Continuous-batching server through the C ABI: requests that arrive while
others run share the batched kernels, each request's image is the same
served alone or in the mix, every request reaches the objective gap against
the FP64 oracle's Phi*, and admission respects the device-memory budget."""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.em import build_problem, map_reference
from paper_2106_03172_gb300.phantoms import Geometry, Workload, make_data

pytestmark = pytest.mark.gpu

TEMPLATES = [
    Workload("s0", Geometry(48, 48, 66, 69), n_subsets=6, counts=3e5, bg_frac=0.1, beta=0.005, n_ellipses=5,
             methods=("svrem",)),
    Workload("s1", Geometry(64, 64, 90, 91), n_subsets=12, counts=1e6, bg_frac=0.1, beta=0.005, n_ellipses=6,
             methods=("saga",)),
    Workload("s2", Geometry(48, 48, 66, 69), n_subsets=6, counts=2e6, bg_frac=0.1, beta=0.005, n_ellipses=5,
             methods=("saga",)),
    Workload("s3", Geometry(64, 64, 90, 91), n_subsets=12, counts=5e5, bg_frac=0.1, beta=0.005, n_ellipses=6,
             methods=("svrem",)),
]


@functools.lru_cache(maxsize=None)
def _template(i):
    work = TEMPLATES[i]
    data = make_data(work, 40 + i)
    prob = build_problem(work.geometry, data["g"], data["w"], work.n_subsets, work.beta)
    _, phi, _ = map_reference(prob)
    return work, data, phi


def _requests(arrivals):
    from paper_2106_03172_gb300.serving import Request
    out = []
    for rid, t in enumerate(arrivals):
        work, data, phi = _template(rid % len(TEMPLATES))
        out.append(Request(rid, work, data["g"], data["w"], phi, arrival=t, seed=900 + rid))
    return out


SERVERS = {"batch": lambda **kw: _srv("Server", tick=3, **kw),
           "batch-window4": lambda **kw: _srv("Server", tick=3, window=4, **kw),
           "streams": lambda **kw: _srv("StreamServer", depth=2, **kw)}


def _srv(kind, **kw):
    from paper_2106_03172_gb300 import serving
    return getattr(serving, kind)(**kw)


@pytest.mark.parametrize("kind", list(SERVERS))
def test_results_same_alone_and_in_the_mix(kind):
    """Served in a mix (one batch, with one or four ticks per host round
    trip, or one stream per request) a request returns what it returns
    served alone."""
    from paper_2106_03172_gb300.serving import Server, latency_summary
    arrivals = [0.0, 0.0005, 0.001, 0.0015, 0.002, 0.0025]
    mixed = SERVERS[kind](budget_bytes=1 << 34, max_epochs=40).serve(_requests(arrivals))
    summary = latency_summary(mixed)
    assert summary["completed"] == len(arrivals) and summary["reached_gap"] == len(arrivals)
    for r in mixed:
        alone = Server(budget_bytes=1 << 34, tick=3, max_epochs=40).serve(_requests(arrivals)[r.rid:r.rid + 1])[0]
        assert alone.epochs == r.epochs
        np.testing.assert_array_equal(alone.image, r.image)


def test_plain_path_gives_the_same_results():
    """The one-at-a-time per-reconstruction path (State epochs, captured
    graphs) and both servers agree bit for bit."""
    from paper_2106_03172_gb300.serving import serve_plain
    arrivals = [0.0, 0.0005, 0.001, 0.0015]
    plain = serve_plain(_requests(arrivals), max_epochs=40)
    for kind in ("batch-window4", "streams"):
        served = SERVERS[kind](budget_bytes=1 << 34, max_epochs=40).serve(_requests(arrivals))
        for a, b in zip(served, plain):
            assert a.epochs == b.epochs and a.reached and b.reached
            np.testing.assert_array_equal(a.image, b.image)


def test_pooled_slots_are_reused_without_changing_results():
    """Requests of one shape arriving one after another reuse the first
    one's slot (problem update, warm start, state reset: no allocation) and
    return what fresh slots return."""
    from paper_2106_03172_gb300.phantoms import make_data
    from paper_2106_03172_gb300.serving import Request, Server
    work, _, phi = _template(0)
    # one shape and method, different counts and backgrounds (noise seeds)
    datas = [make_data(work, 40 + k) for k in range(3)]

    def reqs():
        return [Request(k, work, d["g"], d["w"], phi, 0.0, seed=950 + k) for k, d in enumerate(datas)]

    for kind in ("batch", "streams"):
        srv = SERVERS[kind](budget_bytes=1 << 34, max_epochs=40)
        rs = reqs()
        done = srv.serve(rs[:1]) + srv.serve(rs[1:2]) + srv.serve(rs[2:])
        assert srv.stats.slots_reused == 2 and srv.stats.slots_created == 1
        for r, fresh_req in zip(done, reqs()):
            fresh = Server(budget_bytes=1 << 34, tick=3, max_epochs=40).serve([fresh_req])[0]
            assert fresh.epochs == r.epochs
            np.testing.assert_array_equal(fresh.image, r.image)


@pytest.mark.parametrize("kind", ["batch", "streams"])
def test_admission_respects_the_memory_budget(kind):
    from paper_2106_03172_gb300.serving import Server
    reqs = _requests([0.0] * 6)
    probe = Server(budget_bytes=1 << 40)
    need = max(probe.bytes_needed(r) for r in reqs)
    budget = 2 * need + need // 2
    srv = SERVERS[kind](budget_bytes=budget, max_epochs=40)
    done = srv.serve(reqs)
    assert all(np.isfinite(r.done) for r in done)
    assert srv.stats.peak_bytes <= budget and srv.stats.admissions_deferred > 0
    assert srv.stats.max_active < len(reqs)
    assert srv.active_bytes == 0 and not srv.active


@functools.lru_cache(maxsize=None)
def _distinct(k):
    """Request k of a stream whose every request has its own phantom and
    counts (log-uniform in [3e5, 3e6]) on the first template's shape and
    method, with the oracle's Phi* of its own data."""
    import dataclasses
    base = TEMPLATES[0]
    counts = float(10.0 ** np.random.default_rng(600 + k).uniform(np.log10(3e5), np.log10(3e6)))
    work = dataclasses.replace(base, name=f"d{k}", counts=counts)
    data = make_data(work, 700 + k)
    prob = build_problem(work.geometry, data["g"], data["w"], work.n_subsets, work.beta)
    _, phi, _ = map_reference(prob)
    return work, data, phi


@pytest.mark.parametrize("kind", ["batch", "streams"])
def test_distinct_requests_reach_their_own_gap(kind):
    """Requests that share only a shape (each its own phantom, counts and
    Phi*) all reach the 1e-4 gap against their own Phi* in the mix, reuse
    pooled slots across different data, and return what the plain path
    returns."""
    from paper_2106_03172_gb300.serving import Request, serve_plain

    def reqs():
        out = []
        for k, t in enumerate([0.0, 0.0005, 0.001, 0.0015, 0.002, 0.0025, 0.003, 0.0035]):
            work, data, phi = _distinct(k)
            out.append(Request(k, work, data["g"], data["w"], phi, arrival=t, seed=980 + k))
        return out

    srv = SERVERS[kind](budget_bytes=1 << 34, max_slots=3, max_epochs=60)
    done = srv.serve(reqs())
    assert all(r.reached and r.gap <= 1e-4 for r in done), [(r.rid, r.gap) for r in done]
    # at most three slots at a time, all of one key: every later request reuses one
    assert srv.stats.slots_created <= 3 and srv.stats.slots_reused == len(done) - srv.stats.slots_created
    for a, b in zip(done, serve_plain(reqs(), max_epochs=60)):
        assert a.epochs == b.epochs
        np.testing.assert_array_equal(a.image, b.image)


def test_native_loop_gives_the_plain_results():
    """serve_native (the library's arrival-gated host loop, pet_serve_jobs)
    returns, request by request, the epochs and images of the plain path,
    and starts no request before its arrival."""
    from paper_2106_03172_gb300.serving import Request, serve_native, serve_plain

    def reqs():
        out = []
        for k, t in enumerate([0.0, 0.0005, 0.001, 0.02, 0.021, 0.05]):
            work, data, phi = _template(k % len(TEMPLATES))
            out.append(Request(k, work, data["g"], data["w"], phi, arrival=t, seed=990 + k))
        return out

    native, stats = serve_native(reqs(), max_epochs=40, n_streams=3)
    plain = serve_plain(reqs(), max_epochs=40)
    for a, b in zip(native, plain):
        assert a.epochs == b.epochs and a.reached == b.reached
        np.testing.assert_array_equal(a.image, b.image)
        assert a.admitted >= a.arrival and a.done > a.admitted
    assert stats["slots_created"] + stats["slots_reused"] == len(native)


def test_native_loop_respects_the_memory_budget():
    """With a budget of two and a half of the largest slots the library's
    loop defers admissions, evicts pooled slots of other kinds to make room,
    never holds more than the budget, and still returns the plain path's
    results."""
    from paper_2106_03172_gb300 import petvr
    from paper_2106_03172_gb300.serving import Request, _table, serve_native, serve_plain

    def reqs():
        out = []
        for k in range(8):
            work, data, phi = _template(k % len(TEMPLATES))
            out.append(Request(k, work, data["g"], data["w"], phi, arrival=0.0, seed=970 + k))
        return out

    slot = 0
    for work in TEMPLATES:                     # a slot: problem, state, counts staging and image
        plan = petvr.Plan(work.geometry, work.n_subsets)
        algo = work.methods[0]
        slot = max(slot, petvr.pet_problem_bytes(plan.handle, False)
                   + petvr.pet_plan_state_bytes(plan.handle, algo, _table(algo))
                   + 4 * (work.geometry.n_rays + work.geometry.n_pixels))
    budget = int(2.5 * slot)
    native, stats = serve_native(reqs(), max_epochs=40, n_streams=4, budget_bytes=budget)
    assert stats["peak_bytes"] <= budget and stats["admissions_deferred"] > 0 and stats["slots_evicted"] > 0, stats
    for a, b in zip(native, serve_plain(reqs(), max_epochs=40)):
        assert a.epochs == b.epochs
        np.testing.assert_array_equal(a.image, b.image)
