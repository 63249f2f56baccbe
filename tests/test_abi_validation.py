"""Argument checks of the C ABI that return before any CUDA call, exercised on
the CPU: each bad input is refused with PET_ERR_INVALID and a message from
pet_last_error, and nothing is created."""
import ctypes
from ctypes import byref, c_void_p

import pytest

from paper_2106_03172_gb300 import build, petvr
from paper_2106_03172_gb300.phantoms import Geometry

PET_ERR_INVALID = 1


@pytest.fixture(scope="module")
def lib():
    build.build()
    petvr._lib = None
    return petvr.lib()


def _create(lib, geom, n_subsets=1, scheme=0):
    g = petvr.pet_geometry(geom.nx, geom.ny, geom.nz, geom.pixel_mm, geom.n_angles, geom.n_bins,
                           geom.bin_mm if geom.bin_mm is not None else 0.0, geom.n_rings, geom.ring_mm,
                           geom.radius_mm, geom.slice_mm)
    h = c_void_p(12345)
    st = lib.pet_plan_create(byref(g), byref(petvr.pet_subsets(n_subsets, scheme)), byref(h))
    return st, h.value, lib.pet_last_error().decode()


@pytest.mark.parametrize("geom,n_subsets,scheme,needle", [
    (Geometry(0, 8, 4, 9), 1, 0, "sizes must be >= 1"),
    (Geometry(8, 8, 4, 9, nz=0), 1, 0, "sizes must be >= 1"),
    (Geometry(20000, 8, 4, 9), 1, 0, "<= 16384"),
    (Geometry(8, 8, 2000, 9), 1, 0, "n_angles must be <= 1024"),
    (Geometry(8, 8, 4, 9, pixel_mm=0.0), 1, 0, "pixel_mm"),
    (Geometry(8, 8, 4, 9, pixel_mm=float("nan")), 1, 0, "pixel_mm"),
    (Geometry(8, 8, 4, 9), 5, 0, "n_subsets <= n_angles"),
    (Geometry(8, 8, 4, 9), 0, 0, "n_subsets <= n_angles"),
    (Geometry(8, 8, 4, 9), 2, 1, "subset scheme"),
    (Geometry(8, 8, 4, 9, nz=2, n_rings=5, ring_mm=4.0, radius_mm=40.0, slice_mm=2.0), 1, 0, "n_rings"),
    (Geometry(8, 8, 4, 9, nz=2, n_rings=2, ring_mm=4.0, radius_mm=40.0, slice_mm=0.0), 1, 0, "slice_mm"),
    (Geometry(8, 8, 4, 9, nz=2, n_rings=2, ring_mm=-1.0, radius_mm=40.0, slice_mm=2.0), 1, 0, "ring_mm"),
    (Geometry(8, 8, 4, 9, nz=2, n_rings=2, ring_mm=4.0, radius_mm=5.0, slice_mm=2.0), 1, 0, "radius_mm"),
    (Geometry(16384, 16384, 4, 9, nz=16), 1, 0, "2^31"),
    (Geometry(8, 8, 1024, 16384, nz=256), 1, 0, "2^31"),
])
def test_plan_create_refuses_bad_geometry(lib, geom, n_subsets, scheme, needle):
    st, handle, msg = _create(lib, geom, n_subsets, scheme)
    assert st == PET_ERR_INVALID
    assert handle is None                       # *out is cleared before any check that can fail
    assert needle in msg, msg


def test_null_arguments_are_refused(lib):
    assert lib.pet_plan_create(None, None, None) == PET_ERR_INVALID
    assert "null" in lib.pet_last_error().decode()
    g = petvr.pet_geometry(8, 8, 1, 2.0, 4, 9, 0.0, 0, 0.0, 0.0, 0.0)
    assert lib.pet_plan_create(byref(g), None, byref(c_void_p())) == PET_ERR_INVALID


def test_destroy_accepts_null(lib):
    """Destroying nothing is a no-op (the create calls above left no object)."""
    for name in ("pet_plan_destroy", "pet_problem_destroy", "pet_state_destroy", "pet_batch_destroy"):
        fn = getattr(lib, name)
        fn(None)


def test_every_entry_point_refuses_null_handles(lib):
    """Every status-returning call given null handles and pointers (zeros for
    the scalars) returns PET_ERR_INVALID instead of touching memory."""
    from ctypes import c_double, c_float, c_int32, c_int64, c_size_t
    skip = {"pet_state_destroy", "pet_batch_destroy",      # null is a no-op by contract
            "pet_profile_enable", "pet_profile_reset"}     # no handle to check
    zero = {c_int32: 0, c_int64: 0, c_size_t: 0, c_float: 0.0, c_double: 0.0}
    checked = 0
    for name, (res, args) in petvr._SIGS.items():
        if res is not c_int32 or not args or name in skip:
            continue
        vals = [zero.get(t, None) for t in args]
        st = getattr(lib, name)(*vals)
        assert st == PET_ERR_INVALID, f"{name} -> {st}: {lib.pet_last_error().decode()}"
        checked += 1
    assert checked >= 35


def test_noalloc_objective_refuses_bad_arguments(lib):
    """pet_objective_noalloc checks its pointers, beta and background before it
    reads the plan or makes any CUDA call; the stand-in handles below are never
    dereferenced."""
    import math
    from ctypes import c_float
    fake = [c_void_p(0x1000), c_void_p(0x2000), c_void_p(0x3000), c_void_p(0x4000)]   # plan, img, counts, phi
    fn = lib.pet_objective_noalloc

    def call(plan, img, counts, phi, bg=0.1, beta=0.01):
        st = fn(plan, img, counts, None, c_float(bg), c_float(beta), phi, None)
        return st, lib.pet_last_error().decode()

    for k in range(4):                       # each pointer null in turn
        args = list(fake)
        args[k] = None
        st, msg = call(*args)
        assert st == PET_ERR_INVALID and "null" in msg, (k, msg)
    for beta in (-1.0, math.nan, math.inf):
        st, msg = call(*fake, beta=beta)
        assert st == PET_ERR_INVALID and "beta" in msg, (beta, msg)
    for bg in (math.nan, math.inf, -math.inf):
        st, msg = call(*fake, bg=bg)
        assert st == PET_ERR_INVALID and "background" in msg, (bg, msg)


def test_state_run_refuses_bad_objective_arguments(lib):
    """pet_state_run checks objective_every and d_phi before it reads the
    state; the stand-in handle below is never dereferenced."""
    from ctypes import c_float
    fake = c_void_p(0x1000)
    seq = (ctypes.c_int32 * 2)(0, 0)
    for every, phi, needle in ((-1, c_void_p(0x2000), "objective_every"), (3, None, "d_phi")):
        st = lib.pet_state_run(fake, seq, 2, c_float(1.0), c_float(0.0), 1, every, phi, None)
        assert st == PET_ERR_INVALID and needle in lib.pet_last_error().decode()


def test_executor_refuses_bad_arguments_before_reading_states(lib):
    """pet_run_to_gap's argument checks that come before it reads any worker
    state (the stand-in handle below is never dereferenced)."""
    from ctypes import c_double, c_float, c_int32
    w = (c_void_p * 1)(0x1000)
    seq = (c_int32 * 4)(0, 0, 0, 0)
    ep = (c_int32 * 1)()
    gp = (c_double * 1)()
    ms = (c_double * 1)()

    def call(workers=w, n_workers=1, n_jobs=1, seqs=seq, max_epochs=2, phi_star=1.0, gap=1e-4, outs=True):
        o = (ep, gp, ms) if outs else (None, None, None)
        st = lib.pet_run_to_gap(workers, n_workers, n_jobs, seqs, max_epochs, c_float(1.0), c_float(0.0), 1,
                                c_double(phi_star), c_double(gap), None, *o, None)
        return st, lib.pet_last_error().decode()

    for kw, needle in (({"workers": None}, "worker"), ({"n_workers": 0}, "worker"), ({"n_jobs": -1}, "n_jobs"),
                       ({"max_epochs": 0}, "max_epochs"), ({"seqs": None}, "null"), ({"outs": False}, "null"),
                       ({"phi_star": 0.0}, "phi_star"), ({"phi_star": float("nan")}, "phi_star"),
                       ({"gap": -1.0}, "gap"), ({"gap": float("inf")}, "gap")):
        st, msg = call(**kw)
        assert st == PET_ERR_INVALID and needle in msg, (kw, msg)


def test_jobs_executor_refuses_bad_arguments_before_reading_states(lib):
    """pet_run_jobs_to_gap's checks before it reads any state."""
    from ctypes import c_double, c_float, c_int32
    st = (c_void_p * 1)(0x1000)
    sq = (c_void_p * 1)(0x2000)
    a = (c_float * 1)(1.0)
    d = (c_float * 1)(0.0)
    e = (c_int32 * 1)(1)
    ps = (c_double * 1)(1.0)
    outs = ((c_int32 * 1)(), (c_double * 1)(), (c_double * 1)())

    def call(states=st, seqs=sq, n_jobs=1, n_streams=2, max_epochs=2, gap=1e-4, alpha=a, phi=ps):
        r = lib.pet_run_jobs_to_gap(states, seqs, alpha, d, e, phi, n_jobs, n_streams, max_epochs, c_double(gap),
                                    *outs, None)
        return r, lib.pet_last_error().decode()

    for kw, needle in (({"states": None}, "null"), ({"seqs": None}, "null"), ({"alpha": None}, "null"),
                       ({"phi": None}, "null"), ({"n_jobs": -1}, "n_jobs"), ({"n_streams": 0}, "n_streams"),
                       ({"max_epochs": 0}, "max_epochs"), ({"gap": float("nan")}, "gap")):
        r, msg = call(**kw)
        assert r == PET_ERR_INVALID and needle in msg, (kw, msg)


def test_serve_requests_refuses_bad_arguments_before_any_cuda_call(lib):
    """pet_serve_requests's checks on the call's own arguments and on each
    request's host fields (the stand-in plan is read only for its subset
    number after these checks, so it is never reached here)."""
    from ctypes import c_double, c_int32, c_size_t
    req = (petvr.pet_request * 1)()
    seq = (c_int32 * 4)(0, 0, 0, 0)
    counts = (ctypes.c_float * 4)()
    req[0].plan, req[0].h_counts, req[0].h_seq = 0x1000, ctypes.addressof(counts), ctypes.addressof(seq)
    req[0].phi_star, req[0].arrival_s, req[0].algo = 1.0, 0.0, 0
    outs = ((c_int32 * 1)(), (c_double * 1)(), (c_double * 1)(), (c_double * 1)())
    st = petvr.pet_serve_stats()

    def call(reqs=req, n=1, n_streams=2, max_epochs=2, stats=True):
        r = lib.pet_serve_requests(reqs, n, n_streams, c_size_t(1 << 20), max_epochs, c_double(1e-4), *outs,
                                   byref(st) if stats else None, None)
        return r, lib.pet_last_error().decode()

    for kw, needle in (({"reqs": None}, "null"), ({"n": -1}, "n_jobs"), ({"n_streams": 0}, "n_streams"),
                       ({"max_epochs": 0}, "max_epochs"), ({"stats": False}, "null")):
        r, msg = call(**kw)
        assert r == PET_ERR_INVALID and needle in msg, (kw, msg)
    for field, value, needle in (("algo", 9, "algorithm"), ("table_dtype", 5, "table"), ("bg", float("nan"), "background"),
                                 ("phi_star", 0.0, "phi_star"), ("arrival_s", -1.0, "arrival")):
        old = getattr(req[0], field)
        setattr(req[0], field, value)
        r, msg = call()
        setattr(req[0], field, old)
        assert r == PET_ERR_INVALID and needle in msg, (field, msg)
