"""Python binding of libpetvr (include/petvr.h): argument marshalling only.

Every function named ``pet_*`` here calls the C entry point of the same name
with device pointers taken from CUDA torch tensors and the current torch
stream; every step of the reconstruction runs in the library's kernels.  The
binding raises ``PetError`` on a nonzero status and refuses to run if the
compiled library is missing: there is no fallback path.

The small classes ``Plan``, ``Problem`` and ``State`` own the C handles and
release them when garbage collected.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_double, c_float, c_int32, c_size_t, c_uint64, c_void_p

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpetvr.so")

ALGO = {"osem": 0, "svrem": 1, "saga": 2, "svrg": 3, "sga": 4, "sem": 5, "sagaem": 6}
TABLE = {"fp32": 0, "bf16": 1}
PRECOND = {"constant": 0, "iterate": 1}
STATUS = {0: "PET_OK", 1: "PET_ERR_INVALID", 2: "PET_ERR_OOM", 3: "PET_ERR_CUDA",
          4: "PET_ERR_TIMEOUT", 5: "PET_ERR_NUMERIC", 6: "PET_ERR_STATE"}


class PetError(RuntimeError):
    def __init__(self, func, status, msg):
        super().__init__(f"{func} -> {STATUS.get(status, status)}: {msg}")
        self.status = status


class pet_geometry(ctypes.Structure):
    _fields_ = [("nx", c_int32), ("ny", c_int32), ("nz", c_int32), ("pixel_mm", c_double),
                ("n_angles", c_int32), ("n_bins", c_int32), ("bin_mm", c_double),
                ("n_rings", c_int32), ("ring_mm", c_double), ("radius_mm", c_double), ("slice_mm", c_double)]


class pet_subsets(ctypes.Structure):
    _fields_ = [("n_subsets", c_int32), ("scheme", c_int32)]


class pet_penalty(ctypes.Structure):
    _fields_ = [("potential", c_int32), ("beta", c_float), ("delta", c_float)]


class pet_request(ctypes.Structure):
    _fields_ = [("plan", c_void_p), ("h_counts", c_void_p), ("bg", c_float), ("penalty", pet_penalty),
                ("algo", c_int32), ("table_dtype", c_int32), ("h_seq", c_void_p), ("alpha", c_float),
                ("decay", c_float), ("eta", c_int32), ("phi_star", c_double), ("arrival_s", c_double),
                ("h_image", c_void_p)]


class pet_serve_stats(ctypes.Structure):
    _fields_ = [("peak_bytes", c_size_t), ("slots_created", c_int32), ("slots_reused", c_int32),
                ("slots_evicted", c_int32), ("admissions_deferred", c_int32)]


_SIGS = {
    "pet_plan_create": (c_int32, [POINTER(pet_geometry), POINTER(pet_subsets), POINTER(c_void_p)]),
    "pet_plan_destroy": (None, [c_void_p]),
    "pet_plan_subset_views": (c_int32, [c_void_p, c_int32, POINTER(c_int32)]),
    "pet_plan_sensitivity": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p]),
    "pet_plan_nnz": (c_int32, [c_void_p, c_int32, POINTER(ctypes.c_int64)]),
    "pet_plan_set_tuning": (c_int32, [c_void_p, c_int32, c_int32]),
    "pet_plan_get_tuning": (c_int32, [c_void_p, POINTER(c_int32), POINTER(c_int32)]),
    "pet_plan_autotune": (c_int32, [c_void_p, POINTER(c_int32), POINTER(c_int32)]),
    "pet_forward": (c_int32, [c_void_p, c_void_p, c_void_p, c_float, c_int32, c_void_p, c_void_p]),
    "pet_back": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    "pet_problem_create": (c_int32, [c_void_p, c_void_p, c_void_p, c_float, POINTER(pet_penalty),
                                     POINTER(c_void_p), c_void_p]),
    "pet_problem_destroy": (None, [c_void_p]),
    "pet_problem_update": (c_int32, [c_void_p, c_void_p, c_void_p, c_float, c_void_p]),
    "pet_profile_enable": (c_int32, [c_int32]),
    "pet_profile_reset": (c_int32, []),
    "pet_profile_read": (c_int32, [c_int32, POINTER(ctypes.c_int64), POINTER(c_double)]),
    "pet_warm_start": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "pet_objective": (c_int32, [c_void_p, c_void_p, POINTER(c_double), c_void_p]),
    "pet_objective_async": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "pet_batch_set_mode": (c_int32, [c_void_p, c_int32]),
    "pet_batch_set_wait_limit": (c_int32, [c_void_p, ctypes.c_int64]),
    "pet_batch_sync": (c_int32, [c_void_p, c_void_p]),
    "pet_objective_noalloc": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_float, c_float, c_void_p,
                                        c_void_p]),
    "pet_state_create": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, POINTER(c_size_t),
                                   POINTER(c_void_p), c_void_p]),
    "pet_state_destroy": (c_int32, [c_void_p]),
    "pet_state_reset": (c_int32, [c_void_p, c_void_p]),
    "pet_state_set_preconditioner": (c_int32, [c_void_p, c_int32]),
    "pet_batch_create": (c_int32, [POINTER(c_void_p), c_int32, POINTER(c_void_p)]),
    "pet_batch_destroy": (c_int32, [c_void_p]),
    "pet_batch_set_graphs": (c_int32, [c_void_p, c_int32]),
    "pet_plan_bytes": (c_int32, [c_void_p, POINTER(c_size_t)]),
    "pet_problem_bytes": (c_int32, [c_void_p, c_int32, POINTER(c_size_t)]),
    "pet_plan_state_bytes": (c_int32, [c_void_p, c_int32, c_int32, POINTER(c_size_t)]),
    "pet_batch_epoch": (c_int32, [c_void_p, c_void_p, c_int32, POINTER(c_float), POINTER(c_int32), c_void_p]),
    "pet_batch_objective_async": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "pet_osem_epoch": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p]),
    "pet_svrem_epoch": (c_int32, [c_void_p, c_float, c_int32, c_void_p, c_int32, c_void_p]),
    "pet_saga_epoch": (c_int32, [c_void_p, c_float, c_void_p, c_int32, c_void_p]),
    "pet_svrg_epoch": (c_int32, [c_void_p, c_float, c_int32, c_void_p, c_int32, c_void_p]),
    "pet_sga_epoch": (c_int32, [c_void_p, c_float, c_float, c_void_p, c_int32, c_void_p]),
    "pet_sem_epoch": (c_int32, [c_void_p, c_float, c_float, c_void_p, c_int32, c_void_p]),
    "pet_sagaem_epoch": (c_int32, [c_void_p, c_float, c_void_p, c_int32, c_void_p]),
    "pet_state_sync": (c_int32, [c_void_p, c_void_p]),
    "pet_state_objective_async": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "pet_state_run": (c_int32, [c_void_p, c_void_p, c_int32, c_float, c_float, c_int32, c_int32, c_void_p,
                                c_void_p]),
    "pet_run_to_gap": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_int32, c_float, c_float, c_int32,
                                 c_double, c_double, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "pet_run_jobs_to_gap": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int32,
                                      c_int32, c_double, c_void_p, c_void_p, c_void_p, c_void_p]),
    "pet_serve_jobs": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int32,
                                 c_int32, c_int32, c_double, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "pet_serve_requests": (c_int32, [c_void_p, c_int32, c_int32, c_size_t, c_int32, c_double, c_void_p, c_void_p,
                                     c_void_p, c_void_p, c_void_p, c_void_p]),
    "pet_kernel_launches": (c_uint64, []),
    "pet_last_error": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """Load libpetvr.so (after torch has loaded the CUDA runtime)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(handle, name)
            fn.restype, fn.argtypes = res, args
        _lib = handle
    return _lib


def _call(name, *args):
    st = getattr(lib(), name)(*args)
    if st != 0:
        raise PetError(name, st, lib().pet_last_error().decode())


def _dev(t: torch.Tensor | None, dtype=torch.float32):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"expected a contiguous CUDA {dtype} tensor, got {t.dtype} on {t.device}")
    return c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return c_void_p(s.cuda_stream)


def _seq(seq):
    arr = (c_int32 * max(1, len(seq)))(*[int(x) for x in seq])
    return arr, len(seq)


# ---- thin wrappers with the C names ---------------------------------------------

def pet_plan_create(geom, n_subsets: int) -> c_void_p:
    g = pet_geometry(geom.nx, geom.ny, geom.nz, geom.pixel_mm, geom.n_angles, geom.n_bins,
                     geom.bin_mm if geom.bin_mm is not None else 0.0,
                     getattr(geom, "n_rings", 0), getattr(geom, "ring_mm", 0.0),
                     getattr(geom, "radius_mm", 0.0), getattr(geom, "slice_mm", 0.0))
    h = c_void_p()
    _call("pet_plan_create", byref(g), byref(pet_subsets(n_subsets, 0)), byref(h))
    return h


def pet_plan_subset_views(plan, t: int) -> int:
    n = c_int32()
    _call("pet_plan_subset_views", plan, t, byref(n))
    return n.value


def pet_plan_nnz(plan, t: int) -> int:
    n = ctypes.c_int64()
    _call("pet_plan_nnz", plan, t, byref(n))
    return n.value


def pet_plan_set_tuning(plan, fwd_chunks: int, back_run: int):
    _call("pet_plan_set_tuning", plan, fwd_chunks, back_run)


def pet_plan_get_tuning(plan):
    c, r = c_int32(), c_int32()
    _call("pet_plan_get_tuning", plan, byref(c), byref(r))
    return c.value, r.value


def pet_plan_autotune(plan):
    """Time the launch shapes on this plan and keep the fastest; returns (chunks, run)."""
    c, r = c_int32(), c_int32()
    _call("pet_plan_autotune", plan, byref(c), byref(r))
    return c.value, r.value


def pet_plan_sensitivity(plan, t: int, out: torch.Tensor, stream=None):
    _call("pet_plan_sensitivity", plan, t, _dev(out), _stream(stream))


def pet_forward(plan, img, bg, bg_scalar: float, subset: int, sino, stream=None):
    _call("pet_forward", plan, _dev(img), _dev(bg), bg_scalar, subset, _dev(sino), _stream(stream))


def pet_back(plan, sino, subset: int, img, stream=None):
    _call("pet_back", plan, _dev(sino), subset, _dev(img), _stream(stream))


POTENTIAL = {"quadratic": 0, "huber": 1, "logcosh": 2, "hyperbola": 3}


def pet_problem_create(plan, counts, bg, bg_scalar: float, beta: float, stream=None,
                       potential: str = "quadratic", delta: float = 1.0) -> c_void_p:
    h = c_void_p()
    _call("pet_problem_create", plan, _dev(counts), _dev(bg), bg_scalar,
          byref(pet_penalty(POTENTIAL[potential], beta, delta)), byref(h), _stream(stream))
    return h


def pet_problem_update(problem, counts, bg, bg_scalar: float, stream=None):
    _call("pet_problem_update", problem, _dev(counts), _dev(bg), bg_scalar, _stream(stream))


def pet_profile_enable(on: bool):
    _call("pet_profile_enable", 1 if on else 0)


def pet_profile_reset():
    _call("pet_profile_reset")


def pet_profile_read(kind: int):
    """(launches, total ms) of kernel kind 0 forward, 1 back+update, 2 multi-subset back."""
    n, ms = ctypes.c_int64(), c_double()
    _call("pet_profile_read", kind, byref(n), byref(ms))
    return n.value, ms.value


def pet_warm_start(problem, img, stream=None):
    _call("pet_warm_start", problem, _dev(img), _stream(stream))


def pet_objective(problem, img, stream=None) -> float:
    phi = c_double()
    _call("pet_objective", problem, _dev(img), byref(phi), _stream(stream))
    return phi.value


def pet_objective_async(problem, img, phi_out: torch.Tensor, stream=None):
    """Enqueue Phi, L, R of ``img`` into the float64 CUDA tensor ``phi_out`` (3 values)."""
    _call("pet_objective_async", problem, _dev(img), _dev(phi_out, torch.float64), _stream(stream))


def pet_objective_noalloc(plan, img, counts, bg, bg_scalar: float, beta: float, phi_out: torch.Tensor,
                          stream=None):
    """Objective into ``phi_out`` (3 float64) with no device allocation; see
    the C declaration for who needs this and its fixed-scratch limits."""
    _call("pet_objective_noalloc", plan, _dev(img), _dev(counts), _dev(bg), bg_scalar, beta,
          _dev(phi_out, torch.float64), _stream(stream))


def pet_state_bytes(problem, algo: str, table: str = "fp32") -> int:
    n = c_size_t()
    _call("pet_state_create", problem, ALGO[algo], TABLE[table], None, byref(n), None, None)
    return n.value


def pet_state_create(problem, algo: str, table: str, img, stream=None) -> c_void_p:
    h = c_void_p()
    n = c_size_t()
    _call("pet_state_create", problem, ALGO[algo], TABLE[table], _dev(img), byref(n), byref(h),
          _stream(stream))
    return h


def pet_state_reset(state, stream=None):
    _call("pet_state_reset", state, _stream(stream))


def pet_state_set_preconditioner(state, kind: str):
    """``"constant"``: d = N_s f^(0) / A^T 1; ``"iterate"``: d_t(f^k) = f^k / A_t^T 1."""
    _call("pet_state_set_preconditioner", state, PRECOND[kind])


def pet_osem_epoch(state, seq, stream=None):
    arr, n = _seq(seq)
    _call("pet_osem_epoch", state, arr, n, _stream(stream))


def pet_svrem_epoch(state, alpha: float, eta: int, seq, stream=None):
    arr, n = _seq(seq)
    _call("pet_svrem_epoch", state, alpha, eta, arr, n, _stream(stream))


def pet_saga_epoch(state, alpha: float, seq, stream=None):
    arr, n = _seq(seq)
    _call("pet_saga_epoch", state, alpha, arr, n, _stream(stream))


def pet_svrg_epoch(state, alpha: float, eta: int, seq, stream=None):
    arr, n = _seq(seq)
    _call("pet_svrg_epoch", state, alpha, eta, arr, n, _stream(stream))


def pet_sga_epoch(state, alpha0: float, decay: float, seq, stream=None):
    arr, n = _seq(seq)
    _call("pet_sga_epoch", state, alpha0, decay, arr, n, _stream(stream))


def pet_sem_epoch(state, alpha0: float, decay: float, seq, stream=None):
    arr, n = _seq(seq)
    _call("pet_sem_epoch", state, alpha0, decay, arr, n, _stream(stream))


def pet_sagaem_epoch(state, alpha: float, seq, stream=None):
    arr, n = _seq(seq)
    _call("pet_sagaem_epoch", state, alpha, arr, n, _stream(stream))


def pet_state_run(state, seq, alpha: float = 1.0, decay: float = 0.0, eta: int = 1, objective_every: int = 0,
                  phi_out: torch.Tensor | None = None, stream=None):
    """n_iter updates of the state's algorithm with the objective after every
    ``objective_every``-th update into ``phi_out`` (float64, 3 per point)."""
    arr, n = _seq(seq)
    if objective_every > 0 and (phi_out is None or phi_out.numel() < 3 * (n // objective_every)):
        raise ValueError("phi_out needs 3 float64 per objective point")
    _call("pet_state_run", state, arr, n, alpha, decay, eta, objective_every,
          _dev(phi_out, torch.float64), _stream(stream))


def pet_run_to_gap(workers, seqs, max_epochs: int, phi_star: float, gap: float = 1e-4, alpha: float = 1.0,
                   decay: float = 0.0, eta: int = 1, results: torch.Tensor | None = None, stream=None):
    """Run len(seqs) reconstructions to the gap on the worker States (see the
    C header).  ``seqs``: int32 array [jobs, max_epochs * N_s].  Returns
    (epochs, gap, ms) numpy arrays, one entry per job."""
    import numpy as np
    q = np.ascontiguousarray(seqs, dtype=np.int32)
    n_jobs = q.shape[0] if q.ndim == 2 else 0
    arr = (c_void_p * max(1, len(workers)))(*[w.handle for w in workers])
    epochs = np.zeros(max(1, n_jobs), dtype=np.int32)
    gaps = np.zeros(max(1, n_jobs), dtype=np.float64)
    ms = np.zeros(max(1, n_jobs), dtype=np.float64)
    _call("pet_run_to_gap", arr, len(workers), n_jobs, c_void_p(q.ctypes.data) if n_jobs else None, max_epochs,
          alpha, decay, eta, phi_star, gap, _dev(results), c_void_p(epochs.ctypes.data), c_void_p(gaps.ctypes.data),
          c_void_p(ms.ctypes.data), _stream(stream))
    return epochs[:n_jobs], gaps[:n_jobs], ms[:n_jobs]


def pet_run_jobs_to_gap(states, seqs, alphas, etas, phi_stars, max_epochs: int, gap: float = 1e-4,
                        decays=None, n_streams: int = 8, stream=None):
    """Run job j on States[j] to the gap (see the C header).  ``seqs[j]``:
    max_epochs * N_s indices of that state's plan.  Returns (epochs, gap, ms)."""
    import numpy as np
    n = len(states)
    qs = [np.ascontiguousarray(q, dtype=np.int32) for q in seqs]
    h_states = (c_void_p * max(1, n))(*[st.handle for st in states])
    h_seqs = (c_void_p * max(1, n))(*[q.ctypes.data for q in qs])
    a = np.ascontiguousarray(alphas, dtype=np.float32)
    d = np.ascontiguousarray(decays if decays is not None else [0.0] * n, dtype=np.float32)
    e = np.ascontiguousarray(etas, dtype=np.int32)
    ps = np.ascontiguousarray(phi_stars, dtype=np.float64)
    epochs = np.zeros(max(1, n), dtype=np.int32)
    gaps = np.zeros(max(1, n), dtype=np.float64)
    ms = np.zeros(max(1, n), dtype=np.float64)
    ptr = lambda x: c_void_p(x.ctypes.data)   # noqa: E731
    _call("pet_run_jobs_to_gap", h_states, h_seqs, ptr(a), ptr(d), ptr(e), ptr(ps), n, n_streams, max_epochs, gap,
          ptr(epochs), ptr(gaps), ptr(ms), _stream(stream))
    return epochs[:n], gaps[:n], ms[:n]


def pet_serve_jobs(states, seqs, alphas, etas, phi_stars, arrivals_s, max_epochs: int, gap: float = 1e-4,
                   decays=None, n_streams: int = 8, stream=None):
    """Jobs that arrive over time (see the C header).  Returns (epochs, gap,
    start_ms, done_ms), times in milliseconds since the call."""
    import numpy as np
    n = len(states)
    qs = [np.ascontiguousarray(q, dtype=np.int32) for q in seqs]
    h_states = (c_void_p * max(1, n))(*[st.handle for st in states])
    h_seqs = (c_void_p * max(1, n))(*[q.ctypes.data for q in qs])
    a = np.ascontiguousarray(alphas, dtype=np.float32)
    d = np.ascontiguousarray(decays if decays is not None else [0.0] * n, dtype=np.float32)
    e = np.ascontiguousarray(etas, dtype=np.int32)
    ps = np.ascontiguousarray(phi_stars, dtype=np.float64)
    arr = np.ascontiguousarray(arrivals_s, dtype=np.float64)
    epochs = np.zeros(max(1, n), dtype=np.int32)
    gaps = np.zeros(max(1, n), dtype=np.float64)
    t_start = np.zeros(max(1, n), dtype=np.float64)
    t_done = np.zeros(max(1, n), dtype=np.float64)
    ptr = lambda x: c_void_p(x.ctypes.data)   # noqa: E731
    _call("pet_serve_jobs", h_states, h_seqs, ptr(a), ptr(d), ptr(e), ptr(ps), ptr(arr), n, n_streams, max_epochs,
          gap, ptr(epochs), ptr(gaps), ptr(t_start), ptr(t_done), _stream(stream))
    return epochs[:n], gaps[:n], t_start[:n], t_done[:n]


def pet_serve_requests(requests, n_streams: int, budget_bytes: int, max_epochs: int, gap: float = 1e-4,
                       stream=None):
    """Serve a request stream with admission by a device-memory budget (see
    the C header).  ``requests``: dicts with plan (Plan), counts (float32
    array), bg, beta, potential, delta, algo, table, seq (int array), alpha,
    decay, eta, phi_star, arrival_s.  Returns (epochs, gap, start_ms, done_ms,
    images, stats dict)."""
    import numpy as np
    n = len(requests)
    keep = []
    arr = (pet_request * max(1, n))()
    images = []
    for i, r in enumerate(requests):
        counts = np.ascontiguousarray(r["counts"], dtype=np.float32).ravel()
        seq = np.ascontiguousarray(r["seq"], dtype=np.int32)
        img = np.zeros(r["n_image"], dtype=np.float32)
        keep += [counts, seq]
        images.append(img)
        arr[i] = pet_request(r["plan"].handle.value, counts.ctypes.data, r["bg"],
                             pet_penalty(POTENTIAL[r.get("potential", "quadratic")], r["beta"], r.get("delta", 1.0)),
                             ALGO[r["algo"]], TABLE[r.get("table", "fp32")], seq.ctypes.data, r.get("alpha", 1.0),
                             r.get("decay", 0.0), r.get("eta", 1), r["phi_star"], r["arrival_s"], img.ctypes.data)
    epochs = np.zeros(max(1, n), dtype=np.int32)
    gaps = np.zeros(max(1, n), dtype=np.float64)
    t_start = np.zeros(max(1, n), dtype=np.float64)
    t_done = np.zeros(max(1, n), dtype=np.float64)
    st = pet_serve_stats()
    ptr = lambda x: c_void_p(x.ctypes.data)   # noqa: E731
    _call("pet_serve_requests", arr, n, n_streams, budget_bytes, max_epochs, gap, ptr(epochs), ptr(gaps),
          ptr(t_start), ptr(t_done), byref(st), _stream(stream))
    stats = {k: getattr(st, k) for k, _ in pet_serve_stats._fields_}
    return epochs[:n], gaps[:n], t_start[:n], t_done[:n], images, stats


def pet_state_objective_async(state, phi_out: torch.Tensor, stream=None):
    """Enqueue Phi, L, R of the state's current image into ``phi_out`` (3 float64)."""
    _call("pet_state_objective_async", state, _dev(phi_out, torch.float64), _stream(stream))


def pet_state_sync(state, stream=None):
    _call("pet_state_sync", state, _stream(stream))


def pet_kernel_launches() -> int:
    return int(lib().pet_kernel_launches())


def pet_batch_create(states) -> c_void_p:
    arr = (c_void_p * len(states))(*[st.value if isinstance(st, c_void_p) else st for st in states])
    h = c_void_p()
    _call("pet_batch_create", arr, len(states), byref(h))
    return h


def pet_batch_set_graphs(batch, on: bool):
    _call("pet_batch_set_graphs", batch, 1 if on else 0)


def pet_plan_bytes(plan) -> int:
    n = c_size_t()
    _call("pet_plan_bytes", plan, byref(n))
    return n.value


def pet_problem_bytes(plan, has_bg: bool = False) -> int:
    n = c_size_t()
    _call("pet_problem_bytes", plan, 1 if has_bg else 0, byref(n))
    return n.value


def pet_plan_state_bytes(plan, algo: str, table: str = "fp32") -> int:
    n = c_size_t()
    _call("pet_plan_state_bytes", plan, ALGO[algo], TABLE[table], byref(n))
    return n.value


def pet_batch_epoch(batch, seqs, alphas, etas, stream=None):
    """seqs: one equal-length subset sequence per member."""
    n = len(seqs)
    n_iter = len(seqs[0]) if n else 0
    if any(len(q) != n_iter for q in seqs):
        raise ValueError("every member needs a sequence of the same length")
    flat = (c_int32 * max(1, n * n_iter))(*[int(x) for q in seqs for x in q])
    al = (c_float * n)(*[float(x) for x in alphas])
    et = (c_int32 * n)(*[int(x) for x in etas])
    _call("pet_batch_epoch", batch, flat, n_iter, al, et, _stream(stream))


def pet_batch_objective_async(batch, phi_out: torch.Tensor, stream=None):
    _call("pet_batch_objective_async", batch, _dev(phi_out, torch.float64), _stream(stream))


# ---- owning handles ------------------------------------------------------------

class Plan:
    """Geometry tables and sensitivities on the current CUDA device."""

    def __init__(self, geom, n_subsets: int):
        self.geom, self.n_subsets = geom, n_subsets
        self.handle = pet_plan_create(geom, n_subsets)
        self.subset_views = [pet_plan_subset_views(self.handle, t) for t in range(n_subsets)]

    def subset_rays(self, t: int) -> int:
        return self.subset_views[t] * self.geom.n_bins

    def subset_lines(self, t: int) -> int:
        """Sinogram entries of subset t per slice: rays, times ring pairs on a multi-ring scanner."""
        rings = getattr(self.geom, "n_rings", 0)
        return self.subset_rays(t) * (rings * rings if rings else 1)

    def __del__(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.pet_plan_destroy(self.handle)
            self.handle = None


class Problem:
    """Counts, background and penalty bound to a plan (data copied on the device)."""

    def __init__(self, plan: Plan, counts, bg, bg_scalar: float, beta: float, stream=None,
                 potential: str = "quadratic", delta: float = 1.0):
        self.plan = plan
        self.handle = pet_problem_create(plan.handle, counts, bg, bg_scalar, beta, stream, potential, delta)

    def __del__(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.pet_problem_destroy(self.handle)
            self.handle = None


class Batch:
    """States whose updates run together (one launch per phase for all)."""

    def __init__(self, states, graphs: bool = True):
        self.states = list(states)
        self.handle = pet_batch_create([st.handle for st in self.states])
        if not graphs:
            pet_batch_set_graphs(self.handle, False)

    def epoch(self, seqs, alphas, etas, stream=None):
        pet_batch_epoch(self.handle, seqs, alphas, etas, stream)

    def objective_async(self, phi_out, stream=None):
        pet_batch_objective_async(self.handle, phi_out, stream)

    def set_mode(self, mode: str):
        """'phases' (default), 'dataflow' (one launch per epoch call) or
        'streams' (the members' own graphs on the batch's streams)."""
        _call("pet_batch_set_mode", self.handle, {"phases": 0, "dataflow": 1, "streams": 2}[mode])

    def set_wait_limit(self, polls: int):
        _call("pet_batch_set_wait_limit", self.handle, int(polls))

    def sync(self, stream=None):
        """Synchronise and raise PetError (PET_ERR_TIMEOUT) if a dataflow wait ran out."""
        _call("pet_batch_sync", self.handle, _stream(stream))

    def __del__(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.pet_batch_destroy(self.handle)
            self.handle = None


class State:
    """One running reconstruction of ``algo`` on the borrowed image ``img``."""

    def __init__(self, problem: Problem, algo: str, img, table: str = "fp32", stream=None):
        self.problem, self.algo, self.img = problem, algo, img
        self.handle = pet_state_create(problem.handle, algo, table, img, stream)

    def epoch(self, seq, alpha: float = 1.0, eta: int = 1, stream=None, decay: float = 0.0):
        if self.algo == "osem":
            pet_osem_epoch(self.handle, seq, stream)
        elif self.algo == "sga":
            pet_sga_epoch(self.handle, alpha, decay, seq, stream)
        elif self.algo == "sem":
            pet_sem_epoch(self.handle, alpha, decay, seq, stream)
        elif self.algo == "sagaem":
            pet_sagaem_epoch(self.handle, alpha, seq, stream)
        elif self.algo == "svrem":
            pet_svrem_epoch(self.handle, alpha, eta, seq, stream)
        elif self.algo == "saga":
            pet_saga_epoch(self.handle, alpha, seq, stream)
        else:
            pet_svrg_epoch(self.handle, alpha, eta, seq, stream)

    def run(self, seq, alpha: float = 1.0, eta: int = 1, objective_every: int = 0, phi=None, stream=None,
            decay: float = 0.0):
        """The updates of ``epoch`` with the objective after every
        ``objective_every``-th one written into ``phi`` ([points, 3] float64)."""
        pet_state_run(self.handle, seq, alpha, decay, eta, objective_every, phi, stream)

    def reset(self, stream=None):
        pet_state_reset(self.handle, stream)

    def set_preconditioner(self, kind: str):
        pet_state_set_preconditioner(self.handle, kind)

    def objective_async(self, phi_out, stream=None):
        pet_state_objective_async(self.handle, phi_out, stream)

    def __del__(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.pet_state_destroy(self.handle)
            self.handle = None
