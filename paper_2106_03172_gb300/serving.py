"""Continuous-batching reconstruction server: a host scheduler over the C ABI.

Requests (a geometry, counts, a method and a target objective Phi*) arrive
over time.  The server admits a request as soon as it has arrived and both a
slot and device memory are free: its budget counts the plan (shared by every
request of the same geometry and subset count), the problem and the state
bytes the library reports, SAGA's gradient table included.  All admitted
requests advance together: every tick runs `tick` updates of every active
state in one batched launch per phase (pet_batch_epoch), so requests that
arrive while others run join the next tick and their work shares the
kernels.  At the end of each of its epochs a request's objective is enqueued
and its image copied aside; once the relative gap to its Phi* is at most
`gap` (or it has run `max_epochs` epochs) the image of that epoch is its
result and its memory is released.

The host meets the device once per `window` ticks: it enqueues the window's
ticks back to back, then synchronises once, reads every epoch-end objective
of the window in order, retires finished requests and admits new ones.  A
request that finished early in a window runs the rest of it (updates past
its stopping epoch, which do not change its result); the price of a longer
window is that waste and a later admission, the gain is one host round trip
per window instead of per tick.

A request's result depends only on the request: its subset sequence is
seeded by the request, ticks are counted from its own admission, and the
batched kernels give each member exactly what its own epoch calls would.
Served alone or in a mix, it returns the same image.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import petvr
from .phantoms import Workload, subset_sequence

STEP = {"svrem": (0.7, 1), "saga": (1.0, 1), "svrg": (2.0, 2), "osem": (1.0, 1)}


@dataclass
class Request:
    rid: int
    work: Workload
    counts: np.ndarray          # float32 sinogram [view][bin]
    w: float                    # uniform background per bin
    phi_star: float             # target objective (from the FP64 oracle)
    arrival: float              # seconds after the stream starts
    seed: int = 0
    algo: str = ""
    # filled in by the server
    admitted: float = float("nan")
    done: float = float("nan")
    epochs: int = 0
    gap: float = float("nan")
    reached: bool = False
    image: np.ndarray | None = None
    bytes: int = 0

    def __post_init__(self):
        if not self.algo:
            self.algo = self.work.methods[0]


@dataclass
class _Slot:
    req: Request
    problem: petvr.Problem
    state: petvr.State
    img: torch.Tensor
    seq: np.ndarray
    pos: int = 0


@dataclass
class ServerStats:
    ticks: int = 0
    max_active: int = 0
    active_sum: int = 0
    admissions_deferred: int = 0
    batches_built: int = 0
    peak_bytes: int = 0
    extra: dict = field(default_factory=dict)


class Server:
    def __init__(self, budget_bytes: int, max_slots: int = 64, gap: float = 1e-4, max_epochs: int = 60,
                 tick: int = 3, window: int = 1):
        if tick < 1 or max_slots < 1 or window < 1:
            raise ValueError("tick, window and max_slots must be positive")
        self.budget, self.max_slots = int(budget_bytes), int(max_slots)
        self.gap, self.max_epochs, self.tick, self.window = gap, max_epochs, tick, window
        self.plans = {}                 # (nx, ny, views, bins, subsets) -> (Plan, bytes, users)
        self.used = 0
        self.active: list[_Slot] = []
        self.stats = ServerStats()
        self._batch = None
        # one objective row per epoch end a window can hold
        rows = max_slots * window
        self._phi = torch.zeros(rows, 3, dtype=torch.float64, device="cuda")
        self._phi_host = torch.zeros(rows, 3, dtype=torch.float64).pin_memory()

    # ---- memory accounting -------------------------------------------------
    @staticmethod
    def _key(work):
        g = work.geometry
        return (g.nx, g.ny, g.n_angles, g.n_bins, work.n_subsets)

    def _plan(self, work):
        key = self._key(work)
        if key not in self.plans:
            plan = petvr.Plan(work.geometry, work.n_subsets)
            self.plans[key] = [plan, petvr.pet_plan_bytes(plan.handle), 0]
        return self.plans[key]

    def bytes_needed(self, req: Request) -> int:
        """Device bytes admitting `req` adds (its plan only if no active request holds it)."""
        plan, plan_bytes, users = self._plan(req.work)
        table = "bf16" if req.algo == "saga" else "fp32"
        return ((plan_bytes if users == 0 else 0) + petvr.pet_problem_bytes(plan.handle, False)
                + petvr.pet_plan_state_bytes(plan.handle, req.algo, table))

    def prepare(self, works):
        """Build the plans of these request shapes ahead of the stream (a
        plan is computed once per geometry and subset count)."""
        for w in works:
            self._plan(w)
        torch.cuda.synchronize()

    # ---- admission and retirement -----------------------------------------
    def _admit(self, req: Request, now: float):
        entry = self._plan(req.work)
        plan = entry[0]
        need = self.bytes_needed(req)
        counts = torch.from_numpy(np.ascontiguousarray(req.counts, dtype=np.float32).ravel()).cuda()
        problem = petvr.Problem(plan, counts, None, req.w, req.work.beta)
        img = torch.empty(req.work.geometry.n_pixels, device="cuda")
        petvr.pet_warm_start(problem.handle, img)
        table = "bf16" if req.algo == "saga" else "fp32"
        state = petvr.State(problem, req.algo, img, table=table)
        ns = req.work.n_subsets
        if ns % self.tick:
            raise ValueError(f"tick {self.tick} must divide the request's {ns} subsets")
        # updates past max_epochs (the rest of a window) read the tail
        seq = subset_sequence(req.seed, ns, self.max_epochs * ns + self.window * self.tick)
        entry[2] += 1
        self.used += need
        self.stats.peak_bytes = max(self.stats.peak_bytes, self.used)
        req.admitted, req.bytes = now, need
        self.active.append(_Slot(req, problem, state, img, seq))
        self._batch = None

    def _retire(self, slot: _Slot, now: float, image: torch.Tensor):
        slot.req.image = image.cpu().numpy()
        slot.req.done = now
        self.used -= slot.req.bytes
        entry = self.plans[self._key(slot.req.work)]
        entry[2] -= 1
        self.active.remove(slot)
        self._batch = None

    # ---- the loop ------------------------------------------------------------
    def serve(self, requests, clock=time.perf_counter):
        """Serve `requests` (arrival times in seconds from now); returns them
        with admission/completion times, epochs, final gap and image."""
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        t0 = clock()
        stream = torch.cuda.current_stream()
        while pending or self.active:
            now = clock() - t0
            while pending and pending[0].arrival <= now and len(self.active) < self.max_slots:
                if self.used + self.bytes_needed(pending[0]) > self.budget and self.active:
                    self.stats.admissions_deferred += 1
                    break
                self._admit(pending.pop(0), clock() - t0)
            if not self.active:
                wait = pending[0].arrival - (clock() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.001))
                continue
            if self._batch is None:
                self._batch = petvr.Batch([s.state for s in self.active], graphs=False)
                self.stats.batches_built += 1
            alphas = [STEP[s.req.algo][0] for s in self.active]
            etas = [STEP[s.req.algo][1] for s in self.active]
            checks = []                 # (slot, objective row, image at that epoch end, epoch)
            for _ in range(self.window):
                seqs = [s.seq[s.pos:s.pos + self.tick] for s in self.active]
                self._batch.epoch(seqs, alphas, etas, stream=stream)
                for s in self.active:
                    s.pos += self.tick
                    ns = s.req.work.n_subsets
                    if s.pos % ns == 0 and s.pos <= self.max_epochs * ns:   # an epoch of this request ended
                        row = len(checks)
                        s.state.objective_async(self._phi[row], stream=stream)
                        checks.append((s, row, s.img.clone(), s.pos // ns))
                self.stats.ticks += 1
                self.stats.active_sum += len(self.active)
            self.stats.max_active = max(self.stats.max_active, len(self.active))
            if checks:
                self._phi_host[:len(checks)].copy_(self._phi[:len(checks)], non_blocking=True)
            torch.cuda.synchronize()
            now = clock() - t0
            retired = set()
            for s, row, image, epoch in checks:             # in the order the epochs ended
                if id(s) in retired:
                    continue
                r = s.req
                r.epochs = epoch
                r.gap = (r.phi_star - float(self._phi_host[row, 0])) / abs(r.phi_star)
                if r.gap <= self.gap or r.epochs >= self.max_epochs:
                    r.reached = r.gap <= self.gap
                    self._retire(s, now, image)
                    retired.add(id(s))
        return requests


def serve_plain(requests, gap: float = 1e-4, max_epochs: int = 60, clock=time.perf_counter):
    """The plain per-reconstruction path, for comparison with Server: requests
    are taken in arrival order, one at a time, each run epoch by epoch through
    its own State (one captured graph per epoch shape) with the objective
    checked after every epoch.  A request uses the same subset sequence, step
    size and stopping rule as under Server, so it returns the same image."""
    pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
    plans = {}
    for r in pending:                       # plans ahead of the stream, as Server.prepare
        key = Server._key(r.work)
        if key not in plans:
            plans[key] = petvr.Plan(r.work.geometry, r.work.n_subsets)
    stream = torch.cuda.current_stream()
    phi = torch.zeros(3, dtype=torch.float64, device="cuda")
    phi_host = torch.zeros(3, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = clock()
    for r in pending:
        wait = r.arrival - (clock() - t0)
        if wait > 0:
            time.sleep(wait)
        r.admitted = clock() - t0
        counts = torch.from_numpy(np.ascontiguousarray(r.counts, dtype=np.float32).ravel()).cuda()
        problem = petvr.Problem(plans[Server._key(r.work)], counts, None, r.w, r.work.beta)
        img = torch.empty(r.work.geometry.n_pixels, device="cuda")
        petvr.pet_warm_start(problem.handle, img)
        state = petvr.State(problem, r.algo, img, table="bf16" if r.algo == "saga" else "fp32")
        ns = r.work.n_subsets
        seq = subset_sequence(r.seed, ns, max_epochs * ns)
        alpha, eta = STEP[r.algo]
        for e in range(max_epochs):
            state.epoch(seq[e * ns:(e + 1) * ns], alpha=alpha, eta=eta, stream=stream)
            state.objective_async(phi, stream=stream)
            phi_host.copy_(phi, non_blocking=True)
            torch.cuda.synchronize()
            r.epochs = e + 1
            r.gap = (r.phi_star - float(phi_host[0])) / abs(r.phi_star)
            if r.gap <= gap:
                break
        r.reached = r.gap <= gap
        r.image = img.cpu().numpy()
        r.done = clock() - t0
        del state, problem
    return requests


def latency_summary(requests):
    lat = np.array([r.done - r.arrival for r in requests if np.isfinite(r.done)])
    wait = np.array([r.admitted - r.arrival for r in requests if np.isfinite(r.admitted)])
    span = max(r.done for r in requests) - min(r.arrival for r in requests)
    return {"completed": int(len(lat)), "reached_gap": int(sum(r.reached for r in requests)),
            "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "mean_wait_ms": 1e3 * float(wait.mean()), "recon_per_s": len(lat) / span,
            "epochs_mean": float(np.mean([r.epochs for r in requests]))}
