"""Continuous-batching reconstruction servers: host schedulers over the C ABI.

Requests (a geometry, counts, a method and a target objective Phi*) arrive
over time.  A server admits a request as soon as it has arrived and both a
slot and device memory are free.  The budget counts every plan (built once
per geometry and subset count and kept), and the problem and state bytes the
library reports for each slot, SAGA's gradient table included.  A retired
request's slot (problem, state, image buffer) is kept in a pool: a later
request of the same shape, method and penalty reuses it through
pet_problem_update, pet_warm_start and pet_state_reset, which allocate
nothing; pooled slots are released, oldest first, when an admission needs
their memory.  Plans get their launch shapes from the library's autotuner,
timed once per request shape (tuned_plan) and shared by every path.

Two ways to let the work of concurrent requests overlap on the device:

* ``Server`` (one batch): all admitted requests advance together; every tick
  runs `tick` updates of every active state through one pet_batch_epoch call
  (by default in the streams batch mode, the members' own graphs on the
  batch's streams; or in persistent phases, one batched launch per phase), so
  requests that arrive while others run join the next tick.  The host meets the device once per `window`
  ticks: it enqueues the window's ticks back to back, synchronises once,
  reads every epoch-end objective of the window in order, retires finished
  requests and admits new ones.  A request that finished early in a window
  runs the rest of it (updates past its stopping epoch, whose image is not
  the result).

* ``StreamServer`` (one stream per request): every active request runs whole
  epochs through its own State (captured graphs) on its own CUDA stream, so
  the kernels of different requests run concurrently on the device; the host
  polls events and launches a request's next epoch as soon as its previous
  one is checked, or (while fewer than `speculate_below` requests are active)
  up to `depth` epochs ahead of the check.

At the end of each of its epochs a request's objective is enqueued and its
image copied aside; once the relative gap to its Phi* is at most `gap` (or it
has run `max_epochs` epochs) the image of that epoch is its result.  A
request's result depends only on the request: its subset sequence is seeded
by the request and counted from its admission, and the batched kernels give
each member exactly what its own epoch calls would.  Served alone, in a mix,
by either server or by the plain one-at-a-time path (serve_plain), it
returns the same image.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import petvr
from .phantoms import Workload, subset_sequence

STEP = {"svrem": (0.7, 1), "saga": (1.0, 1), "svrg": (2.0, 2), "osem": (1.0, 1)}

# Launch shapes per request shape: timed once per process by the library's
# autotuner on the first plan of that shape and set on every later one, so
# that every path (either server, the plain path) runs a shape with the same
# kernels and returns the same image.
_TUNING: dict = {}


def tuned_plan(work: Workload):
    """A plan of this request shape with its process-wide launch shapes."""
    plan = petvr.Plan(work.geometry, work.n_subsets)
    key = _Base._plan_key(work)
    if key not in _TUNING:
        _TUNING[key] = petvr.pet_plan_autotune(plan.handle)
    else:
        petvr.pet_plan_set_tuning(plan.handle, *_TUNING[key])
    return plan


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


def _table(algo: str) -> str:
    return "bf16" if algo == "saga" else "fp32"


@dataclass
class _Slot:
    key: tuple                  # (plan key, algo, table, beta): what a pooled slot can serve
    problem: petvr.Problem
    state: petvr.State
    img: torch.Tensor
    bytes: int
    stream: torch.cuda.Stream | None = None
    req: Request | None = None
    seq: np.ndarray | None = None
    pos: int = 0                # Server: updates issued
    launched: int = 0           # StreamServer: epochs issued
    inflight: collections.deque = field(default_factory=collections.deque)
    phi: torch.Tensor | None = None
    phi_host: torch.Tensor | None = None
    retiring: tuple | None = None


@dataclass
class ServerStats:
    ticks: int = 0
    max_active: int = 0
    active_sum: int = 0
    admissions_deferred: int = 0
    batches_built: int = 0
    peak_bytes: int = 0
    slots_created: int = 0
    slots_reused: int = 0
    slots_released: int = 0
    epochs_launched: int = 0    # request epochs enqueued (a batch counts each member's)
    extra: dict = field(default_factory=dict)


class _Base:
    """Plans, the slot pool and the device-memory budget."""

    def __init__(self, budget_bytes: int, max_slots: int, gap: float, max_epochs: int):
        if max_slots < 1:
            raise ValueError("max_slots must be positive")
        self.budget, self.max_slots = int(budget_bytes), int(max_slots)
        self.gap, self.max_epochs = gap, max_epochs
        self.plans = {}                 # (nx, ny, views, bins, subsets) -> (Plan, bytes)
        self.used = 0                   # plans + active slots + pooled slots
        self.active: list[_Slot] = []
        self.pool: collections.OrderedDict = collections.OrderedDict()   # id -> idle _Slot, oldest first
        self.stats = ServerStats()

    @staticmethod
    def _plan_key(work):
        g = work.geometry
        return (g.nx, g.ny, g.n_angles, g.n_bins, work.n_subsets)

    def _slot_key(self, req: Request):
        return (self._plan_key(req.work), req.algo, _table(req.algo), float(req.work.beta))

    def _plan(self, work):
        key = self._plan_key(work)
        if key not in self.plans:
            plan = tuned_plan(work)
            nbytes = petvr.pet_plan_bytes(plan.handle)
            self.plans[key] = (plan, nbytes)
            self._charge(nbytes)
        return self.plans[key][0]

    def _charge(self, nbytes: int):
        self.used += nbytes
        self.stats.peak_bytes = max(self.stats.peak_bytes, self.used)

    @property
    def active_bytes(self) -> int:
        return sum(s.bytes for s in self.active)

    def prepare(self, works):
        """Build the plans of these request shapes ahead of the stream."""
        for w in works:
            self._plan(w)
        torch.cuda.synchronize()

    def slot_bytes(self, req: Request) -> int:
        plan = self._plan(req.work)
        return (petvr.pet_problem_bytes(plan.handle, False)
                + petvr.pet_plan_state_bytes(plan.handle, req.algo, _table(req.algo)))

    def bytes_needed(self, req: Request) -> int:
        """Device bytes admitting `req` adds: none if a pooled slot fits it,
        else its problem and state (and its plan, if not built yet)."""
        key = self._slot_key(req)
        if any(s.key == key for s in self.pool.values()):
            return 0
        if self._plan_key(req.work) in self.plans:
            return self.slot_bytes(req)
        plan = petvr.Plan(req.work.geometry, req.work.n_subsets)
        return (petvr.pet_plan_bytes(plan.handle) + petvr.pet_problem_bytes(plan.handle, False)
                + petvr.pet_plan_state_bytes(plan.handle, req.algo, _table(req.algo)))

    def _fits(self, req: Request) -> bool:
        """Make room for `req` by releasing pooled slots (oldest first) that
        it cannot use; True if it then fits the budget."""
        need = self.bytes_needed(req)
        if need == 0:
            return True
        for sid in list(self.pool):
            if self.used + need <= self.budget:
                break
            slot = self.pool.pop(sid)
            self.used -= slot.bytes
            self.stats.slots_released += 1
            del slot
        return self.used + need <= self.budget

    def _take_slot(self, req: Request, stream) -> _Slot:
        """A slot holding `req`'s data and a warm-started state, enqueued on
        `stream`: a pooled one when its shape, method and penalty match."""
        key = self._slot_key(req)
        counts_host = np.ascontiguousarray(req.counts, dtype=np.float32).ravel()
        with torch.cuda.stream(stream):
            counts = torch.from_numpy(counts_host).to("cuda")
        for sid, slot in self.pool.items():
            if slot.key == key:
                del self.pool[sid]
                petvr.pet_problem_update(slot.problem.handle, counts, None, req.w, stream)
                petvr.pet_warm_start(slot.problem.handle, slot.img, stream)
                slot.state.reset(stream)
                self.stats.slots_reused += 1
                return slot
        plan = self._plan(req.work)
        nbytes = self.slot_bytes(req)
        problem = petvr.Problem(plan, counts, None, req.w, req.work.beta, stream=stream)
        with torch.cuda.stream(stream):
            img = torch.empty(req.work.geometry.n_pixels, device="cuda")
        petvr.pet_warm_start(problem.handle, img, stream)
        state = petvr.State(problem, req.algo, img, table=_table(req.algo), stream=stream)
        self._charge(nbytes)
        self.stats.slots_created += 1
        return _Slot(key, problem, state, img, nbytes)

    def _release(self, slot: _Slot):
        """Back to the pool (its memory stays charged until it is evicted)."""
        self.active.remove(slot)
        slot.req, slot.seq, slot.retiring = None, None, None
        slot.inflight.clear()
        self.pool[id(slot)] = slot

    def _admit_arrivals(self, pending, t0, clock, stream_for):
        """Admit every request that has arrived while a slot and memory are
        free (a request that does not fit waits, and so do those behind it)."""
        while pending and pending[0].arrival <= clock() - t0 and len(self.active) < self.max_slots:
            req = pending[0]
            if not self._fits(req) and self.active:
                self.stats.admissions_deferred += 1
                return
            pending.pop(0)
            stream = stream_for()
            slot = self._take_slot(req, stream)
            slot.req, slot.stream = req, stream
            req.admitted, req.bytes = clock() - t0, slot.bytes
            self._start(slot)
            self.active.append(slot)
            self.stats.max_active = max(self.stats.max_active, len(self.active))

    def _start(self, slot: _Slot):
        raise NotImplementedError


class Server(_Base):
    """One batch: every tick advances all active requests by `tick` updates
    in one batched launch per phase; the host synchronises once per
    `window` ticks."""

    def __init__(self, budget_bytes: int, max_slots: int = 64, gap: float = 1e-4, max_epochs: int = 60,
                 tick: int = 3, window: int = 1, batch_mode: str = "streams"):
        if tick < 1 or window < 1:
            raise ValueError("tick and window must be positive")
        # pet_batch_set_mode of the tick batches: the members' own graphs on the batch's streams measured
        # 20.5 reconstructions/s against 20.0 in persistent phases on the 96 distinct requests (same p50)
        self.batch_mode = batch_mode
        super().__init__(budget_bytes, max_slots, gap, max_epochs)
        self.tick, self.window = tick, window
        self._batch = None
        rows = max_slots * window       # one objective row per epoch end a window can hold
        self._phi = torch.zeros(rows, 3, dtype=torch.float64, device="cuda")
        self._phi_host = torch.zeros(rows, 3, dtype=torch.float64).pin_memory()

    def _start(self, slot: _Slot):
        ns = slot.req.work.n_subsets
        if ns % self.tick:
            raise ValueError(f"tick {self.tick} must divide the request's {ns} subsets")
        # updates past max_epochs (the rest of a window) read the tail
        slot.seq = subset_sequence(slot.req.seed, ns, self.max_epochs * ns + self.window * self.tick)
        slot.pos = 0
        self._batch = None

    def serve(self, requests, clock=time.perf_counter):
        """Serve `requests` (arrival times in seconds from now); returns them
        with admission/completion times, epochs, final gap and image."""
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        stream = torch.cuda.current_stream()
        t0 = clock()
        while pending or self.active:
            self._admit_arrivals(pending, t0, clock, lambda: stream)
            if not self.active:
                wait = pending[0].arrival - (clock() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.001))
                continue
            if self._batch is None:
                self._batch = petvr.Batch([s.state for s in self.active], graphs=False)
                if self.batch_mode != "phases":
                    self._batch.set_mode(self.batch_mode)
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
                    if s.pos % ns == 0:
                        self.stats.epochs_launched += 1
                    if s.pos % ns == 0 and s.pos <= self.max_epochs * ns:   # an epoch of this request ended
                        row = len(checks)
                        s.state.objective_async(self._phi[row], stream=stream)
                        checks.append((s, row, s.img.clone(), s.pos // ns))
                self.stats.ticks += 1
                self.stats.active_sum += len(self.active)
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
                    r.image = image.cpu().numpy()
                    r.done = now
                    retired.add(id(s))
                    self._release(s)
                    self._batch = None
        return requests


@dataclass
class _Epoch:
    event: torch.cuda.Event
    epoch: int
    row: int
    image: torch.Tensor


class StreamServer(_Base):
    """One stream per request: whole epochs through each request's own State
    (captured graphs) on its own stream, up to `depth` epochs ahead of the
    host's gap checks."""

    def __init__(self, budget_bytes: int, max_slots: int = 64, gap: float = 1e-4, max_epochs: int = 60,
                 depth: int = 2, speculate_below: int = 16):
        if depth < 1:
            raise ValueError("depth must be positive")
        super().__init__(budget_bytes, max_slots, gap, max_epochs)
        self.depth = depth
        # epochs beyond the one the host has not checked yet are speculative
        # (wasted if the gap was reached): worth it only while few requests
        # share the device and an idle gap between epochs would show
        self.speculate_below = speculate_below
        self._streams: list[torch.cuda.Stream] = []

    def _stream(self):
        return self._streams.pop() if self._streams else torch.cuda.Stream()

    def _start(self, slot: _Slot):
        ns = slot.req.work.n_subsets
        slot.seq = subset_sequence(slot.req.seed, ns, self.max_epochs * ns)
        slot.launched = 0
        if slot.phi is None:
            slot.phi = torch.zeros(self.depth, 3, dtype=torch.float64, device="cuda")
            slot.phi_host = torch.zeros(self.depth, 3, dtype=torch.float64).pin_memory()

    def _launch_epoch(self, slot: _Slot):
        r = slot.req
        ns = r.work.n_subsets
        e = slot.launched
        row = e % self.depth
        alpha, eta = STEP[r.algo]
        with torch.cuda.stream(slot.stream):
            slot.state.epoch(slot.seq[e * ns:(e + 1) * ns], alpha=alpha, eta=eta, stream=slot.stream)
            slot.state.objective_async(slot.phi[row], stream=slot.stream)
            image = slot.img.clone()
            slot.phi_host[row].copy_(slot.phi[row], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(slot.stream)
        slot.inflight.append(_Epoch(ev, e + 1, row, image))
        slot.launched += 1
        self.stats.epochs_launched += 1

    def _poll(self, slot: _Slot, now) -> bool:
        """Advance one request; True if anything happened."""
        if slot.retiring is not None:           # its result is on the way to the host
            ev, host = slot.retiring
            if not ev.query():
                return False
            slot.req.image = host.numpy().copy()
            slot.req.done = now()
            self._streams.append(slot.stream)
            self._release(slot)
            return True
        progressed = False
        ahead = self.depth if len(self.active) < self.speculate_below else 1
        while len(slot.inflight) < ahead and slot.launched < self.max_epochs:
            self._launch_epoch(slot)
            progressed = True
        head = slot.inflight[0]
        if not head.event.query():
            return progressed
        slot.inflight.popleft()
        r = slot.req
        r.epochs = head.epoch
        r.gap = (r.phi_star - float(slot.phi_host[head.row, 0])) / abs(r.phi_star)
        if r.gap <= self.gap or r.epochs >= self.max_epochs:
            r.reached = r.gap <= self.gap
            with torch.cuda.stream(slot.stream):
                host = torch.empty(head.image.shape, dtype=head.image.dtype).pin_memory()
                host.copy_(head.image, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(slot.stream)
            slot.retiring = (ev, host)
        return True

    def serve(self, requests, clock=time.perf_counter):
        """Serve `requests` (arrival times in seconds from now); returns them
        with admission/completion times, epochs, final gap and image."""
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        t0 = clock()
        now = lambda: clock() - t0       # noqa: E731
        while pending or self.active:
            self._admit_arrivals(pending, t0, clock, self._stream)
            progressed = False
            for slot in list(self.active):
                progressed |= self._poll(slot, now)
            if not progressed:
                if not self.active and pending:
                    wait = pending[0].arrival - now()
                    if wait > 0:
                        time.sleep(min(wait, 0.001))
                else:
                    time.sleep(0)
        return requests


def serve_native(requests, gap: float = 1e-4, max_epochs: int = 60, n_streams: int = 64,
                 budget_bytes: int = 1 << 30):
    """The stream server's policy with the whole loop in the library
    (pet_serve_requests): a request is admitted once it has arrived, one of
    `n_streams` streams is free and its slot fits the device-memory budget
    (problem, state, image and counts staging; slots are pooled by plan,
    method, table and penalty and freed least recently used first), then runs
    its epochs with the objective after each until the gap or max_epochs, all
    from C++.  A request's subset sequence, launch shapes and result are
    those of the other paths.  Returns the requests (filled in) and the
    call's slot statistics."""
    reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
    plans, specs = {}, []
    for r in reqs:
        key = _Base._plan_key(r.work)
        if key not in plans:
            plans[key] = tuned_plan(r.work)
        alpha, eta = STEP[r.algo]
        specs.append({"plan": plans[key], "counts": r.counts, "bg": r.w, "beta": r.work.beta, "algo": r.algo,
                      "table": _table(r.algo), "seq": subset_sequence(r.seed, r.work.n_subsets,
                                                                       max_epochs * r.work.n_subsets),
                      "alpha": alpha, "eta": eta, "phi_star": r.phi_star, "arrival_s": r.arrival,
                      "n_image": r.work.geometry.n_pixels})
    torch.cuda.synchronize()
    epochs, gaps, t_start, t_done, images, stats = petvr.pet_serve_requests(specs, n_streams, budget_bytes,
                                                                           max_epochs, gap)
    for r, e, g, t0, t1, im in zip(reqs, epochs, gaps, t_start, t_done, images):
        r.epochs, r.gap = int(e), float(g)
        r.reached = r.gap <= gap
        r.admitted, r.done = float(t0) / 1e3, float(t1) / 1e3
        r.image = im
    return requests, stats


def serve_plain(requests, gap: float = 1e-4, max_epochs: int = 60, clock=time.perf_counter):
    """The plain per-reconstruction path, for comparison with the servers:
    requests are taken in arrival order, one at a time, each run epoch by
    epoch through its own State (one captured graph per epoch shape) with
    the objective checked after every epoch.  A request uses the same subset
    sequence, step size and stopping rule as under the servers, so it
    returns the same image."""
    pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
    plans = {}
    for r in pending:                       # plans ahead of the stream, as Server.prepare
        key = _Base._plan_key(r.work)
        if key not in plans:
            plans[key] = tuned_plan(r.work)
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
        problem = petvr.Problem(plans[_Base._plan_key(r.work)], counts, None, r.w, r.work.beta)
        img = torch.empty(r.work.geometry.n_pixels, device="cuda")
        petvr.pet_warm_start(problem.handle, img)
        state = petvr.State(problem, r.algo, img, table=_table(r.algo))
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
    """Completion latency (arrival to result on the host) percentiles, queueing
    (arrival to admission), and rates over the span from the first arrival to
    the last completion: all completed requests, and those that reached the
    objective gap (the others stopped at max_epochs)."""
    lat = np.array([r.done - r.arrival for r in requests if np.isfinite(r.done)])
    wait = np.array([r.admitted - r.arrival for r in requests if np.isfinite(r.admitted)])
    span = max(r.done for r in requests) - min(r.arrival for r in requests)
    reached = int(sum(r.reached for r in requests))
    return {"completed": int(len(lat)), "reached_gap": reached,
            "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "mean_wait_ms": 1e3 * float(wait.mean()), "recon_per_s": len(lat) / span,
            "reached_per_s": reached / span, "epochs_mean": float(np.mean([r.epochs for r in requests]))}


def per_template(requests):
    """Requests, gap reached and mean epochs per request template."""
    out = {}
    for r in requests:
        e = out.setdefault(r.work.name, {"requests": 0, "reached": 0, "epochs": 0.0, "algo": r.algo,
                                         "size": r.work.geometry.nx, "subsets": r.work.n_subsets})
        e["requests"] += 1
        e["reached"] += int(r.reached)
        e["epochs"] += r.epochs
    for e in out.values():
        e["epochs"] /= max(1, e["requests"])
    return out
