#!/usr/bin/env python
"""Benchmark of the penalised stochastic-EM hot path on one GB300 per rank.

Workload (default ``c256``): 256x256 image of 2 mm pixels, 180 views x 367
bins, 21 angle-interleaved subsets, seeded 20-ellipse phantom with 6 hot
lesions, 1e7 expected counts plus a 10% uniform background, quadratic
penalty beta = 0.005.  The warm start is one unpenalised OSEM epoch.

One step = one epoch (21 subset updates) of each of OSEM, SVREM (alpha 0.7,
eta 1), SAGA (alpha 1, FP32 table) and SVRG (alpha 2, eta 2), each followed by
its FP64 objective; anchor passes (SVREM every epoch, SVRG every second
epoch) run inside the step when due.  The metric counts subset forward+back
projection pairs (A_t f then A_t^T r): 84 per step plus 21 per anchor pass.

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events
on the launching stream; a 256 MiB buffer is written between steps (outside
the events) so every step starts with a cold L2.  ``e2e`` repeats the steps
through the public API with the counts copied in from pinned host memory and
the four images and objectives copied back, inside the events; the host
enqueues one step after another without waiting, as a pipeline would.  Per-kernel
durations for the roofline come from a separate profiled pass (event pairs
around every projector launch, methods run one after another, no graphs).
The four reconstructions of a step are independent and run on four streams;
each method's epoch is one captured CUDA graph.

``--impl reference`` times the FP64 CPU oracle on the host cores instead (the
same step on the same workload), on rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METHODS = ("osem", "svrem", "saga", "svrg")
FP32_LANES_PER_SM = 128
N_SMS = 152
SM_MAX_MHZ = 2070.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c256")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--recon", type=int, default=200, help="reconstructions per method for the gap metric")
    ap.add_argument("--tuning", default="", help="pin launch shapes 'chunks,run' instead of autotuning")
    ap.add_argument("--requests", type=int, default=1000, help="serve workload: number of requests")
    ap.add_argument("--rate", type=float, default=200.0, help="serve workload: mean arrivals per second")
    ap.add_argument("--budget-gib", type=float, default=1.0, help="serve workload: device-memory budget")
    ap.add_argument("--window", type=int, default=4, help="serve workload, batch server: ticks per host round trip")
    ap.add_argument("--max-epochs", type=int, default=200,
                    help="serve workload: epochs after which a request stops without reaching the gap")
    ap.add_argument("--depth", type=int, default=2, help="serve workload, stream server: epochs in flight per request")
    ap.add_argument("--distinct", action="store_true",
                    help="serve workload: requests with their own phantoms and counts (the stored-Phi* sample) "
                         "instead of draws from the request templates")
    ap.add_argument("--server", choices=["native", "streams", "batch"], default="native",
                    help="serve workload: the server the headline value is taken from (the other is reported too)")
    ap.add_argument("--batch", dest="batch", action="store_true",
                    help="run the four methods as one batch (one launch per phase) instead of four streams")
    ap.add_argument("--on", default="c256", help="converge workload: the problem the methods are compared on")
    ap.add_argument("--epochs", type=int, default=40, help="converge workload: update epochs per method")
    ap.add_argument("--step-epochs", type=int, default=50,
                    help="update epochs of each method per step (50: the 256^2 configuration's run length)")
    ap.add_argument("--legs", default="batched,batch64,stack,ring,serve,parity",
                    help="short extra measurements after the headline (comma list, or 'none')")
    return ap.parse_args()


def workload_config(work, epochs=50):
    g = work.geometry
    return {
        "workload": f"{work.name}: {g.nx}x{g.ny}" + (f"x{g.nz} volume ({g.n_rings} rings {g.ring_mm:g} mm apart, "
                                                      f"cylinder radius {g.radius_mm:g} mm, {g.slice_mm:g} mm layers, "
                                                      f"{g.n_pairs} lines per ray)" if g.multiring else " image")
                    + f" ({g.pixel_mm:g} mm pixels), {g.n_angles} views x "
                    f"{g.n_bins} bins, {work.n_subsets} angle-interleaved subsets, {work.counts:.0e} counts, "
                    f"{int(round(work.bg_frac * 100))}% background, {work.potential}"
                    + (f" (delta={work.delta:g})" if work.potential != "quadratic" else "") + f" beta={work.beta}",
        "step": f"{epochs} update epochs each of OSEM, SVREM(alpha={work.alpha_svrem}, eta={work.eta_svrem}), "
                f"SAGA(alpha={work.alpha_saga}, fp32 table), SVRG(alpha={work.alpha_svrg}, eta={work.eta_svrg}), "
                "each epoch followed by its FP64 objective; each method's step one pet_state_run call on its own "
                "stream (an objective's forward pass also gives the next SVREM/SVRG anchor's ratios)",
        "l2": "flushed between steps (256 MiB write outside the timed events)",
        "n_subsets": work.n_subsets,
        "image": [g.ny, g.nx],
        "sinogram": [g.n_angles, g.n_bins],
    }


def seqs_for_step(step: int, ns: int):
    from paper_2106_03172_gb300.phantoms import subset_sequence
    return [subset_sequence(2000 + 4 * step + i, ns, ns) for i in range(4)]


def alphas(work):
    return {"osem": (1.0, 1), "svrem": (work.alpha_svrem, work.eta_svrem),
            "saga": (work.alpha_saga, 1), "svrg": (work.alpha_svrg, work.eta_svrg)}


class Replica:
    """Host bookkeeping of one rank's four reconstructions (counts anchor passes)."""

    def __init__(self, work):
        self.work = work
        self.k = {m: 0 for m in METHODS}

    def step_pairs(self):
        ns = self.work.n_subsets
        pairs = 4 * ns
        anchors = []
        for m in ("svrem", "svrg"):
            eta = alphas(self.work)[m][1]
            if self.k[m] % (eta * ns) == 0:
                pairs += ns
                anchors.append(m)
        return pairs, anchors

    def advance(self):
        for m in METHODS:
            self.k[m] += self.work.n_subsets


def combine_ranks(total_ms: float, units: float, device=None):
    """Whole-job throughput of independent replicas: the units every rank
    processed, summed, over the slowest rank's time (max over ranks).
    Returns (value per second, max ms, summed units)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return units / (total_ms / 1e3), total_ms, units
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / (float(t.item()) / 1e3), float(t.item()), float(u.item())


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits", "-lms", "50",
                 "-i", str(self.idx)], stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.06)                # one more sample interval, so a short region is not cut short
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def visible_index(torch):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    dev = torch.cuda.current_device()
    if vis:
        ids = [v.strip() for v in vis.split(",")]
        if dev < len(ids) and ids[dev].isdigit():
            return int(ids[dev])
    return dev


# --------------------------------------------------------------------------- oracle timing

def oracle_steps(work, data, n_steps: int, warmup: int = 0, min_seconds: float = 0.0, max_steps: int = 64):
    """Time ``n_steps`` oracle steps (the bench step in FP64 on the host),
    continuing up to ``max_steps`` while fewer than ``min_seconds`` have been
    timed; returns (per-step seconds, per-step pairs, setup seconds)."""
    from oracle import em
    from oracle.em import build_problem
    t0 = time.perf_counter()
    prob = build_problem(work.geometry, data["g"], data["w"], work.n_subsets, work.beta, work.potential, work.delta)
    f0 = prob.initial_image()
    setup = time.perf_counter() - t0
    a = alphas(work)
    algs = {"svrem": em.SVREM(prob, f0, *a["svrem"]), "saga": em.SAGA(prob, f0, a["saga"][0]),
            "svrg": em.SVRG(prob, f0, *a["svrg"])}
    f_osem = f0.copy()
    rep = Replica(work)
    times, pairs = [], []
    step = 0
    while step < warmup + n_steps or (sum(times) < min_seconds and len(times) < max_steps):
        seqs = seqs_for_step(step, work.n_subsets)
        p, _ = rep.step_pairs()
        t = time.perf_counter()
        f_osem = em.osem_epoch(prob, f_osem, seqs[0])
        prob.objective(f_osem)
        for i, m in enumerate(("svrem", "saga", "svrg")):
            for s in seqs[i + 1]:
                algs[m].step(int(s))
            prob.objective(algs[m].f)
        dt = time.perf_counter() - t
        rep.advance()
        if step >= warmup:
            times.append(dt)
            pairs.append(p)
        step += 1
    return times, pairs, setup


def run_reference(args):
    from paper_2106_03172_gb300.phantoms import WORKLOADS, make_data
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    work = WORKLOADS[args.workload]
    data = make_data(work, 0)
    times, pairs, setup = oracle_steps(work, data, args.steps, args.warmup)
    total = sum(times)
    value = sum(pairs) / total
    unit = "subset fwd+back projections/s"
    line = {
        "impl": "reference",
        "metric": "subset fwd+back projections/s and reconstructions/s to 1e-4 objective gap; p50/p99",
        "value": value, "unit": unit, "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded ellipse phantom, Poisson counts)",
        "config": workload_config(work),
        "p50_ms": 1e3 * float(np.percentile(times, 50)), "p99_ms": 1e3 * float(np.percentile(times, 99)),
        "cpu_baseline": {"value": value, "unit": unit, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} full bench steps after {args.warmup} warm-up steps "
                                   f"(system matrix build and warm start, {setup:.1f} s, untimed)"},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def kernel_source_digest() -> str:
    """SHA-256 of the projector sources with comments and whitespace removed,
    to tell whether a recorded ncu measurement still describes the kernels
    being run (a comment edit does not change them)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in ("forward.cu", "backward.cu", "bodies.cuh", "epilogue.cuh", "petvr_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2106_03172_gb300", "csrc", name)) as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()


def measured_hbm_peak():
    """Copy bandwidth (GB/s) measured on the GB300s (MEASURED_PEAKS.json),
    else the fallback figure, with which one it is."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))["hbm_gbs"]), "of measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, KeyError):
        return 6800.0, "of fallback (6.8 TB/s)"


def sm_max_mhz() -> float:
    """Maximum SM clock of the GB300s (MEASURED_PEAKS.json), else the
    device's reported maximum, else 2070 MHz."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"])
    except (OSError, ValueError, KeyError):
        pass
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits", "-i", "0"],
                             capture_output=True, text=True, timeout=10).stdout.strip().splitlines()
        return float(out[0])
    except Exception:
        return 2070.0


def _profile_record(workload: str):
    """Fields of profiles/roofline_traffic.txt, or {} when the record is for
    another workload or was taken on other projector sources."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.txt")
    if not os.path.exists(path):
        return {}
    rec = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            key, val = line.split(":", 1)
            rec[key.strip()] = val.strip()
    if rec.get("workload", "c256") != workload or rec.get("source_sha256") != kernel_source_digest():
        return {}
    return rec


def ncu_issue_record(kind: int, workload: str = "c256"):
    """ncu issue-active fraction (smsp__issue_active, of peak sustained active)
    of the dominant kernel kind from the committed record, or None."""
    val = _profile_record(workload).get(f"kind{kind}_issue_active_pct")
    return float(val) / 100.0 if val is not None else None


def dram_traffic_record(kind: int, workload: str = "c256"):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary (profiles/roofline_traffic.txt), or None when that summary was
    taken on other kernel sources, another workload, or does not cover this
    kernel kind."""
    val = _profile_record(workload).get(f"kind{kind}_dram_bytes_per_launch")
    return float(val) if val is not None else None


# --------------------------------------------------------------------------- objective gap

GAP = 1e-4


def phi_star_for(work, data):
    """Phi* of the workload: the value stored by tests/golden/make_phi_star.py
    (FP64 oracle) when the generated counts match its checksum, else None (the
    GPU arm does not run the oracle; the gap measurements are then skipped)."""
    import hashlib
    path = os.path.join(ROOT, "tests", "golden", "phi_star.json")
    sha = hashlib.sha256(data["g"].astype("<f4").tobytes()).hexdigest()
    if os.path.exists(path):
        table = json.load(open(path))
        ent = table.get(work.name)
        if ent and ent["counts_sha256"] == sha:
            return ent["phi_star"], "tests/golden/phi_star.json (FP64 oracle, L-BFGS-B)"
    return None, "no stored Phi* for these counts (run tests/golden/make_phi_star.py)"


def measure_recon(torch, petvr, prob, states, imgs, work, phi_star: float, n_rec: int, max_epochs: int = 60,
                  depth: int = 1):
    """Reconstructions to a relative objective gap <= GAP: warm start, state
    reset, then epochs, each followed by its objective, until the host sees
    the gap reached.  The host keeps `depth` epochs in flight (at depth 2 it
    checks epoch e while epoch e + 1 runs; each epoch's image is copied
    aside, so the result is the image of the epoch that reached the gap).  A
    reconstruction's latency runs from the event before its warm start to
    the event after the objective that reached the gap; recon_per_s is
    n_rec over the wall time of all of them, the speculative epochs after
    each one's gap included."""
    a = alphas(work)
    phi_dev = torch.zeros(depth, 3, dtype=torch.float64, device="cuda")
    phi_host = torch.zeros(depth, 3, dtype=torch.float64).pin_memory()
    stream = torch.cuda.current_stream()
    from paper_2106_03172_gb300.phantoms import subset_sequence
    out = {}
    for m in METHODS:
        snap = torch.empty(depth, imgs[m].numel(), device="cuda")
        lat, epochs, reached = [], [], 0
        done_ev = [torch.cuda.Event(enable_timing=True) for _ in range(depth)]
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        # the subset sequences are inputs: made before the timed reconstructions
        # (the first `ahead` epochs of each; later epochs, rarely reached, on the way)
        ahead = 8
        seqs = [[subset_sequence(90000 + 1000 * r + ep, work.n_subsets, work.n_subsets) for ep in range(ahead)]
                for r in range(n_rec)]
        t0.record(stream)
        for r in range(n_rec):
            e0 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            petvr.pet_warm_start(prob.handle, imgs[m])
            states[m].reset()

            def launch(ep):
                j = ep % depth
                seq = (seqs[r][ep] if ep < ahead else
                       subset_sequence(90000 + 1000 * r + ep, work.n_subsets, work.n_subsets))
                states[m].epoch(seq, alpha=a[m][0], eta=a[m][1])
                states[m].objective_async(phi_dev[j])
                snap[j].copy_(imgs[m])
                phi_host[j].copy_(phi_dev[j], non_blocking=True)
                done_ev[j].record(stream)

            launched = 0
            while launched < min(depth, max_epochs):
                launch(launched)
                launched += 1
            ep = 0
            while True:
                j = ep % depth
                done_ev[j].synchronize()
                gap = (phi_star - float(phi_host[j, 0])) / abs(phi_star)
                ep += 1
                if gap <= GAP or ep >= max_epochs:
                    reached += int(gap <= GAP)
                    lat.append(e0.elapsed_time(done_ev[j]))
                    epochs.append(ep)
                    break
                if launched < max_epochs:
                    launch(launched)
                    launched += 1
        t1.record(stream)
        torch.cuda.synchronize()
        out[m] = {"recon_per_s": n_rec / (t0.elapsed_time(t1) / 1e3), "p50_ms": float(np.percentile(lat, 50)),
                  "p99_ms": float(np.percentile(lat, 99)), "epochs_mean": float(np.mean(epochs)),
                  "reached": reached, "n": n_rec, "epochs_in_flight": depth}
    return out


def recon_executor(torch, petvr, prob, work, phi_star: float, n_rec: int, workers: int, max_epochs: int = 60):
    """The reconstructions of measure_recon (same subset sequences) through
    the library's executor (pet_run_to_gap): `workers` worker states, each on
    its own stream, the host's gap check after every epoch done in C++.
    Latency from a job's start to the host reading its last objective;
    recon_per_s over the call's wall time."""
    from paper_2106_03172_gb300.phantoms import subset_sequences
    ns = work.n_subsets
    n = work.geometry.n_pixels * work.geometry.nz
    a = alphas(work)
    seeds = np.arange(n_rec, dtype=np.uint64)[:, None] * np.uint64(1000) + np.uint64(90000) + \
        np.arange(max_epochs, dtype=np.uint64)[None, :]
    seqs = subset_sequences(seeds.ravel(), ns, ns).reshape(n_rec, max_epochs * ns)
    out = {}
    for m in METHODS:
        states = [petvr.State(prob, m, torch.zeros(n, device="cuda")) for _ in range(workers)]
        petvr.pet_run_to_gap(states, seqs[:min(n_rec, 2 * workers)], max_epochs, phi_star, GAP,
                             alpha=a[m][0], eta=a[m][1])          # graphs captured, streams warm
        t = time.perf_counter()
        epochs, gaps, ms = petvr.pet_run_to_gap(states, seqs, max_epochs, phi_star, GAP, alpha=a[m][0], eta=a[m][1])
        wall = time.perf_counter() - t
        out[m] = {"recon_per_s": int((gaps <= GAP).sum()) / wall, "p50_ms": float(np.percentile(ms, 50)),
                  "p99_ms": float(np.percentile(ms, 99)), "epochs_mean": float(np.mean(epochs)),
                  "reached": int((gaps <= GAP).sum()), "n": n_rec, "workers": workers}
    return out


# --------------------------------------------------------------------------- GPU arm

def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2106_03172_gb300 import build as _build
    from paper_2106_03172_gb300 import petvr
    from paper_2106_03172_gb300.phantoms import WORKLOADS, make_data

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the library has no CPU path)")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()
    petvr.lib()

    work = WORKLOADS[args.workload]
    geom = work.geometry
    ns = work.n_subsets
    data = make_data(work, 0)
    g_host = torch.from_numpy(data["g"].ravel()).pin_memory()
    g_dev = g_host.cuda()
    plan = petvr.Plan(geom, ns)
    if args.tuning:                                     # pinned launch shapes (e.g. for profiler runs)
        c, r = (int(x) for x in args.tuning.split(","))
        petvr.pet_plan_set_tuning(plan.handle, c, r)
        tuning = petvr.pet_plan_get_tuning(plan.handle)
        tune_src = "pinned by --tuning"
    else:
        tuning = petvr.pet_plan_autotune(plan.handle)   # launch shapes timed on this geometry
        tune_src = "pet_plan_autotune"
    prob = petvr.Problem(plan, g_dev, None, data["w"], work.beta, potential=work.potential, delta=work.delta)
    f0 = torch.empty(geom.n_pixels * geom.nz, device="cuda")
    petvr.pet_warm_start(prob.handle, f0)
    imgs = {m: f0.clone() for m in METHODS}
    states = {m: petvr.State(prob, m, imgs[m]) for m in METHODS}
    E = max(1, args.step_epochs)
    phi = torch.zeros(4, 3, dtype=torch.float64, device="cuda")          # epoch-call steps: the last objectives
    phi_run = torch.zeros(4, E, 3, dtype=torch.float64, device="cuda")   # run-call steps: every epoch's
    a = alphas(work)
    # nonzeros of one slice's A_t (a stack repeats them on every slice)
    slices = 1 if geom.multiring else geom.nz
    nnz_t = [slices * petvr.pet_plan_nnz(plan.handle, t) for t in range(ns)]
    nnz_all = slices * petvr.pet_plan_nnz(plan.handle, -1)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MiB > L2
    stream = torch.cuda.current_stream()
    rep = Replica(work)

    side = {m: torch.cuda.Stream() for m in METHODS}
    batch = petvr.Batch([states[m] for m in METHODS]) if args.batch else None

    def one_epoch(ep, concurrent=True):
        """One update epoch of each of the four independent reconstructions,
        each followed by its objective: by default each runs on its own stream
        (forked from and joined back into the timing stream); with --batch one
        persistent batched launch per phase covers all four."""
        seqs = seqs_for_step(ep, ns)
        if batch is not None and concurrent:
            batch.epoch(seqs, [a[m][0] for m in METHODS], [a[m][1] for m in METHODS], stream=stream)
            batch.objective_async(phi, stream=stream)
            return seqs
        fork = torch.cuda.Event()
        fork.record(stream)
        for i, m in enumerate(METHODS):
            s = side[m] if concurrent else stream
            s.wait_event(fork)
            states[m].epoch(seqs[i], alpha=a[m][0], eta=a[m][1], stream=s)
            petvr.pet_state_objective_async(states[m].handle, phi[i], stream=s)
        if concurrent:
            for m in METHODS:
                stream.wait_stream(side[m])
        return seqs

    step_seq_cache = {}

    def step_seqs(step):
        """Each method's subset sequence of a step's E epochs (the epochs'
        sequences back to back), made before the step is timed."""
        if step not in step_seq_cache:
            per_epoch = [seqs_for_step(step * E + e, ns) for e in range(E)]
            step_seq_cache[step] = [np.concatenate([q[i] for q in per_epoch]) for i in range(4)]
        return step_seq_cache[step]

    def one_step(step, concurrent=True):
        """One step: E update epochs of each method (epoch indices step*E ...),
        each epoch followed by its objective.  On four streams each method's
        step is one pet_state_run call (objective after every N_s updates, an
        objective's forward pass also giving the next anchor's ratios); with
        --batch, or on one stream, epoch by epoch."""
        if batch is not None or not concurrent:
            for e in range(E):
                one_epoch(step * E + e, concurrent)
            return
        seqs = step_seqs(step)
        fork = torch.cuda.Event()
        fork.record(stream)
        for i, m in enumerate(METHODS):
            side[m].wait_event(fork)
            states[m].run(seqs[i], alpha=a[m][0], eta=a[m][1], objective_every=ns, phi=phi_run[i], stream=side[m])
        for m in METHODS:
            stream.wait_stream(side[m])

    def count_step():
        """Subset forward+back pairs of the next step's E epochs (anchor passes
        included), advancing the host's update counters."""
        total = 0
        for _ in range(E):
            p, _ = rep.step_pairs()
            total += p
            rep.advance()
        return total

    for w in range(args.warmup):
        one_step(w)
        count_step()
    torch.cuda.synchronize()

    # ---- timed region (kernel-only: inputs resident in HBM)
    events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
    pairs = 0
    clocks = ClockSampler(visible_index(torch))
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = petvr.pet_kernel_launches()
    for k in range(args.steps):
        step_seqs(args.warmup + k)
        flush.zero_()
        pairs += count_step()
        events[k][0].record(stream)
        one_step(args.warmup + k)
        events[k][1].record(stream)
    torch.cuda.synchronize()
    launches = petvr.pet_kernel_launches() - launches0
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in events]
    total_ms = float(sum(step_ms))
    phi_host = (phi if args.batch else phi_run[:, E - 1, :]).cpu().numpy()
    value, total_max, pairs_all = combine_ranks(total_ms, float(pairs), device="cuda")

    # ---- where a step's time goes (after the timed region): each method's step alone on the GPU, then the
    # four together with an event at the end of each method's stream
    breakdown = None
    if batch is None:
        b0 = args.warmup + args.steps
        alone = {}
        seqs = step_seqs(b0)
        for i, m in enumerate(METHODS):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            states[m].run(seqs[i], alpha=a[m][0], eta=a[m][1], objective_every=ns, phi=phi_run[i], stream=stream)
            e1.record(stream)
            e1.synchronize()
            alone[m] = e0.elapsed_time(e1)
        count_step()
        seqs = step_seqs(b0 + 1)
        flush.zero_()
        fork = torch.cuda.Event(enable_timing=True)
        fork.record(stream)
        ends = {}
        for i, m in enumerate(METHODS):
            side[m].wait_event(fork)
            states[m].run(seqs[i], alpha=a[m][0], eta=a[m][1], objective_every=ns, phi=phi_run[i], stream=side[m])
            ends[m] = torch.cuda.Event(enable_timing=True)
            ends[m].record(side[m])
        for m in METHODS:
            stream.wait_stream(side[m])
        torch.cuda.synchronize()
        count_step()
        breakdown = {"alone_ms": alone, "together_end_ms": {m: fork.elapsed_time(ends[m]) for m in METHODS},
                     "how": "one step of each method's run call alone on the GPU, then one step of all four on "
                            "their streams with an event at the end of each (after the timed region)"}

    # ---- profiled pass: per-kernel durations for the roofline (a few epochs, methods one after another)
    n_prof = min(E, 4)
    fk, bk = (("ring_forward_kernel", "ring_back_column_kernel" if geom.nz <= 8 else "ring_back_kernel")
              if geom.multiring else
              ("forward_stack_kernel", "back_stack_kernel") if geom.nz > 1 else ("forward_tile_kernel", "back_tile_kernel"))
    bk_all = bk if (geom.multiring or geom.nz > 1) else "back_tile_wide_kernel"
    kinds_named = {0: f"{fk} (subset update, ratio)", 1: f"{bk} (update epilogue)",
                   2: f"{bk_all} (anchor, all subsets)", 3: f"{fk} (all rays: anchor/objective)"}
    alg_flops = {k: 0.0 for k in kinds_named}
    alg_bytes = {k: 0.0 for k in kinds_named}
    N, M = geom.n_pixels * geom.nz, geom.n_rays * geom.n_pairs * slices   # image and sinogram floats
    # algorithmic bytes per pixel of the fused update epilogue (4 B per float read or written):
    # OSEM f, sens_t, f_out; SVREM f, s_hat r+w, f_anc, B_t, s_anc, sens, f_out;
    # SAGA (FP32 table) f, sens_t, q_t r+w, qbar r+w, d, f_out; SVRG f, B_t, q~, d, f_out
    upd_bytes = {"osem": 12, "svrem": 32, "saga": 32, "svrg": 20}
    petvr.pet_profile_reset()
    petvr.pet_profile_enable(True)
    prof_base = (args.warmup + args.steps) * E
    for k in range(n_prof):
        flush.zero_()
        p, anchors = rep.step_pairs()
        seqs = one_epoch(prof_base + k, concurrent=False)
        for i, m in enumerate(METHODS):
            for t in seqs[i]:
                rays = plan.subset_lines(int(t)) * (1 if geom.multiring else geom.nz)
                alg_flops[0] += 2.0 * nnz_t[int(t)]
                alg_bytes[0] += 4.0 * N + 8.0 * rays
                alg_flops[1] += 2.0 * nnz_t[int(t)]
                alg_bytes[1] += 4.0 * rays + upd_bytes[m] * N
            alg_flops[3] += 2.0 * nnz_all                      # objective forward
            alg_bytes[3] += 4.0 * N + 4.0 * M
        for m in anchors:
            alg_flops[3] += 2.0 * nnz_all
            alg_bytes[3] += 4.0 * N + 8.0 * M
            alg_flops[2] += 2.0 * nnz_all
            alg_bytes[2] += 4.0 * M + 4.0 * N * ns
        rep.advance()
    torch.cuda.synchronize()
    petvr.pet_profile_enable(False)
    kinds = {}
    for kind, name in kinds_named.items():
        n, ms = petvr.pet_profile_read(kind)
        kinds[kind] = {"name": name, "launches": n, "total_ms": ms, "avg_us": 1e3 * ms / n if n else None}
    petvr.pet_profile_reset()
    tot = sum(v["total_ms"] for v in kinds.values()) or 1.0
    for v in kinds.values():
        v["share"] = v["total_ms"] / tot
    dom = max(kinds, key=lambda k: kinds[k]["total_ms"])
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    n_sms = props.multi_processor_count
    sm_mhz = sm_max_mhz()
    peak_alu = n_sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12   # TFLOP/s
    achieved = alg_flops[dom] / (kinds[dom]["total_ms"] / 1e3) / 1e12
    traffic = dram_traffic_record(dom, work.name)
    issue = ncu_issue_record(dom, work.name)
    roofline = {"bound": "alu", "kernel": kinds[dom]["name"], "achieved": achieved, "peak": peak_alu,
                "unit": "TFLOP/s", "frac": achieved / peak_alu, "traffic": traffic,
                "peak_source": f"{n_sms} SMs (this device) x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x "
                               f"{sm_mhz:g} MHz (maximum SM clock)",
                "algorithmic_bytes_per_launch": alg_bytes[dom] / max(1, kinds[dom]["launches"]),
                "hbm_achieved_gbs": alg_bytes[dom] / (kinds[dom]["total_ms"] / 1e3) / 1e9,
                "issue_active_frac": issue,
                "issue_active_source": "ncu smsp__issue_active of this kernel on this workload "
                                       "(profiles/roofline_traffic.txt; null when the sources changed since)",
                "kernels": {v["name"]: {k2: v[k2] for k2 in ("launches", "avg_us", "share")}
                            for v in kinds.values()}}
    # context for the per-launch durations above: one tiny kernel timed the same way
    # (events on both sides of a single launch on an idle stream)
    tiny = torch.zeros(1, device="cuda")
    floor = []
    for _ in range(50):
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        tiny.add_(1.0)
        t1.record(stream)
        t1.synchronize()
        floor.append(1e3 * t0.elapsed_time(t1))
    roofline["launch_floor_us"] = float(np.median(floor))
    roofline["launch_floor_how"] = ("median of 50 one-element kernels, each bracketed by events like the projector "
                                    "launches of the profiled pass")
    hbm_peak, hbm_src = measured_hbm_peak()
    roofline["hbm_peak_gbs"] = hbm_peak
    roofline["hbm_frac"] = roofline["hbm_achieved_gbs"] / hbm_peak
    roofline["hbm_peak_source"] = hbm_src

    # ---- end to end through the public API with host buffers
    img_host = torch.empty(4, geom.n_pixels * geom.nz, dtype=torch.float32).pin_memory()
    phi_step = phi if args.batch else phi_run                     # the step's objectives (every epoch's with run calls)
    phi_host_buf = torch.empty(phi_step.shape, dtype=torch.float64).pin_memory()
    # The host enqueues step after step (as a pipeline would); each step's
    # events bracket its counts upload, problem update, epochs, objectives and
    # result downloads on the device, and the L2 flush between steps stays
    # outside them.
    e2e_events = []
    e2e_pairs = 0
    e2e_base = (prof_base + n_prof + E - 1) // E
    for k in range(args.steps):
        step_seqs(e2e_base + k)
        flush.zero_()
        e2e_pairs += count_step()
        s_ev, e_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s_ev.record(stream)
        g_dev.copy_(g_host, non_blocking=True)
        petvr.pet_problem_update(prob.handle, g_dev, None, data["w"])
        one_step(e2e_base + k)
        for i, m in enumerate(METHODS):
            img_host[i].copy_(imgs[m], non_blocking=True)
        phi_host_buf.copy_(phi_step, non_blocking=True)
        e_ev.record(stream)
        e2e_events.append((s_ev, e_ev))
    torch.cuda.synchronize()
    e2e_ms = [s_ev.elapsed_time(e_ev) for s_ev, e_ev in e2e_events]
    e2e_value, _, _ = combine_ranks(float(sum(e2e_ms)), float(e2e_pairs), device="cuda")
    h2d = g_host.numel() * g_host.element_size()                     # the counts copied in every step
    d2h = img_host.numel() * img_host.element_size() + phi_host_buf.numel() * phi_host_buf.element_size()

    # ---- reconstructions to a 1e-4 relative objective gap (Phi* from the oracle)
    phi_star, phi_src = phi_star_for(work, data)
    recon = (measure_recon(torch, petvr, prob, states, imgs, work, phi_star, n_rec=args.recon)
             if phi_star is not None and args.recon > 0 else None)
    # the same with the next epoch launched before the host's check (lower latency; the speculative
    # epoch after each gap costs throughput)
    recon2 = (measure_recon(torch, petvr, prob, states, imgs, work, phi_star, n_rec=args.recon, depth=2)
              if phi_star is not None and args.recon > 0 else None)
    recon_ex = ({f"workers_{k}": recon_executor(torch, petvr, prob, work, phi_star, args.recon, k) for k in (1, 8)}
                if phi_star is not None and args.recon > 0 else None)
    recon_line = {"gap": GAP, "phi_star": phi_star, "phi_star_source": phi_src,
                  "start": "constant image + one unpenalised OSEM epoch (counted in the latency)",
                  "per_method": recon, "two_epochs_in_flight": recon2, "executor": recon_ex}

    unit = "subset fwd+back projections/s"
    legs = {}
    if rank == 0 and world == 1:
        legs = run_legs(args, torch, petvr, work, data, prob, f0, value, stream, flush)
    line = {
        "metric": "subset fwd+back projections/s and reconstructions/s to 1e-4 objective gap; p50/p99",
        "value": value, "unit": unit, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded ellipse phantom, Poisson counts)",
        "config": dict(workload_config(work, E), parallelism=f"replicas x{world}",
                       concurrency="one batch (pet_batch_epoch)" if args.batch else "four streams",
                       launch_shapes={"forward_band_chunks": tuning[0], "back_run_pixels": tuning[1],
                                      "source": tune_src}),
        "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
        "pairs_per_step": pairs / args.steps,
        "gpu_launches": int(launches),
        "clocks": clk,
        "roofline": roofline,
        "step_breakdown": breakdown,
        "e2e": {"value": e2e_value, "unit": unit, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "recon": recon_line,
        "objective_last_step": [float(x) for x in phi_host[:, 0]],
    }
    line.update(legs)
    if args.batch:      # the batched step runs epoch by epoch through pet_batch_epoch
        line["config"]["step"] = line["config"]["step"].split(";")[0] + "; one pet_batch_epoch call per epoch"
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        times, cpairs, setup = oracle_steps(work, data, 2, min_seconds=12.0)
        line["cpu_baseline"] = {
            "value": sum(cpairs) / sum(times), "unit": unit, "cores": 1, "kind": "oracle",
            "sample": f"{len(times)} epochs of each of the four methods (each followed by its objective) of the "
                      f"FP64 oracle, one thread (about {sum(times):.0f} s; system matrix build and warm start, "
                      f"{setup:.1f} s, untimed)"}
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- short legs after the headline

def _sub_bench(extra, timeout=600):
    """Run this script in a child process (same GPU, this process idle) and
    return its JSON line, or {"error": ...}."""
    cmd = [sys.executable, os.path.abspath(__file__)] + extra
    try:
        res = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout)
    except subprocess.TimeoutExpired:
        return {"error": f"timed out after {timeout} s: {' '.join(extra)}"}
    lines = [ln for ln in res.stdout.strip().splitlines() if ln.startswith("{")]
    if res.returncode != 0 or not lines:
        return {"error": f"rc={res.returncode}: {res.stderr.strip().splitlines()[-1:] or ''}"}
    return json.loads(lines[-1])


def leg_batched(torch, petvr, prob, f0, work, streams_value, stream, flush, steps=3, epochs=10, mode="phases"):
    """The same four reconstructions as one batch (pet_batch_epoch: persistent
    phases, or one dependency-driven launch per call), timed like the headline."""
    imgs = {m: f0.clone() for m in METHODS}
    states = {m: petvr.State(prob, m, imgs[m]) for m in METHODS}
    batch = petvr.Batch([states[m] for m in METHODS])
    batch.set_mode(mode)
    a = alphas(work)
    phi = torch.zeros(4, 3, dtype=torch.float64, device="cuda")
    rep = Replica(work)
    ns = work.n_subsets

    def step(k):
        pairs = 0
        for e in range(epochs):
            p, _ = rep.step_pairs()
            pairs += p
            rep.advance()
            batch.epoch(seqs_for_step(50000 + k * epochs + e, ns), [a[m][0] for m in METHODS],
                        [a[m][1] for m in METHODS], stream=stream)
            batch.objective_async(phi, stream=stream)
        return pairs

    step(0)
    torch.cuda.synchronize()
    ms, pairs = [], 0
    for k in range(1, steps + 1):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pairs += step(k)
        e1.record(stream)
        ms.append((e0, e1))
    torch.cuda.synchronize()
    batch.sync()
    total = sum(x.elapsed_time(y) for x, y in ms)
    value = pairs / (total / 1e3)
    return {"value": value, "unit": "subset fwd+back projections/s", "ms_per_epoch": total / (steps * epochs),
            "vs_four_streams": value / streams_value,
            "how": f"{steps} steps of {epochs} epochs of the four methods as one batch ({mode}), "
                   "objectives batched too; L2 flushed between steps"}


def leg_parity(torch, petvr, work, data, prob):
    """Untimed checker: the FP64 oracle on this workload from the same start,
    against the GPU, per result: the warm start, then for each method the
    first update and one epoch (relative L2) and the objective after it."""
    from oracle import em
    from oracle.em import build_problem
    from paper_2106_03172_gb300.phantoms import subset_sequence
    t0 = time.perf_counter()
    ora = build_problem(work.geometry, data["g"], data["w"], work.n_subsets, work.beta, work.potential, work.delta)
    f0_ora = ora.initial_image()
    geom, ns = work.geometry, work.n_subsets
    f0 = torch.empty(geom.n_pixels * geom.nz, device="cuda")
    petvr.pet_warm_start(prob.handle, f0)
    torch.cuda.synchronize()
    got0 = f0.double().cpu().numpy().reshape(f0_ora.shape)

    def rel(x, y):
        return float(np.linalg.norm(x - y) / np.linalg.norm(y))

    out = {"warm_start": rel(got0, f0_ora)}
    f_start = got0                                      # both sides continue from the GPU's FP32 warm start
    a = alphas(work)
    seq = subset_sequence(2000, ns, ns)
    for label, m, table in (("osem", "osem", "fp32"), ("svrem", "svrem", "fp32"), ("saga", "saga", "fp32"),
                            ("saga_bf16", "saga", "bf16"), ("svrg", "svrg", "fp32")):
        img = torch.from_numpy(f_start.astype(np.float32).ravel()).cuda()
        st = petvr.State(prob, m, img, table=table)
        alg = {"osem": None, "svrem": lambda: em.SVREM(ora, f_start, *a["svrem"]),
               "saga": lambda: em.SAGA(ora, f_start, a["saga"][0], table=table),
               "svrg": lambda: em.SVRG(ora, f_start, *a["svrg"])}[m]
        alg = alg() if alg else None
        f = f_start
        errs = []
        for t in seq:
            st.epoch([int(t)], alpha=a[m][0], eta=a[m][1])
            f = em.osem_step(ora, f, int(t)) if alg is None else alg.step(int(t))
            torch.cuda.synchronize()
            errs.append(rel(img.double().cpu().numpy().reshape(f.shape), f))
        phi_gpu = petvr.pet_objective(prob.handle, img)
        phi_ora = ora.objective(f)
        out[label] = {"first_update": errs[0], "epoch_max": max(errs), "epoch_end": errs[-1],
                      "phi_rel": abs(phi_gpu - phi_ora) / abs(phi_ora)}
    out["how"] = ("FP64 oracle (oracle/) from the GPU's FP32 warm start, the same subset sequence; relative L2 of "
                  "every iterate of one epoch against the oracle's, |dPhi|/|Phi| at its end; BF16 table against "
                  "the oracle's BF16 rounding")
    out["seconds"] = round(time.perf_counter() - t0, 1)
    return out


def run_legs(args, torch, petvr, work, data, prob, f0, streams_value, stream, flush):
    """Short measurements after the headline, each reported under its own key."""
    want = set() if args.legs == "none" else {x.strip() for x in args.legs.split(",") if x.strip()}
    legs = {}
    if "batched" in want and not work.geometry.multiring and work.geometry.nz == 1:
        legs["batched_four_methods"] = {
            mode: leg_batched(torch, petvr, prob, f0, work, streams_value, stream, flush, mode=mode)
            for mode in ("phases", "dataflow", "streams")}
    if "batch64" in want:
        legs["batch64"] = _sub_bench(["--workload", "batch64", "--steps", "3", "--warmup", "1"])
    if "stack" in want:
        sub = _sub_bench(["--workload", "c128x47", "--steps", "3", "--warmup", "1", "--step-epochs", "2",
                          "--legs", "none", "--no-cpu-baseline", "--recon", "0"])
        legs["c128x47"] = {k: sub.get(k) for k in ("value", "unit", "ms_per_step", "error") if k in sub}
        if "roofline" in sub:
            legs["c128x47"]["roofline_frac"] = sub["roofline"].get("frac")
            legs["c128x47"]["achieved_tflops"] = sub["roofline"].get("achieved")
    if "ring" in want:
        sub = _sub_bench(["--workload", "ring2_128", "--steps", "3", "--warmup", "1", "--step-epochs", "2",
                          "--legs", "none", "--no-cpu-baseline", "--recon", "0"])
        legs["ring2_128"] = {k: sub.get(k) for k in ("value", "unit", "ms_per_step", "error") if k in sub}
        if "roofline" in sub:
            legs["ring2_128"]["roofline_frac"] = sub["roofline"].get("frac")
            legs["ring2_128"]["achieved_tflops"] = sub["roofline"].get("achieved")
    if "serve" in want:
        sub = _sub_bench(["--workload", "serve", "--requests", "192", "--distinct"])
        leg = {k: sub.get(k) for k in ("value", "unit", "latency", "speedup_vs_plain", "p50_speedup_vs_plain",
                                       "bit_identical_to_plain", "error") if k in sub}
        if "plain" in sub:
            leg["plain_latency"] = sub["plain"]["latency"]
        if "native_loop" in sub:
            leg["native_loop_latency"] = sub["native_loop"]["latency"]
        if "config" in sub:
            leg["requests"] = sub["config"].get("workload")
        legs["serve_distinct192"] = leg
    if "parity" in want:
        legs["parity_vs_oracle"] = leg_parity(torch, petvr, work, data, prob)
    return legs


def run_batch64(args):
    """Batched form: 64 independent SAGA reconstructions (BF16 table) of mixed
    sizes; one step = 21 updates of every member plus its objective, all
    members in one launch per phase, against the same work run member by
    member on one stream."""
    import torch

    from paper_2106_03172_gb300 import build as _build
    from paper_2106_03172_gb300 import petvr
    from paper_2106_03172_gb300.phantoms import batched_workloads, make_data, subset_sequence

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    _build.build()
    petvr.lib()
    works = batched_workloads(0, 64)
    members = []
    for i, w in enumerate(works):
        data = make_data(w, 100 + i)
        plan = petvr.Plan(w.geometry, w.n_subsets)
        petvr.pet_plan_autotune(plan.handle)
        prob = petvr.Problem(plan, torch.from_numpy(data["g"].ravel()).cuda(), None, data["w"], w.beta)
        img = torch.empty(w.geometry.n_pixels, device="cuda")
        petvr.pet_warm_start(prob.handle, img)
        solo_img, df_img, st_img = img.clone(), img.clone(), img.clone()
        members.append({"work": w, "plan": plan, "prob": prob, "img": img, "solo_img": solo_img, "df_img": df_img,
                        "st_img": st_img,
                        "state": petvr.State(prob, "saga", img, table="bf16"),
                        "solo": petvr.State(prob, "saga", solo_img, table="bf16"),
                        "df": petvr.State(prob, "saga", df_img, table="bf16"),
                        "st": petvr.State(prob, "saga", st_img, table="bf16")})
    batch = petvr.Batch([m["state"] for m in members])
    batch_df = petvr.Batch([m["df"] for m in members])
    batch_df.set_mode("dataflow")
    n_iter = 21
    phi = torch.zeros(len(members), 3, dtype=torch.float64, device="cuda")
    phi_solo = torch.zeros(len(members), 3, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def seqs(step):
        return [subset_sequence(7000 + 100 * step + j, m["work"].n_subsets, n_iter) for j, m in enumerate(members)]

    def step_batched(step):
        batch.epoch(seqs(step), [1.0] * len(members), [1] * len(members), stream=stream)
        batch.objective_async(phi, stream=stream)

    def step_dataflow(step):
        batch_df.epoch(seqs(step), [1.0] * len(members), [1] * len(members), stream=stream)
        batch_df.objective_async(phi, stream=stream)

    def step_solo(step):
        for j, (m, q) in enumerate(zip(members, seqs(step))):
            m["solo"].epoch(q, alpha=1.0, stream=stream)
            m["solo"].objective_async(phi_solo[j], stream=stream)

    batch_st = petvr.Batch([m["st"] for m in members])
    batch_st.set_mode("streams")
    phi_st = torch.zeros(len(members), 3, dtype=torch.float64, device="cuda")

    def step_streams(step):
        """The same batch in PET_BATCH_STREAMS mode: the members' own epoch calls on the batch's streams."""
        batch_st.epoch(seqs(step), [1.0] * len(members), [1] * len(members), stream=stream)
        batch_st.objective_async(phi_st, stream=stream)

    def timed(fn, offset):
        for w in range(args.warmup):
            fn(offset + w)
        torch.cuda.synchronize()
        ms = []
        for k in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(offset + args.warmup + k)
            e1.record(stream)
            ms.append((e0, e1))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ms]

    launches0 = petvr.pet_kernel_launches()
    clocks = ClockSampler(visible_index(torch))
    clocks.start()
    t_batch = timed(step_batched, 0)
    clk = clocks.stop()
    launches = petvr.pet_kernel_launches() - launches0
    t_solo = timed(step_solo, 0)
    t_df = timed(step_dataflow, 0)
    t_st = timed(step_streams, 0)
    batch_df.sync()
    # same subset sequences in all runs: the results must agree bit for bit
    torch.cuda.synchronize()
    same = all(torch.equal(m["img"], m["solo_img"]) and torch.equal(m["df_img"], m["solo_img"])
               and torch.equal(m["st_img"], m["solo_img"]) for m in members)
    pairs_step = len(members) * n_iter
    value = pairs_step * args.steps / (sum(t_batch) / 1e3)
    # algorithmic work of the timed steps: 2 nnz(A_t) per update (forward + back), nnz(A) per objective
    nnz_steps = 0
    for k in range(args.steps):
        for m, q in zip(members, seqs(args.warmup + k)):
            nz_t = [petvr.pet_plan_nnz(m["plan"].handle, t) for t in range(m["work"].n_subsets)]
            nnz_steps += sum(2 * nz_t[int(t)] for t in q) + petvr.pet_plan_nnz(m["plan"].handle, -1)
    flops = 2.0 * nnz_steps / (sum(t_batch) / 1e3) / 1e12
    solo_value = pairs_step * args.steps / (sum(t_solo) / 1e3)
    sizes = sorted({m["work"].geometry.nx for m in members})
    line = {
        "metric": "subset fwd+back projections/s and reconstructions/s to 1e-4 objective gap; p50/p99",
        "value": value, "unit": "subset fwd+back projections/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(np.mean(t_batch)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (bf16 SAGA table)",
        "data": "synthetic (seeded ellipse phantoms, Poisson counts)",
        "config": {"workload": f"batch64: 64 SAGA reconstructions (BF16 table, alpha 1), images "
                               f"{'/'.join(str(x) for x in sizes)} px square, views round(1.4 N), bins ~1.43 N, "
                               "counts 1e5-1e7 log-uniform, 6/12/21 subsets; step = 21 updates of every member "
                               "+ its FP64 objective",
                   "l2": "flushed between steps (256 MiB write outside the timed events)"},
        "p50_ms": float(np.percentile(t_batch, 50)), "p99_ms": float(np.percentile(t_batch, 99)),
        "gpu_launches": int(launches), "clocks": clk,
        "sequential": {"value": solo_value, "ms_per_step": float(np.mean(t_solo)),
                       "how": "the same 64 states stepped one after another on one stream (graph per state)"},
        "speedup_vs_sequential": value / solo_value,
        "dataflow": {"value": pairs_step * args.steps / (sum(t_df) / 1e3), "ms_per_step": float(np.mean(t_df)),
                     "how": "the same batch as one dependency-driven launch per call (pet_batch_set_mode dataflow)"},
        "streams": {"value": pairs_step * args.steps / (sum(t_st) / 1e3), "ms_per_step": float(np.mean(t_st)),
                    "how": "the same batch in PET_BATCH_STREAMS mode: the members' own epoch calls (captured graphs) "
                           "on the batch's 8 streams"},
        "algorithmic": {"nonzeros_per_step": nnz_steps / args.steps, "achieved_tflops": flops,
                        "note": "2 flops per system-matrix nonzero per projection"},
        "bit_identical_to_sequential": bool(same),
    }
    if args.recon > 0:
        line["recon"] = batch64_recon(torch, petvr, works, [make_data(w, 100 + i) for i, w in enumerate(works)])
    print(json.dumps(line), flush=True)
    return 0


def batch64_recon(torch, petvr, works, datas, max_epochs=200):
    """Reconstructions of the 64 members to the 1e-4 relative gap (each
    against its own Phi* from the FP64 oracle, tests/golden/phi_star.json):
    all 64 admitted at once and advanced as one batch (serving.Server, three
    updates per tick, objectives checked every epoch), against the plain
    per-reconstruction path, one member after another (serve_plain).  Both
    return the same image for every member."""
    import hashlib

    from paper_2106_03172_gb300.serving import Request, Server, latency_summary, serve_plain
    golden = json.load(open(os.path.join(ROOT, "tests", "golden", "phi_star.json")))
    phis = []
    for i, d in enumerate(datas):
        ent = golden.get(f"batch64_{i}")
        sha = hashlib.sha256(d["g"].astype("<f4").tobytes()).hexdigest()
        if not ent or ent["counts_sha256"] != sha:
            return {"unavailable": f"no stored Phi* for member {i} (tests/golden/make_phi_star.py batch64_0-64)"}
        phis.append(ent["phi_star"])

    def requests():
        return [Request(i, w, d["g"], d["w"], phi, arrival=0.0, seed=9000 + i, algo="saga")
                for i, (w, d, phi) in enumerate(zip(works, datas, phis))]

    srv = Server(budget_bytes=16 << 30, max_slots=64, gap=GAP, max_epochs=max_epochs, tick=3, window=4)
    srv.prepare(works)
    torch.cuda.synchronize()
    done = srv.serve(requests())
    plain = serve_plain(requests(), gap=GAP, max_epochs=max_epochs)
    same = all(x.epochs == y.epochs and np.array_equal(x.image, y.image) for x, y in zip(done, plain))
    b, p = latency_summary(done), latency_summary(plain)
    ex = batch64_executor(torch, petvr, works, datas, phis, plain, max_epochs)
    return {"gap": GAP, "batched": b, "plain": p, "speedup_reached_per_s": b["reached_per_s"] / p["reached_per_s"],
            "executor": ex,
            "bit_identical_to_plain": bool(same),
            "how": "64 SAGA (BF16 table) reconstructions from their warm starts, all arriving at once: one batch "
                   "(serving.Server: 3 updates per tick, host check every 4 ticks) against one after another "
                   "through each member's own epochs (serve_plain); Phi* per member from the FP64 oracle"}


def batch64_executor(torch, petvr, works, datas, phis, plain, max_epochs, n_streams=8):
    """The same 64 reconstructions (same subset sequences and launch shapes)
    through the library's executor for jobs with their own states
    (pet_run_jobs_to_gap), up to n_streams at a time; a first call captures
    the states' graphs, the second is timed on the host clock."""
    from paper_2106_03172_gb300.phantoms import subset_sequence
    from paper_2106_03172_gb300.serving import tuned_plan
    keep, states, seqs = [], [], []
    for i, (w, d) in enumerate(zip(works, datas)):
        plan = tuned_plan(w)
        prob = petvr.Problem(plan, torch.from_numpy(np.ascontiguousarray(d["g"]).ravel()).cuda(), None, d["w"],
                             w.beta)
        st = petvr.State(prob, "saga", torch.zeros(w.geometry.n_pixels, device="cuda"), table="bf16")
        keep.append((plan, prob))
        states.append(st)
        seqs.append(subset_sequence(9000 + i, w.n_subsets, max_epochs * w.n_subsets))
    n = len(states)
    args = (states, seqs, [1.0] * n, [1] * n, phis, max_epochs, GAP)
    petvr.pet_run_jobs_to_gap(*args, n_streams=n_streams)
    t = time.perf_counter()
    epochs, gaps, ms = petvr.pet_run_jobs_to_gap(*args, n_streams=n_streams)
    wall = time.perf_counter() - t
    same = all(int(e) == r.epochs and np.array_equal(st.img.cpu().numpy(), r.image)
               for e, st, r in zip(epochs, states, plain))
    reached = int((gaps <= GAP).sum())
    return {"reached_per_s": reached / wall, "reached_gap": reached, "completed": n,
            "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
            "epochs_mean": float(np.mean(epochs)), "streams": n_streams, "bit_identical_to_plain": bool(same),
            "how": "pet_run_jobs_to_gap: each member on its own state, up to 8 at a time on their own streams, the "
                   "host's gap check in C++; latency from a job's start (all 64 queued at once)"}


def _server_stats(srv):
    st = srv.stats
    return {"max_active": st.max_active, "admissions_deferred": st.admissions_deferred,
            "peak_bytes": st.peak_bytes, "slots_created": st.slots_created, "slots_reused": st.slots_reused,
            "slots_released": st.slots_released, "ticks": st.ticks, "batches_built": st.batches_built,
            "epochs_launched": st.epochs_launched}


def run_serve(args):
    """Serving: an open-loop Poisson stream of SVREM/SAGA requests, image size
    uniform in 128^2-512^2, counts log-uniform in 1e6-1e8, 6/12/21 subsets,
    each stopped at a relative objective gap of 1e-4 against the FP64
    oracle's Phi* of its data; continuous batching with admission by
    device-memory budget, against the same stream served one request at a
    time through the plain per-reconstruction path.  By default requests are
    drawn from twelve templates (phantom and counts shared by a template's
    requests, which differ in their subset sequences); with --distinct every
    request has its own phantom and counts (as many requests as have a stored
    Phi*)."""
    import hashlib

    import torch

    from paper_2106_03172_gb300 import build as _build
    from paper_2106_03172_gb300 import petvr
    from paper_2106_03172_gb300.phantoms import make_data, serving_pool, serving_requests
    from paper_2106_03172_gb300.serving import (Request, Server, StreamServer, latency_summary, per_template,
                                                serve_native, serve_plain)

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    _build.build()
    petvr.lib()
    golden = json.load(open(os.path.join(ROOT, "tests", "golden", "phi_star.json")))

    def with_phi_star(w, seed):
        data = make_data(w, seed)
        ent = golden.get(w.name)
        sha = hashlib.sha256(data["g"].astype("<f4").tobytes()).hexdigest()
        return (w, data, ent["phi_star"]) if ent and ent["counts_sha256"] == sha else None

    rng = np.random.default_rng(77)
    n_req = args.requests
    pool, skipped = [], []
    if args.distinct:
        # every request its own phantom and counts: the first n_req requests of
        # the distinct stream, each with the oracle's Phi* of its own data
        for w, seed in serving_requests(n_req):
            ent = with_phi_star(w, seed)
            if ent is None:
                skipped.append(w.name)
            else:
                pool.append(ent)
        n_req = len(pool)
        picks = list(range(n_req))
        arrivals = np.cumsum(rng.exponential(1.0 / args.rate, n_req))
    else:
        for w in serving_pool():
            ent = with_phi_star(w, 0)
            if ent is None:
                skipped.append(w.name)
            else:
                pool.append(ent)
        arrivals = np.cumsum(rng.exponential(1.0 / args.rate, n_req))
        # image size uniform over the pool's sizes, then a template of that size
        by_size = {}
        for k, (w, _, _) in enumerate(pool):
            by_size.setdefault(w.geometry.nx, []).append(k)
        size_keys = sorted(by_size)
        picks = []
        for _ in range(n_req):
            group = by_size[size_keys[int(rng.integers(len(size_keys)))]]
            picks.append(group[int(rng.integers(len(group)))])
    if n_req == 0:
        print(json.dumps({"metric": "reconstructions/s to 1e-4 objective gap", "value": None,
                          "error": f"no request has a stored Phi* (missing: {', '.join(skipped[:8])})"}), flush=True)
        return 1

    def requests():
        return [Request(i, pool[k][0], pool[k][1]["g"], pool[k][1]["w"], pool[k][2], arrival=float(t),
                        seed=5000 + i) for i, (t, k) in enumerate(zip(arrivals, picks))]

    budget = int(args.budget_gib * (1 << 30))
    me = args.max_epochs
    servers = {"streams": lambda: StreamServer(budget_bytes=budget, max_slots=64, gap=GAP, max_epochs=me,
                                               depth=args.depth),
               "batch": lambda: Server(budget_bytes=budget, max_slots=64, gap=GAP, max_epochs=me, tick=3,
                                       window=args.window)}
    order = ([args.server] if args.server in servers else []) + [k for k in servers if k != args.server]
    runs = {}
    for kind in order:
        srv = servers[kind]()
        srv.prepare([w for w, _, _ in pool])
        clocks = ClockSampler(visible_index(torch))
        launches0 = petvr.pet_kernel_launches()
        clocks.start()
        done = srv.serve(requests())
        clk = clocks.stop()
        runs[kind] = (srv, done, clk, petvr.pet_kernel_launches() - launches0)
        del srv
    # the same stream through the library's own serving loop (pet_serve_requests, same budget)
    clocks = ClockSampler(visible_index(torch))
    launches0 = petvr.pet_kernel_launches()
    clocks.start()
    native_done, native_stats = serve_native(requests(), gap=GAP, max_epochs=args.max_epochs, n_streams=64,
                                             budget_bytes=budget)
    runs["native"] = (None, native_done, clocks.stop(), petvr.pet_kernel_launches() - launches0)
    native = latency_summary(native_done)
    srv, done, clk, launches = runs[args.server]
    summ = latency_summary(done)
    # the same stream through the plain per-reconstruction path, one request at a time
    plain = serve_plain(requests(), gap=GAP, max_epochs=args.max_epochs)
    plain_summ = latency_summary(plain)
    same = all(a.epochs == b.epochs and np.array_equal(a.image, b.image)
               for d in [r[1] for r in runs.values()] for a, b in zip(d, plain))
    sizes = sorted({w.geometry.nx for w, _, _ in pool})
    others = [k for k in ("streams", "batch") if k != args.server]
    line = {
        "metric": "subset fwd+back projections/s and reconstructions/s to 1e-4 objective gap; p50/p99",
        "value": summ["reached_per_s"], "unit": "reconstructions/s", "n_gpus": 1, "steps": n_req, "warmup": 0,
        "ms_per_step": summ["p50_ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (bf16 SAGA tables)", "data": "synthetic (seeded ellipse phantoms, Poisson counts)",
        "config": {"workload": (f"serve: {n_req} distinct requests (own phantom and counts, log-uniform "
                                f"1e6-1e8), Poisson arrivals at {args.rate:g}/s, "
                                if args.distinct else
                                f"serve: {n_req} requests, Poisson arrivals at {args.rate:g}/s, templates "
                                f"{', '.join(w.name for w, _, _ in pool)} ")
                               + f"({'/'.join(f'{n}^2' for n in sizes)}, SVREM/SAGA), "
                               f"stop at relative gap {GAP:g} against the oracle's Phi*",
                   "requests": "distinct" if args.distinct else "templates",
                   "server": args.server, "budget_gib": args.budget_gib, "max_slots": 64, "max_epochs": me,
                   "streams_depth_epochs": args.depth, "batch_tick_updates": 3, "batch_window_ticks": args.window,
                   "without_phi_star": skipped},
        "latency": summ, "gpu_launches": int(launches), "clocks": clk,
        "plain": {"latency": plain_summ, "how": "the same requests one at a time in arrival order, each "
                  "through its own State epochs (captured graphs), objective after every epoch"},
        "per_template": per_template(done),
        "speedup_vs_plain": summ["reached_per_s"] / plain_summ["reached_per_s"],
        "p50_speedup_vs_plain": plain_summ["p50_ms"] / summ["p50_ms"],
        "bit_identical_to_plain": bool(same),
        "server_stats": native_stats if srv is None else _server_stats(srv),
        "other_servers": {k: {"latency": latency_summary(runs[k][1]), "stats": _server_stats(runs[k][0])}
                          for k in others},
        "native_loop": {"latency": native, "stats": native_stats,
                        "how": "pet_serve_requests: the whole loop in C++, each request admitted once it has arrived, "
                               "one of 64 streams is free and its slot fits the same device-memory budget"},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- convergence comparison

# (label, state algorithm, alpha0, eta, step decay): the paper's methods and
# non-variance-reduced baselines (§5.1) with the step sizes of the workload
# (alpha_k = alpha0 / (decay k + 1) for SGA, BSREM and SEM)
def converge_methods(work):
    return [("OSEM", "osem", 1.0, 1, 0.0), ("SVREM", "svrem", work.alpha_svrem, work.eta_svrem, 0.0),
            ("SAGA", "saga", work.alpha_saga, 1, 0.0), ("SVRG", "svrg", work.alpha_svrg, work.eta_svrg, 0.0),
            ("SGA", "sga", 1.0, 1, 0.0), ("BSREM", "sga", 1.0, 1, 0.001), ("SEM", "sem", 1.0, 1, 0.001),
            ("SAGA-EM", "sagaem", work.alpha_svrem, 1, 0.0)]


def run_converge(args):
    """Relative objective gap (Phi* - Phi(f_k)) / |Phi*| after every update
    epoch for every method, from the same warm start and subset sequences on
    the GPU, beside the passes over the data each has made (anchor passes and
    table fills counted as the paper counts epochs).  A synthetic counterpart
    of the paper's convergence comparisons (§5)."""
    import torch

    from paper_2106_03172_gb300 import build as _build
    from paper_2106_03172_gb300 import petvr
    from paper_2106_03172_gb300.phantoms import WORKLOADS, make_data, subset_sequence

    _build.build()
    petvr.lib()
    work = WORKLOADS[args.on]
    data = make_data(work, 0)
    phi_star, phi_src = phi_star_for(work, data)
    if phi_star is None:
        print(json.dumps({"workload": f"converge on {work.name}", "unavailable": phi_src}), flush=True)
        return 0
    geom, ns = work.geometry, work.n_subsets
    plan = petvr.Plan(geom, ns)
    petvr.pet_plan_autotune(plan.handle)
    prob = petvr.Problem(plan, torch.from_numpy(data["g"].ravel()).cuda(), None, data["w"], work.beta,
                         potential=work.potential, delta=work.delta)
    f0 = torch.empty(geom.n_pixels * geom.nz, device="cuda")
    petvr.pet_warm_start(prob.handle, f0)
    phi = torch.zeros(args.epochs, 3, dtype=torch.float64, device="cuda")
    out = {}
    for label, algo, alpha, eta, decay in converge_methods(work):
        img = f0.clone()
        state = petvr.State(prob, algo, img)
        passes, p = [], 1.0 if algo in ("saga", "sagaem") else 0.0     # table fill at creation
        if algo == "sem":
            p = 1.0                                                     # s(f0) on the first call
        t0 = time.perf_counter()
        for e in range(args.epochs):
            state.epoch(subset_sequence(70000 + e, ns, ns), alpha=alpha, eta=eta, decay=decay)
            state.objective_async(phi[e])
            p += 1.0 + (1.0 if algo in ("svrem", "svrg") and e % eta == 0 else 0.0)
            passes.append(p)
        torch.cuda.synchronize()
        gaps = [(phi_star - float(x)) / abs(phi_star) for x in phi[:, 0].cpu().numpy()]
        first = next((i + 1 for i, g in enumerate(gaps) if g <= GAP), None)
        out[label] = {"gap": gaps, "passes": passes, "epochs_to_gap": first,
                      "alpha0": alpha, "eta": eta, "decay": decay, "wall_s": time.perf_counter() - t0}
    line = {"workload": f"converge on {work.name}", "phi_star": phi_star, "phi_star_source": phi_src,
            "gap_target": GAP, "epochs": args.epochs, "start": "constant image + one unpenalised OSEM epoch",
            "subsets": "uniform with replacement, seeded (the same sequence for every method)",
            "methods": out}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_batch64(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "converge":
        return run_converge(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
