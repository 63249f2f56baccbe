"""Write tests/golden/phi_star.json: the MAP objective Phi* of the named
workloads (seed 0) from the FP64 oracle's L-BFGS-B solve, with a SHA-256 of
the generated counts so a consumer can tell whether its inputs are the ones
these values belong to.  Calls only the oracle and the input generator.

    python tests/golden/make_phi_star.py [workload ...]

The members of the 64-reconstruction batch (batched_workloads(0, 64), member j
with data seed 100 + j) are named batch64_<j>; ``batch64_<a>-<b>`` solves
members a..b-1.  The distinct requests of the serving stream
(serving_requests, request i with data seed 20000 + i) are named req<i>, and
``req_<a>-<b>`` solves requests a..b-1.
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.em import build_problem, map_reference  # noqa: E402
from paper_2106_03172_gb300.phantoms import (WORKLOADS, batched_workloads, make_data, serving_pool,  # noqa: E402
                                            serving_requests)

OUT = os.path.join(HERE, "phi_star.json")


def counts_sha256(g) -> str:
    return hashlib.sha256(g.astype("<f4").tobytes()).hexdigest()


SERVING_POOL = {w.name: w for w in serving_pool()}


def _store(name, entry):
    """Merge one entry into the table under an exclusive lock (re-read just
    before writing, so that solves run side by side keep each other's
    entries)."""
    import fcntl
    with open(f"{OUT}.lock", "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        table = json.load(open(OUT)) if os.path.exists(OUT) else {}
        table[name] = entry
        tmp = f"{OUT}.{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, OUT)


BATCH64 = batched_workloads(0, 64)


def _expand(names):
    out = []
    for name in names:
        if name.startswith("batch64_") and "-" in name:
            a, b = name[len("batch64_"):].split("-")
            out += [f"batch64_{j}" for j in range(int(a), int(b))]
        elif name.startswith("req_") and "-" in name:
            a, b = name[len("req_"):].split("-")
            out += [f"req{j}" for j in range(int(a), int(b))]
        else:
            out.append(name)
    return out


def _workload(name):
    """(workload, data seed) of a name."""
    if name.startswith("batch64_"):
        j = int(name[len("batch64_"):])
        return BATCH64[j], 100 + j
    if name.startswith("req") and name[3:].isdigit():
        return serving_requests(int(name[3:]) + 1)[-1]
    return WORKLOADS.get(name) or SERVING_POOL[name], 0


def main(names):
    for name in _expand(names):
        work, seed = _workload(name)
        data = make_data(work, seed)
        prob = build_problem(work.geometry, data["g"], data["w"], work.n_subsets, work.beta, work.potential, work.delta)
        t = time.time()
        _, phi, kkt = map_reference(prob)
        entry = {"seed": seed, "phi_star": phi, "kkt_residual": kkt,
                 "counts_sha256": counts_sha256(data["g"]),
                 "solver": "scipy L-BFGS-B on the FP64 oracle objective",
                 "seconds": round(time.time() - t, 1)}
        print(name, entry, flush=True)
        _store(name, entry)


if __name__ == "__main__":
    main(sys.argv[1:] or ["c64", "c256"] + sorted(SERVING_POOL))
