"""Host-side bookkeeping of the servers (CPU): latency and rate summaries,
per-template tallies, and the launch-shape cache key."""
import math

import numpy as np
import pytest

pytest.importorskip("torch")

from paper_2106_03172_gb300 import serving  # noqa: E402
from paper_2106_03172_gb300.phantoms import Geometry, Workload  # noqa: E402


def _req(rid, work, arrival, admitted, done, epochs, reached, algo="saga"):
    r = serving.Request(rid, work, np.zeros(1, np.float32), 0.1, -1.0, arrival, algo=algo)
    r.admitted, r.done, r.epochs, r.reached = admitted, done, epochs, reached
    return r


def test_latency_summary_and_per_template():
    wa = Workload("ta", Geometry(16, 16, 8, 23), n_subsets=4, counts=1e5, bg_frac=0.1, beta=0.01, n_ellipses=3)
    wb = Workload("tb", Geometry(32, 32, 8, 45), n_subsets=6, counts=1e5, bg_frac=0.1, beta=0.01, n_ellipses=3)
    reqs = [_req(0, wa, 0.0, 0.0, 1.0, 3, True), _req(1, wa, 0.5, 1.0, 2.5, 5, True),
            _req(2, wb, 1.0, 1.5, 3.0, 8, False, algo="svrem"), _req(3, wb, 2.0, 2.0, 4.0, 4, True, algo="svrem")]
    s = serving.latency_summary(reqs)
    lat = np.array([1.0, 2.0, 2.0, 2.0])
    assert s["completed"] == 4 and s["reached_gap"] == 3
    assert math.isclose(s["p50_ms"], 1e3 * np.percentile(lat, 50))
    assert math.isclose(s["p99_ms"], 1e3 * np.percentile(lat, 99))
    assert math.isclose(s["mean_wait_ms"], 1e3 * np.mean([0.0, 0.5, 0.5, 0.0]))
    assert math.isclose(s["recon_per_s"], 4 / 4.0) and math.isclose(s["reached_per_s"], 3 / 4.0)
    assert math.isclose(s["epochs_mean"], 5.0)
    t = serving.per_template(reqs)
    assert t["ta"] == {"requests": 2, "reached": 2, "epochs": 4.0, "algo": "saga", "size": 16, "subsets": 4}
    assert t["tb"] == {"requests": 2, "reached": 1, "epochs": 6.0, "algo": "svrem", "size": 32, "subsets": 6}


def test_plan_key_is_the_request_shape():
    """Plans (and their launch shapes) are shared by requests of one geometry
    and subset count, whatever their counts, method or penalty."""
    a = Workload("a", Geometry(64, 64, 90, 91), n_subsets=6, counts=1e6, bg_frac=0.1, beta=0.01, n_ellipses=8,
                 methods=("saga",))
    b = Workload("b", Geometry(64, 64, 90, 91), n_subsets=6, counts=5e7, bg_frac=0.2, beta=0.002, n_ellipses=4,
                 methods=("svrem",))
    c = Workload("c", Geometry(64, 64, 90, 91), n_subsets=12, counts=1e6, bg_frac=0.1, beta=0.01, n_ellipses=8)
    key = serving._Base._plan_key
    assert key(a) == key(b) != key(c)
