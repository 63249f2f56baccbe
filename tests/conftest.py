import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_collection_modifyitems(config, items):
    """GPU tests need CUDA; on a machine without it they are skipped (the CPU
    suite runs with -m "not gpu" anyway)."""
    try:
        import torch
        has_cuda = torch.cuda.is_available()
    except Exception:
        has_cuda = False
    if has_cuda:
        from paper_2106_03172_gb300 import build
        build.build()
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def tiny_geom():
    from paper_2106_03172_gb300.phantoms import Geometry
    return Geometry(16, 16, 24, 23)


def tiny_problem(geom, seed=0, n_subsets=4, beta=0.05, counts=2e4, bg_frac=0.1,
                 potential="quadratic", delta=1.0, w_zero=False):
    """Small seeded problem for oracle pins (ellipse phantom, Poisson data)."""
    from oracle.em import build_problem
    from paper_2106_03172_gb300.phantoms import Workload, make_data
    work = Workload("tiny", geom, n_subsets=n_subsets, counts=counts, bg_frac=bg_frac,
                    beta=beta, n_ellipses=3)
    data = make_data(work, seed)
    w = 0.0 if w_zero else data["w"]
    return build_problem(geom, data["g"], w, n_subsets, beta, potential, delta), data


# Measured errors of the GPU results against the FP64 oracle, one record per
# result (test, case, method, table type, quantity, value).  Written at the end
# of the session to the file named by PETVR_ERROR_RECORD, when it is set.
_ERROR_RECORDS = []


@pytest.fixture(scope="session")
def record_error():
    def record(**fields):
        _ERROR_RECORDS.append({k: (float(v) if isinstance(v, (np.floating, float)) else v)
                               for k, v in fields.items()})
    return record


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("PETVR_ERROR_RECORD")
    if path and _ERROR_RECORDS:
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        with open(path, "w") as f:
            json.dump(_ERROR_RECORDS, f, indent=0)
