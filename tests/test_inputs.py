"""Seeded input generators (CPU only) and the code-independence rule."""
import math
import os
import re

import numpy as np
import pytest

from paper_2106_03172_gb300.phantoms import (WORKLOADS, Ellipse, Geometry, analytic_sinogram,
                                             make_data, splitmix64, subset_sequence)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_splitmix64_published_vector():
    # reference outputs of SplitMix64 seeded with 1234567 (Vigna's test vector)
    assert splitmix64(1234567, 3) == [6457827717110365317, 3203168211198807973,
                                      9817491932198370423]


def test_subset_sequence_uniform():
    seq = subset_sequence(2000, 21, 21000)
    assert seq.min() == 0 and seq.max() == 20
    counts = np.bincount(seq, minlength=21)
    assert np.all(np.abs(counts - 1000) < 150)
    assert np.array_equal(seq, subset_sequence(2000, 21, 21000))


def test_ellipse_projection_closed_form_vs_quadrature():
    """The analytic chord of a rotated ellipse agrees with numerical
    integration of its indicator along the line."""
    geom = Geometry(32, 32, 7, 15, pixel_mm=2.0, bin_mm=3.0)
    e = Ellipse(3.0, -2.0, 14.0, 6.0, 0.4, 1.7)
    sino = analytic_sinogram([e], geom)
    tt = np.linspace(-60, 60, 400001)
    dt = tt[1] - tt[0]
    for i in range(geom.n_angles):
        th = i * math.pi / geom.n_angles
        for j in range(geom.n_bins):
            s = (j - 0.5 * (geom.n_bins - 1)) * geom.ds
            x = s * math.cos(th) - tt * math.sin(th)
            y = s * math.sin(th) + tt * math.cos(th)
            c, sn = math.cos(e.phi), math.sin(e.phi)
            xr = (x - e.cx) * c + (y - e.cy) * sn
            yr = -(x - e.cx) * sn + (y - e.cy) * c
            num = e.value * dt * np.count_nonzero((xr / e.a) ** 2 + (yr / e.b) ** 2 <= 1)
            assert sino[i, j] == pytest.approx(num, abs=2e-3)


def test_make_data_counts_and_background():
    work = WORKLOADS["c64"]
    d = make_data(work, 0)
    g = d["g"]
    assert g.shape == (60, 91) and g.dtype == np.float32
    expect = work.counts * (1.0 + work.bg_frac * 1.0)
    assert abs(g.sum() - expect) < 5 * math.sqrt(expect)
    assert d["w"] == pytest.approx(work.bg_frac * work.counts / g.size, rel=1e-12)
    d2 = make_data(work, 0)
    assert np.array_equal(d2["g"], g)


def test_stack_workload_shapes():
    from dataclasses import replace
    work = WORKLOADS["c128x47"]
    small = replace(work, geometry=Geometry(16, 16, 12, 13, nz=5), counts=1e5)
    d = make_data(small, 1)
    assert d["g"].shape == (12, 13, 5) and d["x_true"].shape == (16, 16, 5)


def _imports(path):
    src = open(path).read()
    return set(re.findall(r"^\s*(?:from|import)\s+([\w\.]+)", src, re.M))


def test_oracle_and_product_share_no_code():
    """The oracle never imports the product path and the product path never
    imports or includes the oracle; the only shared module is the input
    generator, which the oracle does not import either."""
    pkg = os.path.join(ROOT, "paper_2106_03172_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            path = os.path.join(dirpath, f)
            if f.endswith(".py"):
                assert not any(m.startswith("oracle") for m in _imports(path)), f
            elif f.endswith((".cu", ".cuh", ".h", ".cpp", ".c")):
                incs = re.findall(r'#\s*include\s*[<"]([^>"]+)', open(path).read())
                assert not any("oracle" in i for i in incs), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith(".py"):
            mods = _imports(os.path.join(ROOT, "oracle", f))
            assert not any(m.startswith("paper_2106_03172_gb300") for m in mods), f


def test_batched_and_served_shapes():
    """Batched and served request shapes follow the stated rules: views
    round(1.4 N) (720 at 512^2), bins the odd integer nearest 1.43 N, counts
    and subsets in their ranges (64^2 -> 90 x 91, 128^2 -> 179 x 183, 192^2 ->
    269 x 275, 256^2 -> 358 x 367, 384^2 -> 538 x 549, 512^2 -> 720 x 733)."""
    from paper_2106_03172_gb300.phantoms import batched_workloads, serving_pool, serving_workloads
    want = {64: (90, 91), 128: (179, 183), 192: (269, 275), 256: (358, 367), 384: (538, 549), 512: (720, 733)}
    batch = batched_workloads(7, 64)
    assert {w.geometry.nx for w in batch} == {64, 128, 192, 256}
    served = serving_workloads(0, 40) + serving_workloads(1, 4, sizes=(384, 512))
    for w in batch + served:
        g = w.geometry
        assert g.nx == g.ny and (g.n_angles, g.n_bins) == want[g.nx]
        assert w.n_subsets in (6, 12, 21)
        assert w.methods[0] in (("saga",) if w in batch else ("svrem", "saga"))
    assert all(1e5 <= w.counts <= 1e7 for w in batch)
    assert all(1e6 <= w.counts <= 1e8 for w in served)
    pool = serving_pool()
    assert [w.name for w in pool][-4:] == ["serve384_0", "serve384_1", "serve512_0", "serve512_1"]
    assert {(w.geometry.nx, w.methods[0], w.n_subsets) for w in pool[-4:]} == {
        (384, "svrem", 21), (384, "saga", 6), (512, "svrem", 6), (512, "saga", 12)}


def test_distinct_serving_requests():
    """The distinct serving stream: request i is workload req<i> with data
    seed 20000 + i, sizes drawn from all four of 128^2-512^2 with the stated
    views and bins, counts log-uniform in [1e6, 1e8] and different per
    request, and a prefix of a longer stream equal to the shorter one."""
    from paper_2106_03172_gb300.phantoms import serving_requests
    want = {128: (179, 183), 256: (358, 367), 384: (538, 549), 512: (720, 733)}
    reqs = serving_requests(40)
    assert [w.name for w, _ in reqs] == [f"req{i}" for i in range(40)]
    assert [s for _, s in reqs] == [20000 + i for i in range(40)]
    assert {w.geometry.nx for w, _ in reqs} == set(want)
    for w, _ in reqs:
        assert (w.geometry.n_angles, w.geometry.n_bins) == want[w.geometry.nx]
        assert 1e6 <= w.counts <= 1e8 and w.n_subsets in (6, 12, 21) and w.methods[0] in ("svrem", "saga")
    assert len({w.counts for w, _ in reqs}) == 40
    assert serving_requests(12) == reqs[:12]


def test_subset_sequences_equal_the_scalar_definition():
    """The array form of the subset sequences gives, row by row, what
    subset_sequence gives (seeds across the 64-bit range, several subset
    numbers, the wrap of the state and the products)."""
    from paper_2106_03172_gb300.phantoms import subset_sequence, subset_sequences
    seeds = [0, 1, 90000, 2**63 + 5, 2**64 - 1, 123456789]
    for ns in (1, 6, 21, 1024):
        rows = subset_sequences(seeds, ns, 50)
        assert rows.dtype == np.int32 and rows.shape == (len(seeds), 50)
        for s, row in zip(seeds, rows):
            assert np.array_equal(row, subset_sequence(s, ns, 50)), (s, ns)
