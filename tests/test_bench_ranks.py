"""The multi-rank bookkeeping of bench.py on CPU: two gloo ranks running
independent replicas; the whole-job value is the summed units over the
slowest rank's time, and a rank that never joins fails the rendezvous."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        total_ms = [250.0, 400.0][rank]
        units = [1000.0, 1500.0][rank]
        value, tmax, uall = bench.combine_ranks(total_ms, units, device="cpu")
        out[rank] = (value, tmax, uall)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_combine_as_replicas():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    for r in range(2):
        value, tmax, uall = out[r]
        assert tmax == 400.0 and uall == 2500.0
        assert value == pytest.approx(2500.0 / 0.4)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(500.0, 100.0) == (200.0, 500.0, 100.0)


def _lonely(rank, port):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=2,
                            timeout=__import__("datetime").timedelta(seconds=3))


def test_missing_rank_fails_on_the_host():
    """A replica that never joins is detected on the host by the rendezvous
    timeout (no GPU involved)."""
    ctx = mp.get_context("spawn")
    p = ctx.Process(target=_lonely, args=(0, _free_port()))
    p.start()
    p.join(60)
    assert not p.is_alive() and p.exitcode != 0


def test_step_pairs_count_anchor_passes():
    """The metric's units per step: 4 N_s subset pairs, plus N_s for each
    anchor pass due (SVREM every eta_svrem epochs, SVRG every eta_svrg), the
    anchors due at the epoch's first update."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2106_03172_gb300.phantoms import WORKLOADS
    for name in ("c256", "c64", "ring2_128"):
        work = WORKLOADS[name]
        ns, e_svrem, e_svrg = work.n_subsets, work.eta_svrem, work.eta_svrg
        rep = bench.Replica(work)
        total = 0
        for step in range(12):
            p, anchors = rep.step_pairs()
            want = ["svrem"] * (step % e_svrem == 0) + ["svrg"] * (step % e_svrg == 0)
            assert anchors == want
            assert p == 4 * ns + ns * len(want)
            total += p
            rep.advance()
        assert total == 12 * 4 * ns + ns * (len(range(0, 12, e_svrem)) + len(range(0, 12, e_svrg)))
