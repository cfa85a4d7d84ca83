"""Replica runs (one process per GPU) on CPU: two gloo ranks, no GPU.

The method has no exchange step between images, so a multi-GPU run is N
independent replicas; what crosses ranks is the barrier and the maximum of
the timed duration.  Two ranks with different durations must both see the
maximum, and the whole-job rate must count every rank's pixels over it.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    from paper_2311_03010_gb300 import replicas

    r, w, local = replicas.env()
    replicas.init(w, "gloo")
    replicas.barrier(w)
    ms = 10.0 * (r + 1)  # rank 1 is the slower one
    mx = replicas.max_over_ranks(ms, w)
    rate = replicas.aggregate_rate(1000.0, 5, w, mx)
    replicas.barrier(w)
    replicas.finalize(w)
    out.put((r, w, local, mx, rate))


def test_two_rank_replicas_take_the_max_over_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(world))
    for r, (rank, w, local, mx, rate) in enumerate(res):
        assert (rank, w, local) == (r, world, r)
        assert mx == pytest.approx(20.0)
        assert rate == pytest.approx(1000.0 * 5 * world / 0.020)


def test_single_process_needs_no_process_group():
    from paper_2311_03010_gb300 import replicas

    assert replicas.max_over_ranks(3.5, 1) == 3.5
    assert replicas.aggregate_rate(100.0, 2, 1, 1000.0) == pytest.approx(200.0)
