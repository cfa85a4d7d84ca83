"""Continuous-batching server: every result is the same alone and in the mix.

Requests of different sizes, PSFs, solvers and storage types arrive while
others are on the device; each result must equal, bitwise, the plan's own
eecmg_restore (the server keeps every job's canonical block count, so the
fixed-order reductions give identical sums), and so lie within the FP32 bar
of the FP64 oracle.  Admission by memory, slot limits, description-only
plans and argument errors are covered too.
"""
import gc
import time

import numpy as np
import pytest

from gpu_helpers import dev, host, rel_l2, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    return require_gpu()


def _specs():
    from paper_2311_03010_gb300 import synth

    return [
        (64, 64, 3, synth.gaussian_psf(1.5, 4), 1000, "mr2", "fp32"),
        (45, 70, 4, synth.motion_psf(7, 30.0), 77, "cgls", "fp32"),
        (97, 131, 4, synth.gaussian_psf(2.0, 6), 78, "mr2", "bf16"),
        (200, 150, 5, synth.motion_psf(11, 120.0), 79, "mr2", "fp32"),
        (256, 256, 5, synth.gaussian_psf(3.0, 9), 80, "cgls", "bf16"),
        (33, 31, 3, synth.gaussian_psf(1.0, 3), 81, "mr2", "fp32"),
        (512, 384, 5, synth.gaussian_psf(2.5, 7), 82, "mr2", "fp32"),
    ]


def _setup(torch, E):
    from paper_2311_03010_gb300 import synth

    reqs = []
    for (h, w, L, psf, seed, smo, st) in _specs():
        p = synth.make_problem(h, w, seed, psf, 0.02)
        plan = E.Plan(w, h, L, psf, smoother=smo, storage=st, delta=p.delta)  # discrepancy stop
        gd = dev(torch, p.g)
        ud = torch.empty_like(gd)
        plan.restore(gd, ud)
        reqs.append((p, L, smo, plan, gd, host(ud)))
    return reqs


def _wait(srv, tickets, timeout=60.0):
    t0 = time.time()
    lat = {}
    while len(lat) < len(tickets):
        for t in tickets:
            if t in lat:
                continue
            done, ms = srv.poll(t)
            if done:
                lat[t] = ms
        assert time.time() - t0 < timeout
        time.sleep(0.001)
    return lat


def test_served_results_equal_alone(gpu, orc):
    torch, E = gpu
    reqs = _setup(torch, E)
    srv = E.Server(4 << 30, 8)
    outs = [torch.full_like(r[4], float("nan")) for r in reqs]
    # staggered arrivals: the later requests join while the first are mid-cascade
    tickets = [srv.submit(reqs[i][3], reqs[i][4], outs[i]) for i in range(3)]
    time.sleep(0.002)
    tickets += [srv.submit(reqs[i][3], reqs[i][4], outs[i]) for i in range(3, len(reqs))]
    lat = _wait(srv, tickets)
    srv.drain()
    for i, r in enumerate(reqs):
        assert np.array_equal(host(outs[i]), r[5]), i
        assert np.isfinite(lat[tickets[i]]) and lat[tickets[i]] > 0.0
    # the same plans resubmitted in another order and mix
    order = [6, 2, 0, 4]
    outs2 = {i: torch.empty_like(reqs[i][4]) for i in order}
    t2 = {i: srv.submit(reqs[i][3], reqs[i][4], outs2[i]) for i in order}
    srv.drain()
    for i in order:
        assert srv.poll(t2[i])[0]
        assert np.array_equal(host(outs2[i]), reqs[i][5]), i
    srv.close()
    # and the served FP32 result of a mixed-size request matches the oracle
    p, L, smo = reqs[3][0], reqs[3][1], reqs[3][2]
    ref, rit, _ = orc.cascade(p.g.astype(np.float64), L, p.psf, smoother=smo, stop="discrepancy",
                              delta=p.delta)
    assert reqs[3][3].stats()[0] == rit
    assert rel_l2(host(outs[3]), ref) <= 1e-4
    for r in reqs:
        r[3].close()


def test_served_in_place_and_aliased_buffers(gpu):
    """The server solves a request's finest level in the caller's buffers when g and u are
    disjoint, and through its own workspace and two copies when they overlap (u_out = g_delta,
    as eecmg_restore allows): both give the plan's own result bitwise, mixed in one batch."""
    torch, E = gpu
    reqs = _setup(torch, E)
    srv = E.Server(4 << 30, 8)
    outs, tickets = [], []
    for i, r in enumerate(reqs):
        if i % 2:
            buf = r[4].clone()  # aliased: the result overwrites the data in place
            tickets.append(srv.submit(r[3], buf, buf))
        else:
            buf = torch.full_like(r[4], float("nan"))
            tickets.append(srv.submit(r[3], r[4], buf))
        outs.append(buf)
    srv.drain()
    for i, r in enumerate(reqs):
        assert srv.poll(tickets[i])[0]
        assert np.array_equal(host(outs[i]), r[5]), i
    srv.close()
    for r in reqs:
        r[3].close()


def test_memory_admission_and_single_slot(gpu):
    """A budget that holds one request at a time, or one slot, still serves all."""
    torch, E = gpu
    reqs = _setup(torch, E)
    biggest = max(r[3].info["workspace_bytes"] for r in reqs)
    for budget, slots in [(biggest + 4096, 8), (4 << 30, 1)]:
        srv = E.Server(budget, slots)
        outs = [torch.empty_like(r[4]) for r in reqs]
        ts = [srv.submit(r[3], r[4], o) for r, o in zip(reqs, outs)]
        srv.drain()
        for t, o, r in zip(ts, outs, reqs):
            assert srv.poll(t)[0]
            assert np.array_equal(host(o), r[5])
        srv.close()
    # a request larger than the whole budget is refused at submission
    srv = E.Server(1 << 20, 4)
    with pytest.raises(E.EecmgError) as ei:
        srv.submit(reqs[-1][3], reqs[-1][4], torch.empty_like(reqs[-1][4]))
    assert ei.value.status == 3  # EECMG_ERR_OOM
    srv.close()
    for r in reqs:
        r[3].close()


def test_description_only_plans(gpu):
    """workspace = 0 plans hold no device memory, serve normally, and cannot restore."""
    torch, E = gpu
    from paper_2311_03010_gb300 import synth

    p = synth.make_problem(120, 90, 83, synth.gaussian_psf(1.5, 4), 0.02)
    full = E.Plan(90, 120, 4, p.psf)
    desc = E.Plan(90, 120, 4, p.psf, workspace=0)
    assert desc.info["workspace_bytes"] == full.info["workspace_bytes"]
    gd = dev(torch, p.g)
    ref = torch.empty_like(gd)
    full.restore(gd, ref)
    with pytest.raises(E.EecmgError) as ei:
        desc.restore(gd, torch.empty_like(gd))
    assert ei.value.status == 1
    srv = E.Server(1 << 30, 4)
    outs = [torch.empty_like(gd) for _ in range(5)]
    ts = [srv.submit(desc, gd, o) for o in outs]  # one description, five resident requests
    srv.drain()
    for t, o in zip(ts, outs):
        assert srv.poll(t)[0]
        assert np.array_equal(host(o), host(ref))
    srv.close()
    full.close()
    desc.close()


def test_served_options_equal_alone(gpu):
    """Algorithm 1 prolongations and other diffusion step counts through the server's batched ops."""
    torch, E = gpu
    from paper_2311_03010_gb300 import synth

    specs = [(96, 80, 4, synth.gaussian_psf(1.5, 4), 84, dict(prolong="iecmg_l", diffusion_steps=2)),
             (70, 110, 4, synth.motion_psf(7, 45.0), 85, dict(prolong="iecmg_p", diffusion_steps=0)),
             (128, 128, 5, synth.gaussian_psf(2.0, 6), 86, dict(diffusion_steps=3)),
             (64, 96, 4, synth.gaussian_psf(1.0, 3), 87, dict(smoother="cgls", diffusion_steps=0))]
    plans, gs, singles = [], [], []
    for (h, w, L, psf, seed, opts) in specs:
        p = synth.make_problem(h, w, seed, psf, 0.02)
        pl = E.Plan(w, h, L, psf, **opts)
        gd = dev(torch, p.g)
        ud = torch.empty_like(gd)
        pl.restore(gd, ud)
        singles.append(host(ud))
        plans.append(pl)
        gs.append(gd)
    srv = E.Server(1 << 30, 8)
    outs = [torch.empty_like(g) for g in gs]
    ts = [srv.submit(pl, g, o) for pl, g, o in zip(plans, gs, outs)]
    srv.drain()
    for t, o, s_ in zip(ts, outs, singles):
        assert srv.poll(t)[0]
        assert np.array_equal(host(o), s_)
    srv.close()
    for pl in plans:
        pl.close()


def test_device_memory_stays_flat_while_serving(gpu):
    """After a warm-up, serving allocates no device memory: the arena and the per-tick tables
    are sized when the server is created."""
    torch, E = gpu
    reqs = _setup(torch, E)
    srv = E.Server(2 << 30, 4)
    outs = [torch.empty_like(r[4]) for r in reqs * 4]
    srv.drain()
    for r, o in zip(reqs, outs):  # warm-up: every kind of request once
        srv.submit(r[3], r[4], o)
    srv.drain()
    gc.collect()  # garbage of earlier tests must not be freed inside the measurement
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for _ in range(3):  # more requests than slots: admission waits for slots and memory
        ts = [srv.submit(r[3], r[4], o) for r, o in zip(reqs * 4, outs)]
        srv.drain()
        assert all(srv.poll(t)[0] for t in ts)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    for k, o in enumerate(outs):
        assert np.array_equal(host(o), reqs[k % len(reqs)][5]), k
    srv.close()
    for r in reqs:
        r[3].close()


def test_server_rejects_requests_beyond_its_table_bounds(gpu):
    """Plans with more diffusion steps than the server's per-tick tables allow are refused at
    submission (the tables are never grown while serving)."""
    torch, E = gpu
    from paper_2311_03010_gb300 import synth

    srv = E.Server(1 << 28, 2)
    plan = E.Plan(32, 32, 3, synth.gaussian_psf(1.0, 2), diffusion_steps=17, workspace=0)
    g = torch.zeros(32, 32, device="cuda")
    with pytest.raises(E.EecmgError) as ei:
        srv.submit(plan, g, torch.empty_like(g))
    assert ei.value.status == 1
    ok = E.Plan(32, 32, 3, synth.gaussian_psf(1.0, 2), diffusion_steps=16, workspace=0)
    u = torch.empty_like(g)
    t = srv.submit(ok, g, u)
    srv.drain()
    assert srv.poll(t)[0]
    srv.close()
    plan.close()
    ok.close()


def test_failed_request_is_isolated(gpu):
    """A request whose data holds a NaN fails alone (EECMG_ERR_NUMERIC); the others complete."""
    torch, E = gpu
    from paper_2311_03010_gb300 import synth

    reqs = []
    for k, (h, w, seed) in enumerate([(64, 64, 88), (96, 72, 89), (80, 80, 90)]):
        p = synth.make_problem(h, w, seed, synth.gaussian_psf(1.5, 4), 0.02)
        pl = E.Plan(w, h, 4, p.psf)
        gd = dev(torch, p.g)
        ud = torch.empty_like(gd)
        pl.restore(gd, ud)
        reqs.append((pl, gd, host(ud)))
    bad = reqs[1][1].clone()
    bad[5, 7] = float("nan")
    srv = E.Server(1 << 30, 4)
    outs = [torch.empty_like(r[1]) for r in reqs]
    ts = [srv.submit(reqs[0][0], reqs[0][1], outs[0]), srv.submit(reqs[1][0], bad, outs[1]),
          srv.submit(reqs[2][0], reqs[2][1], outs[2])]
    srv.drain()
    with pytest.raises(E.EecmgError) as ei:
        srv.poll(ts[1])
    assert ei.value.status == 5  # EECMG_ERR_NUMERIC
    for i in (0, 2):
        assert srv.poll(ts[i])[0]
        assert np.array_equal(host(outs[i]), reqs[i][2])
    # the server keeps serving after the failure
    t = srv.submit(reqs[0][0], reqs[0][1], outs[0])
    srv.drain()
    assert srv.poll(t)[0] and np.array_equal(host(outs[0]), reqs[0][2])
    srv.close()
    for r in reqs:
        r[0].close()


def test_server_argument_errors(gpu):
    torch, E = gpu
    from paper_2311_03010_gb300 import synth

    with pytest.raises(E.EecmgError):
        E.Server(0, 4)
    with pytest.raises(E.EecmgError):
        E.Server(1 << 20, 0)
    srv = E.Server(1 << 26, 2)
    with pytest.raises(E.EecmgError):
        srv.poll(12345)
    plan = E.Plan(32, 32, 3, synth.gaussian_psf(1.0, 2), persistent=0)
    g = torch.zeros(32, 32, device="cuda")
    with pytest.raises(E.EecmgError):
        srv.submit(plan, g, torch.empty_like(g))  # the server needs the persistent solve
    srv.close()
    plan.close()
