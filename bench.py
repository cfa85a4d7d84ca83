"""Throughput benchmark of GB300 EECMG restoration (one JSON line on rank 0).

Default workload (512x512 precision/parity case): one synthetic 512 x 512
image (shapes + gradient + texture band), Gaussian PSF sigma = 2.5 on 15 x
15, two noise draws (1 % and 5 %), 5 levels with the economy schedule,
MR-II, FP32.  One step restores both degraded images.  Metric: Mpixel/s of
restored fine-grid pixels.

Timing: W untimed warm-up steps, then K steps (default: as many as make
about 1.5 s of timed work), each bracketed by CUDA events on the launching
stream; clocks are sampled every 50 ms and only samples stamped inside the
timed region are reported; between steps a 256 MiB buffer is written
to flush the 129 MB L2 (outside the events).  The timed region is bracketed
by a barrier and torch.cuda.synchronize().  With torchrun (N > 1) every rank
restores its own batch (replicas; the method has no cross-image exchange)
and the max time over ranks is used.

Extra objects: ``e2e`` (same metric through eecmg_restore_batched_host with
pinned host buffers, copies inside the timed region), ``roofline`` (dominant kernel
class: algorithmic bytes / event-timed duration from a profiled eager replay
of the same steps, vs the measured HBM copy peak), ``cpu_baseline`` (the
FP64 CPU oracle on a bounded sample of the workload), ``clocks`` and
``gpu_launches``.
``--impl reference`` times the CPU oracle itself on the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (h, w, levels, psf spec, noise levels, seed, noise seeds)
    "512x512-gauss2.5-L5": (512, 512, 5, ("gauss", 2.5, 7), (0.01, 0.05), 2000, (2001, 2002)),
    "64x64-gauss1.5-L3": (64, 64, 3, ("gauss", 1.5, 4), (0.01,), 1000, (1001,)),
    "2048x2048-gauss3-L5": (2048, 2048, 5, ("gauss", 3.0, 10), (0.01,), 3000, (3001,)),
    "4096x4096-gauss3-L5": (4096, 4096, 5, ("gauss", 3.0, 10), (0.01,), 3001, (3002,)),
    "2048x2048-motion15-L5": (2048, 2048, 5, ("motion", 15, 30.0), (0.01,), 3000, (3001,)),
    # 64 images, sides 128..1536 (square or 3:4), Gaussian or motion PSFs, 0.5-5 % noise
    "batch64-uneven-L5": None,
}
DEFAULT_WORKLOAD = "512x512-gauss2.5-L5"


def make_problems(name):
    """List of (clean image, PSF, levels, g FP32) for the workload."""
    from paper_2311_03010_gb300 import synth

    if name == "batch64-uneven-L5":
        out = []
        for spec in synth.batch_specs(64, 4000):
            psf = synth.psf_from_spec(spec["psf"])
            u = synth.synthetic_image(spec["h"], spec["w"], spec["seed"])
            g, _ = synth.degrade(u, psf, spec["v"], spec["seed"] + 1)
            out.append((u, psf, 5, g))
        return out
    h, w, L, spec, vs, seed, nseeds = WORKLOADS[name]
    psf = synth.psf_from_spec(spec)
    u = synth.synthetic_image(h, w, seed, texture=(h * w > 4096))
    return [(u, psf, L, synth.degrade(u, psf, v, ns)[0]) for v, ns in zip(vs, nseeds)]


LEVEL_SOLVE_SOURCES = ("common.cuh", "conv_tile.cuh", "finish.cuh", "persistent.cuh",
                       "level_solve.hpp", "level_solve_impl.cuh", "level_resident.cuh", "level_solve.cu")


def level_solve_source_hash():
    import hashlib

    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2311_03010_gb300", "csrc")
    for f in LEVEL_SOLVE_SOURCES:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()


def profiled_traffic(workload):
    """DRAM bytes per level-solve launch from the committed ncu summary of this
    workload, if it was taken on the current level-solve sources (else None)."""
    path = os.path.join(ROOT, "profiles", f"level_solve_traffic_{workload}.txt")
    if not os.path.exists(path):
        return None, "no ncu capture of this workload"
    kv = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("level_solve_sources_sha256") != level_solve_source_hash():
        return None, "ncu capture predates the current level-solve sources"
    return float(kv["dram_bytes_per_launch"]), path.replace(ROOT + os.sep, "")


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 50 ms from before the
    timed region to after it; only the samples stamped inside the region count."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.idx = device_index
        self.proc = None
        self.path = None
        self.t_begin = self.t_end = None

    def start(self):
        """Starts nvidia-smi and waits (at most 5 s) for its first sample."""
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        t0 = time.time()
        while time.time() - t0 < 5.0 and os.path.getsize(self.path) == 0:
            time.sleep(0.02)

    def begin(self):
        self.t_begin = time.time()

    def end(self):
        self.t_end = time.time()

    def stop(self):
        import datetime

        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)  # one more sample after the region
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        def stamp(text):
            for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
                try:
                    return datetime.datetime.strptime(text, fmt).timestamp()
                except ValueError:
                    pass
            return None

        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                rows.append((stamp(parts[0]), float(parts[2]), float(parts[3]), parts[6:10]))
            except ValueError:
                continue
        os.unlink(self.path)
        if any(r[0] is None for r in rows):
            # unreadable time stamps: every sample, from just before to just after the region
            inside, window = rows, "sampler run around the timed region"
        else:
            inside = [r for r in rows if self.t_begin is not None and self.t_begin <= r[0] <= self.t_end]
            window = "timed region"
        if not inside and rows and self.t_begin is not None:
            # a region shorter than the sampling period: the sample nearest to its middle
            mid = 0.5 * (self.t_begin + self.t_end)
            inside = [min(rows, key=lambda r: abs(r[0] - mid))]
            window = "nearest sample to a region shorter than the sampling period"
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in inside:
            for nm, val in zip(names, r[3]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r[1] for r in inside) if inside else None,
                "sm_max_mhz": max(r[2] for r in inside) if inside else None,
                "samples": len(inside), "window": window,
                "region_s": (self.t_end - self.t_begin) if self.t_begin is not None else None,
                "reasons": sorted(reasons)}


def cpu_baseline(name, max_seconds=12.0):
    """The FP64 oracle on a bounded sample: whole images of the workload, repeated."""
    import oracle

    probs = make_problems(name)
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    oracle.set_threads(threads)
    px = 0
    t0 = time.perf_counter()
    n = 0
    while True:
        _, psf, L, g = probs[n % len(probs)]
        oracle.cascade(g.astype(np.float64), L, psf)
        px += g.size
        n += 1
        if time.perf_counter() - t0 > max_seconds or n >= 64:
            break
    dt = time.perf_counter() - t0
    oracle.set_threads(1)
    return {"value": px / dt / 1e6, "unit": "Mpixel/s", "cores": threads, "kind": "oracle",
            "sample": f"{n} whole restorations of the {name} images (FP64 C oracle, OpenMP)",
            "seconds": dt}


def _percentiles(xs):
    xs = np.asarray(xs, dtype=np.float64)
    return {"p50_ms": float(np.percentile(xs, 50)), "p99_ms": float(np.percentile(xs, 99)),
            "mean_ms": float(xs.mean()), "max_ms": float(xs.max())}


def serving_leg(torch, eecmg, stream, storage, n_req=400, rate=200.0, seed=5000,
                budget=64 << 30, slots=64):
    """Serving form: a Poisson stream of restore requests (sizes 256^2..4096^2
    log-uniform, Gaussian or motion PSF each, 1-5 % noise, 5 levels, MR-II)
    through the continuous-batching server, and the same trace through the
    plain per-image loop (eecmg_restore per request, FIFO on one stream, its
    CUDA graph captured beforehand).  Open loop: requests are submitted at
    their arrival times; latency = arrival -> result ready (device clock).
    Saturated: the whole trace submitted at once, Mpixel/s = capacity.

    Inputs: crops of one synthetic image, blurred on the device by zero-padded
    2-D correlation with each request's (symmetric) PSF, plus seeded Gaussian
    noise with ||e|| = v ||u||.
    """
    from paper_2311_03010_gb300 import synth

    tr = synth.arrival_trace(n_req, rate, seed)
    smax = max(max(r["h"], r["w"]) for r in tr)
    u_clean = torch.from_numpy(synth.synthetic_image(smax, smax, seed).astype(np.float32)).cuda()
    gen = torch.Generator(device="cuda")
    reqs = []
    for r in tr:
        psf = synth.psf_from_spec(r["psf"])
        h, w = r["h"], r["w"]
        x = u_clean[:h, :w].reshape(1, 1, h, w)
        k = torch.from_numpy(np.ascontiguousarray(psf[::-1, ::-1]).astype(np.float32)).cuda()
        hu = torch.nn.functional.conv2d(x, k.reshape(1, 1, *psf.shape),
                                        padding=(psf.shape[0] // 2, psf.shape[1] // 2))[0, 0]
        gen.manual_seed(r["seed"])
        e = torch.randn(h, w, generator=gen, device="cuda")
        g = (hu + e * (r["v"] * x.norm() / e.norm())).contiguous()
        reqs.append({"t": r["t"], "g": g, "u": torch.empty_like(g), "psf": psf, "h": h, "w": w})
    px = sum(r["h"] * r["w"] for r in reqs)
    torch.cuda.synchronize()

    def replay(submit, finish, open_loop):
        t0 = time.perf_counter()
        subs = []
        for r in reqs:
            if open_loop:
                delay = t0 + r["t"] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
            subs.append((time.perf_counter(), submit(r)))
        lat = finish(subs)
        return time.perf_counter() - t0, lat

    out = {"requests": n_req, "rate_per_s": rate, "storage": storage, "levels": 5,
           "pixels": px, "sizes": "256^2..4096^2 log-uniform", "budget_bytes": budget,
           "max_slots": slots}
    # --- continuous-batching server
    descs = [eecmg.Plan(r["w"], r["h"], 5, r["psf"], storage=storage, workspace=0) for r in reqs]
    srv = eecmg.Server(budget, slots)
    for i in range(min(8, n_req)):  # warm-up (occupancy queries, first launches)
        srv.submit(descs[i], reqs[i]["g"], reqs[i]["u"])
    srv.drain()
    idx = {id(r): i for i, r in enumerate(reqs)}

    def srv_submit(r):
        return srv.submit(descs[idx[id(r)]], r["g"], r["u"])

    def srv_finish(subs):
        srv.drain()
        return [srv.poll(t)[1] for (_, t) in subs]

    for mode in ("open", "saturated"):
        dt, lat = replay(srv_submit, srv_finish, mode == "open")
        out[f"server_{mode}"] = dict(_percentiles(lat), mpix_s=px / dt / 1e6, seconds=dt)
    srv.close()
    for d in descs:
        d.close()
    # --- plain per-image loop
    plans = [eecmg.Plan(r["w"], r["h"], 5, r["psf"], storage=storage) for r in reqs]
    for p, r in zip(plans, reqs):
        p.restore(r["g"], r["u"], stream)  # captures each plan's graph
    torch.cuda.synchronize()
    base = torch.cuda.Event(enable_timing=True)
    base.record(stream)
    base.synchronize()
    base_host = time.perf_counter()

    def loop_submit(r):
        plans[idx[id(r)]].restore(r["g"], r["u"], stream)
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(stream)
        return ev

    def loop_finish(subs):
        torch.cuda.synchronize()
        return [(base_host + base.elapsed_time(ev) / 1e3 - t_sub) * 1e3 for (t_sub, ev) in subs]

    for mode in ("open", "saturated"):
        dt, lat = replay(loop_submit, loop_finish, mode == "open")
        out[f"plain_loop_{mode}"] = dict(_percentiles(lat), mpix_s=px / dt / 1e6, seconds=dt)
    for p in plans:
        p.close()
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return
    name = args.workload
    probs = make_problems(name)
    import oracle

    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    oracle.set_threads(threads)
    # one step = a bounded sample: at most 2 whole restorations of the workload's images
    sample = probs[:2]
    step = lambda: [oracle.cascade(g.astype(np.float64), L, psf) for (_, psf, L, g) in sample]
    for _ in range(args.warmup):
        step()
    if args.steps <= 0:
        args.steps = 10
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    px = sum(g.size for (_, _, _, g) in sample) * args.steps
    val = px / dt / 1e6
    print(json.dumps({
        "impl": "reference", "metric": "Mpixel/s restored (EECMG, oracle-matched)", "value": val,
        "unit": "Mpixel/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": name, "images_per_step": len(sample)},
        "cpu_baseline": {"value": val, "unit": "Mpixel/s", "cores": threads, "kind": "oracle",
                         "sample": f"{args.steps} steps of {len(sample)} whole restorations"},
        "e2e": {"value": val, "unit": "Mpixel/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0,
                    help="timed steps (default: enough for about 1.5 s of timed work, 100..5000)")
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--smoother", default="mr2", choices=["mr2", "cgls"])
    ap.add_argument("--precise-conv", type=int, default=1)
    ap.add_argument("--storage", default="fp32", choices=["fp32", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    args = ap.parse_args()

    from paper_2311_03010_gb300 import replicas

    rank, world, local = replicas.env()

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch

    from paper_2311_03010_gb300 import build_lib, eecmg

    torch.cuda.set_device(local)
    replicas.init(world, "nccl", torch.device("cuda", local))
    if rank == 0 or not os.path.exists(build_lib.LIB):
        build_lib.build()
    replicas.barrier(world)
    eecmg.load()

    name = args.workload
    probs = make_problems(name)
    stream = torch.cuda.current_stream()
    gs = [torch.from_numpy(g).cuda() for (_, _, _, g) in probs]

    def plan_opts(psf):
        smo = args.smoother
        if smo == "mr2" and not np.allclose(psf, psf[::-1, ::-1], rtol=0, atol=1e-15):
            smo = "cgls"
        return dict(smoother=smo, precise_conv=args.precise_conv, storage=args.storage)

    # partition of the level solves: autotuned on this workload (before any plan
    # owns a workspace), untimed
    tuning_src = "defaults"
    if not args.no_autotune:
        descs = [eecmg.Plan(g.shape[1], g.shape[0], L, psf, workspace=0, **plan_opts(psf))
                 for (_, psf, L, g) in probs]
        t0 = time.perf_counter()
        eecmg.eecmg_autotune(descs, gs, reps=5, stream=stream)
        tuning_src = f"autotuned on this workload in {time.perf_counter() - t0:.1f} s"
        for d in descs:
            d.close()
    tuning = dict(eecmg.eecmg_get_tuning(), source=tuning_src)
    plans = [eecmg.Plan(g.shape[1], g.shape[0], L, psf, **plan_opts(psf)) for (_, psf, L, g) in probs]
    us = [torch.empty_like(g) for g in gs]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        eecmg.eecmg_restore_batched([p.handle for p in plans], gs, us, stream)

    def barrier():
        replicas.barrier(world)
        torch.cuda.synchronize()

    for _ in range(max(3, args.warmup)):
        step()
    barrier()
    if args.steps <= 0:
        # enough steps for about 1.5 s of timed work (same count on every rank)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(2):  # the second pass is the estimate
            e0.record(stream)
            for _ in range(5):
                flush.zero_()
                step()
            e1.record(stream)
            torch.cuda.synchronize()
        per = e0.elapsed_time(e1) / 5.0
        args.steps = int(replicas.max_over_ranks(min(5000, max(100, int(1500.0 / max(per, 1e-3)))),
                                                 world, "cuda"))

    # timed region
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier()
    clocks.begin()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    barrier()
    clocks.end()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for (a, b) in ev]
    tot_ms = replicas.max_over_ranks(sum(step_ms), world, "cuda")
    px_step = sum(g.numel() for g in gs)
    value = replicas.aggregate_rate(px_step, args.steps, world, tot_ms) / 1e6

    # the plain per-image loop on the same plans (for the batched workload)
    loop_value = None
    if len(plans) > 2:
        for p, g, u in zip(plans, gs, us):
            p.restore(g, u, stream)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        loop_steps = max(3, args.steps // 4)
        loop_ms = 0.0
        for _ in range(loop_steps):
            flush.zero_()
            e0.record(stream)
            for p, g, u in zip(plans, gs, us):
                p.restore(g, u, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            loop_ms += e0.elapsed_time(e1)
        loop_value = px_step * loop_steps / (loop_ms / 1e3) / 1e6

    # parity of this run's output against the oracle (first image, rank 0 only)
    parity = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle

        u_clean, psf0, L0, g0 = probs[0]
        oracle.set_threads(len(os.sched_getaffinity(0)))
        ref, _, _ = oracle.cascade(g0.astype(np.float64), L0, psf0, smoother=args.smoother)
        got = us[0].double().cpu().numpy()
        parity = {"rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                  "dpsnr_db": float(abs(oracle.psnr(u_clean, got) - oracle.psnr(u_clean, ref))),
                  "psnr_db": float(oracle.psnr(u_clean, got))}
        oracle.set_threads(1)

    # end to end through the public host-buffer entry point (pinned memory):
    # the step's images copied in, restored as one batch, copied out, synchronised
    gh = [torch.from_numpy(g).pin_memory() for (_, _, _, g) in probs]
    uh = [torch.empty_like(x).pin_memory() for x in gh]
    hp = [p.handle for p in plans]
    eecmg.eecmg_restore_batched_host(hp, gh, uh, stream)
    barrier()
    e2e_steps = max(3, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        eecmg.eecmg_restore_batched_host(hp, gh, uh, stream)
    barrier()
    e2e_s = replicas.max_over_ranks(time.perf_counter() - t0, world, "cuda")
    e2e_val = replicas.aggregate_rate(px_step, e2e_steps, world, e2e_s * 1e3) / 1e6

    # profiled eager replay of the same restorations (one plan at a time):
    # per-kernel-class event times
    prof_steps = min(args.steps, 20) if len(plans) <= 2 else 1
    for p in plans:
        eecmg.eecmg_plan_profile(p.handle, 1)
    for _ in range(prof_steps):
        flush.zero_()
        for p, g, u in zip(plans, gs, us):
            p.restore(g, u, stream)
    barrier()
    classes = {}
    for p in plans:
        for k, v in eecmg.eecmg_plan_profile_read(p.handle).items():
            c = classes.setdefault(k, {"launches": 0, "ms": 0.0, "bytes": 0.0})
            for f in c:
                c[f] += v[f]
        eecmg.eecmg_plan_profile(p.handle, 0)
    launches_per_step = eecmg.eecmg_batch_info(plans)  # graph nodes of one timed step
    top = max(classes.items(), key=lambda kv: kv[1]["ms"])
    traffic, traffic_src = profiled_traffic(name)
    peak, peak_kind = peaks()
    achieved = top[1]["bytes"] / (top[1]["ms"] / 1e3) / 1e9 if top[1]["ms"] > 0 else 0.0
    prof_total = sum(c["ms"] for c in classes.values())

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(name)

    serving = None
    if not args.no_serving:
        serving = serving_leg(torch, eecmg, stream, args.storage)

    if rank == 0:
        out = {
            "metric": "Mpixel/s restored (EECMG, oracle-matched)",
            "value": value, "unit": "Mpixel/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": name, "images_per_step": len(gs), "levels": probs[0][2],
                       "smoother": args.smoother, "precise_conv": args.precise_conv,
                       "storage": args.storage, "tile": "32x64 + halo", "partition": tuning,
                       "parallelism": f"replicas x{world}", "l2": "flushed between steps"},
            "e2e": {"value": e2e_val, "unit": "Mpixel/s",
                    "h2d_bytes_per_step": int(sum(g.numel() * 4 for g in gs)),
                    "d2h_bytes_per_step": int(sum(g.numel() * 4 for g in gs))},
            "gpu_launches": int(launches_per_step * args.steps),
            "roofline": {"bound": "hbm", "kernel": top[0], "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                         "traffic_source": traffic_src,
                         "peak_kind": peak_kind,
                         "share_of_step": top[1]["ms"] / prof_total if prof_total else None,
                         "method": f"event pairs per launch, eager replay of {prof_steps} steps"},
            "kernel_classes_ms_per_step": {k: v["ms"] / prof_steps for k, v in classes.items()
                                           if v["launches"]},
            "clocks": clk,
            "per_image_loop_value": loop_value,
            "serving": serving,
            "parity": parity,
            "cpu_baseline": cpu,
        }
        print(json.dumps(out), flush=True)
    for p in plans:
        p.close()
    replicas.finalize(world)


if __name__ == "__main__":
    main()
