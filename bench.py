"""Throughput benchmark of the MPPI + contact-rollout hot path.

A step is one MPPI iteration (Alg. 1 loop body: Philox sampling, H-step
contact rollouts of K samples, stage costs, softmax weights, weighted-mean
update).  The headline workload is the largest single-controller one: two
7-DoF arms carrying a 0.10 m ball past 8 static boxes, K = 4096 samples,
H = 64 steps (dt = 0.01 s, 4 PGS sweeps), on synthetic seeded inputs; the
line also carries the smaller ball lift (K = 1024, H = 32) under "lift".
value = simulated sample-steps/s = K * H * steps / time over all ranks (each
rank runs its own independent controller: weak scaling).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload transfer|lift|batched|serve|closed_loop]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the comparison arm for this project).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2511_21264_gb300 import flops, scenes  # noqa: E402

METRIC = "simulated sample-steps/s (MPPI iteration: sample + rollout + cost + weights + update)"
UNIT = "sample-steps/s"
WORKLOAD = "7-DoF bimanual ball lift, K=1024 samples, H=32 steps, dt=0.01 s, 4 PGS sweeps, FP32"


WORKLOADS = {
    "lift": WORKLOAD,
    "transfer": "7-DoF ball transfer past 8 boxes, K=4096 samples, H=64 steps, dt=0.01 s, 4 PGS sweeps, FP32",
}


def _config_json(sc, n_gpus, workload="transfer"):
    return {"workload": WORKLOADS[workload], "scene": sc.name, "K": sc.K, "H": sc.H, "nv": sc.nv, "n_boxes": sc.n_boxes,
            "lambda": sc.lam, "sigma": sc.sigma, "per_rank": "one independent controller (own Philox key)",
            "parallelism": f"replicas x{n_gpus}",
            "l2": "flushed between timed steps (256 MiB write); working set < 1 MiB"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for name, val in zip(names, p[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist_setup(n_gpus):
    import torch
    rank, world = int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, world, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(v, world):
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline(sc, seconds=15.0, nthreads=None):
    """The FP64 oracle on the host cores on a bounded sample of the workload:
    MPPI iterations with K' <= K samples (same H, scene, lambda, sigma)."""
    import oracle
    nthreads = nthreads or os.cpu_count() or 1
    om = oracle.Model(sc.to_blob())
    x = sc.x0.astype(np.float32).astype(np.float64)
    u = np.zeros((sc.H, sc.nu))
    sig = sc.sigma_vec()
    Kp = max(nthreads, 8)
    t0 = time.perf_counter()
    om.mppi_iteration(x, u, Kp, sc.lam, sig, 1, 0, nthreads=nthreads)
    dt = time.perf_counter() - t0
    # grow the sample to fill about `seconds` of work per measurement
    Kp = int(min(sc.K, max(Kp, Kp * seconds / max(dt, 1e-3) / 3)))
    done, t0, it = 0, time.perf_counter(), 0
    while time.perf_counter() - t0 < seconds or it == 0:
        om.mppi_iteration(x, u, Kp, sc.lam, sig, 1, it, nthreads=nthreads)
        done += Kp * sc.H
        it += 1
    el = time.perf_counter() - t0
    # the same oracle on one thread, on a smaller sample
    K1 = max(4, Kp // max(1, nthreads))
    t1 = time.perf_counter()
    om.mppi_iteration(x, u, K1, sc.lam, sig, 1, it, nthreads=1)
    one = K1 * sc.H / (time.perf_counter() - t1)
    return {"value": done / el, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "value_1_thread": one,
            "sample": f"{it} MPPI iterations of K'={Kp} samples (of K={sc.K}), H={sc.H}, same scene; "
                      f"{el:.1f} s of FP64 work on {nthreads} threads; 1-thread figure from one iteration "
                      f"of K'={K1}"}


def _scene(workload):
    if workload in ("lift", "transfer"):
        return scenes.config(3 if workload == "transfer" else 2)
    raise ValueError(workload)


def _metric(workload):
    return METRIC if workload == "lift" else METRIC.replace("MPPI iteration", "MPPI iteration, " + workload)


PROFILE_FILES = {"transfer": "rollout_kernel_dh7_transfer_K4096_H64.md",
                 "lift": "rollout_kernel_dh7_lift_K1024_H32.md"}
KERNEL_SOURCES = ("mppi_device.cuh", "mppi_kernels.cuh", "mppi_task.cuh", "mppi_internal.h")


def kernel_source_hash():
    """sha256 over the source files that make up the rollout kernel (and the
    floating-point flags they are compiled with)."""
    import hashlib
    from paper_2511_21264_gb300 import native
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2511_21264_gb300", "csrc")
    for name in KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    h.update(" ".join(native.FP_FLAGS).encode())
    return h.hexdigest()[:16]


def profile_counters(workload):
    """DRAM traffic and executed FP32 operations of one rollout launch from
    the committed ncu summary of this workload.  The summary carries one
    line `counters: {json}` with the kernel-source hash it was taken at;
    when the sources have changed since, the counters are stale and
    (None, None, reason) is returned."""
    name = PROFILE_FILES.get(workload)
    if name is None:
        return None, None, "no ncu summary for this workload"
    path = os.path.join(ROOT, "profiles", name)
    try:
        with open(path) as f:
            rows = [ln for ln in f if ln.startswith("counters: ")]
    except OSError:
        return None, None, f"profiles/{name} missing"
    if not rows:
        return None, None, f"profiles/{name} has no counters line"
    c = json.loads(rows[-1][len("counters: "):])
    if c.get("source_hash") != kernel_source_hash():
        return None, None, f"profiles/{name}: kernel sources changed since the capture"
    return float(c["dram_bytes_per_launch"]), float(c["fp32_flops_per_launch"]), f"profiles/{name}"


def run_reference(args):
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return 0
    sc = _scene(args.workload)
    nthreads = os.cpu_count() or 1
    import oracle
    om = oracle.Model(sc.to_blob())
    x = sc.x0.astype(np.float32).astype(np.float64)
    u = np.zeros((sc.H, sc.nu))
    # bounded sample per step: the warm-up steps measure the oracle's rate on
    # a small sample, then each timed step takes as many samples (a multiple
    # of the thread count, at most K) as keep the timed steps near a minute
    Kp = max(2 * nthreads, 16)
    tw = time.perf_counter()
    for w in range(args.warmup):
        om.mppi_iteration(x, u, Kp, sc.lam, sc.sigma_vec(), 1, w, nthreads=nthreads)
    rate = Kp * sc.H * args.warmup / max(time.perf_counter() - tw, 1e-9)
    want = int(rate * 60.0 / (sc.H * max(args.steps, 1)))
    Kp = int(min(sc.K, max(Kp, want // nthreads * nthreads)))
    t0 = time.perf_counter()
    for s in range(args.steps):
        om.mppi_iteration(x, u, Kp, sc.lam, sc.sigma_vec(), 1, args.warmup + s, nthreads=nthreads)
    el = time.perf_counter() - t0
    value = Kp * sc.H * args.steps / el
    line = {"impl": "reference", "metric": _metric(args.workload), "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config_json(sc, args.gpus, args.workload),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                             "sample": f"each step: one MPPI iteration with K'={Kp} of K={sc.K} samples"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _measure(args, workload, steps, dev, stream, flush, world, local, rank):
    """Times `steps` MPPI iterations of one workload (per-step CUDA events,
    L2 flushed between steps), then the same iterations end to end through
    mppi_step_host with host buffers.  Returns the numbers of the line."""
    import torch
    from paper_2511_21264_gb300 import native
    sc = _scene(workload)
    K, H = sc.K, sc.H
    model = native.Model(sc.to_blob())
    ctl = native.Controller(model, K, H, sc.lam, sc.sigma_vec(), scenes.controller_key(sc.seed, rank))
    if args.lps or args.place:
        ctl.set_layout(args.lps or 32, args.place)
    if args.spc:
        ctl.set_launch(args.spc)
    if args.elite or args.eta != 1.0 or args.cov:
        ctl.set_update(args.elite or K, args.eta, args.cov, 1e-6)
    if args.qp:
        ctl.set_projection(scenes.projection_bounds(sc), iters=args.qp)
    if args.task is not None:
        ctl.set_task_cost(scenes.ball_task(sc, phase=args.task))
    x = torch.tensor(model.home(), device=dev)
    u = torch.zeros((H, sc.nu), device=dev)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            ctl.step(x, u, u, stream=stream)
        stream.synchronize()
        _barrier(world)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        ctl.profile(steps)
        with ClockSampler(local) as clk:
            time.sleep(0.3)
            for i in range(steps):
                flush.fill_(i & 0xFF)
                ev[i][0].record(stream)
                ctl.step(x, u, u, stream=stream)
                ev[i][1].record(stream)
            stream.synchronize()
        step_ms = [a.elapsed_time(b) for a, b in ev]
        rc = ctl.sync(stream=stream)
        if rc != 0:
            raise RuntimeError(f"device error {rc} during the timed steps")
        total_ms = _max_over_ranks(sum(step_ms), world)
        kt = ctl.profile_read()
        qp_ms = ctl.profile_projection() / max(1, kt["iterations"])
        ctl.profile(0)

        # end to end through the C ABI with host buffers (mppi_step_host): per
        # step one H2D copy of (state, u_nom) through the handle's pinned
        # staging buffer, the iteration, one D2H copy of u_nom', synchronised
        xh = np.asarray(model.home(), np.float32)
        uh = np.zeros((H, sc.nu), np.float32)
        ctl.step_host(xh, uh, uh, stream=stream)  # allocates the staging buffers
        _barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(steps):
            ctl.step_host(xh, uh, uh, stream=stream)
        e1.record(stream)
        stream.synchronize()
        e2e_ms = _max_over_ranks(e0.elapsed_time(e1), world)
    units = K * H * steps * world
    clocks = clk.summary()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_mhz = clocks["sm_mhz"] or 1477.0
    peak = sms * 128 * 2 * sm_mhz * 1e6 / 1e12
    fl = flops.per_sample_step(sc, kt["contacts_per_step"], kt["box_tests_per_step"], kt["lone_ball_per_step"])
    if args.task is not None:
        fl += flops.task_flops(sc, args.task)
    roll_ms = kt["rollout_ms"] / max(1, kt["iterations"])
    achieved = fl * K * H / (roll_ms * 1e-3) / 1e12
    elite = bool(args.elite or args.eta != 1.0 or args.cov)
    plain = not (elite or args.qp or args.task is not None)
    # DRAM traffic and executed FP32 operations of one rollout launch come
    # from the committed ncu summary of the workload, taken at the current
    # kernel sources; null when there is none or it is stale
    traffic, exec_flops, source = profile_counters(workload) if plain else (None, None, "not captured")
    lay = ctl.get_layout()
    kname = f"rollout_kernel<{sc.n_a},{lay[0]},1,{int(args.task is not None)},{lay[1]}>"
    roof = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic, "traffic_source": source,
            "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz (median SM clock "
                          f"sampled during the timed steps)",
            "flops_per_sample_step": fl, "rollout_ms": roll_ms,
            "update_ms": kt["update_ms"] / max(1, kt["iterations"]),
            "contacts_per_step": kt["contacts_per_step"],
            "box_tests_per_step": kt["box_tests_per_step"],
            "lone_ball_per_step": kt["lone_ball_per_step"]}
    if exec_flops is not None:
        ex = exec_flops / (roll_ms * 1e-3) / 1e12
        roof["ncu_executed"] = {
            "flops_per_launch": exec_flops, "achieved": ex, "frac": ex / peak,
            "per_sample_step": exec_flops / (K * H),
            "basis": "ncu FP32 thread instructions of one launch (2 x FFMA + FADD + FMUL) / live mean duration"}
    roof["layout"] = {"lanes_per_sample": lay[0], "placement": "fused" if lay[1] == 0 else "after the factor",
                      "samples_per_cta": lay[2]}
    return {"sc": sc, "value": units / (total_ms * 1e-3), "e2e": units / (e2e_ms * 1e-3),
            "ms_per_step": total_ms / steps, "iters_per_s": steps * world / (total_ms * 1e-3),
            "h2d": int(4 * (x.numel() + u.numel())), "d2h": int(4 * u.numel()),
            "roofline": roof, "clocks": clocks, "qp_ms": qp_ms, "peak": peak, "elite": elite}


def run_ours(args):
    import torch
    from paper_2511_21264_gb300 import native

    rank, world, local = _dist_setup(args.gpus)
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    native.build() if rank == 0 and world == 1 else None
    native.lib()
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    m = _measure(args, args.workload, args.steps, dev, stream, flush, world, local, rank)
    extra = None
    plain = not (m["elite"] or args.qp or args.task is not None)
    if args.workload == "transfer" and plain and not args.no_lift:
        # the smaller single-controller workload, reported beside the headline
        extra = _measure(args, "lift", max(args.steps, 200), dev, stream, flush, world, local, rank)
    if rank != 0:
        return 0
    sc = m["sc"]
    K, H = sc.K, sc.H
    elite = m["elite"]
    line = {
        "metric": _metric(args.workload), "value": m["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": _config_json(sc, world, args.workload),
        "iters_per_s": m["iters_per_s"],
        "e2e": {"value": m["e2e"], "unit": UNIT, "h2d_bytes_per_step": m["h2d"], "d2h_bytes_per_step": m["d2h"]},
        "gpu_launches": (2 + (1 if elite else 0) + (1 if args.qp else 0)) * args.steps,
        "roofline": m["roofline"],
        "clocks": m["clocks"],
    }
    if extra is not None:
        line["lift"] = {"workload": WORKLOADS["lift"], "value": extra["value"], "unit": UNIT,
                        "ms_per_step": extra["ms_per_step"], "iters_per_s": extra["iters_per_s"],
                        "e2e": extra["e2e"], "roofline_frac": extra["roofline"]["frac"],
                        "rollout_ms": extra["roofline"]["rollout_ms"],
                        "flops_per_sample_step": extra["roofline"]["flops_per_sample_step"],
                        "traffic": extra["roofline"]["traffic"], "clocks": extra["clocks"]}
    if elite:
        line["config"]["update"] = {"n_elite": args.elite or K, "eta": args.eta, "covariance": bool(args.cov)}
        line["metric"] = line["metric"].replace("weights + update", "elite set + Eq. 8 update")
    if args.qp:
        qfl = flops.qp_flops(sc.H, args.qp)
        line["config"]["projection"] = {"iters": args.qp, "rho": 1.0,
                                        "bounds": "home +-1 rad, +-pi rad/s, +-10 rad/s^2, +-300 rad/s^3"}
        line["metric"] = line["metric"].replace("sample + rollout", "sample + QP projection + rollout")
        qa = qfl * K * sc.nu / (m["qp_ms"] * 1e-3) / 1e12
        line["qp_projection"] = {"kernel": "qp_project_kernel", "ms": m["qp_ms"], "bound": "alu",
                                 "flops_per_sequence": qfl, "achieved": qa, "peak": m["peak"],
                                 "unit": "TFLOP/s", "frac": qa / m["peak"]}
    if args.task is not None:
        line["config"]["cost"] = {"suite": "ball task (Sec. IV-B)", "phase": "pick" if args.task == 0 else "move"}
        line["metric"] = line["metric"].replace("+ cost +", "+ ball-task cost suite +")
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(sc, seconds=args.cpu_seconds)
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_batched(args):
    """64 independent controllers per iteration: the persistent batched
    launch (autotuned shape, graph replay) against 64 sequential plain
    launches of the same controllers."""
    import torch
    from paper_2511_21264_gb300 import native
    rank, world, local = _dist_setup(args.gpus)
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    native.build() if rank == 0 and world == 1 else None
    native.lib()
    pool = scenes.batched_pool(64, seed=0)
    models = [native.Model(sc.to_blob()) for sc in pool]
    inst = [(m, sc.K, sc.H, sc.lam, sc.sigma_vec(), scenes.controller_key(sc.seed, rank))
            for m, sc in zip(models, pool)]
    units = sum(sc.K * sc.H for sc in pool)
    b = native.Batch(inst)
    full = bool(args.elite or args.eta != 1.0 or args.cov or args.qp)
    if full:  # the full Eq. 8 and/or the projection for every instance (and the sequential controllers)
        if args.elite or args.eta != 1.0 or args.cov:
            b.set_update(-1, args.elite, args.eta, args.cov, 1e-6)
        if args.qp:
            b.set_projection(np.stack([scenes.projection_bounds(sc) for sc in pool]), iters=args.qp)
    stream = torch.cuda.Stream(device=dev)
    xs = [torch.tensor(m.home(), device=dev) for m in models]
    us = [torch.zeros((sc.H, sc.nu), device=dev) for sc in pool]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(fn, steps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            fn()
            ev[i][1].record(stream)
        stream.synchronize()
        return [a.elapsed_time(c) for a, c in ev]

    with torch.cuda.stream(stream):
        tune_ms = b.autotune(xs, [u.clone() for u in us], reps=2, stream=stream)
        spc, order = b.get_launch()
        lps, place = b.get_layout()
        for _ in range(args.warmup):
            b.step(xs, us, stream=stream, graph=True)
        stream.synchronize()
        _barrier(world)
        with ClockSampler(local) as clk:
            time.sleep(0.3)
            t_batch = timed(lambda: b.step(xs, us, stream=stream, graph=True), args.steps)
        rc, errs = b.sync(stream=stream)
        if rc != 0:
            raise RuntimeError(f"device error {rc} in the batched steps")
        # sequential plain launches of the same controllers
        ctls = [native.Controller(m, K, H, lam, sig, key) for (m, K, H, lam, sig, key) in inst]
        for c, sc in zip(ctls, pool):
            if args.elite or args.eta != 1.0 or args.cov:
                c.set_update(min(args.elite, sc.K) or sc.K, args.eta, args.cov, 1e-6)
            if args.qp:
                c.set_projection(scenes.projection_bounds(sc), iters=args.qp)
        useq = [torch.zeros_like(u) for u in us]

        def seq():
            for c, x, u in zip(ctls, xs, useq):
                c.step(x, u, u, stream=stream)
        for _ in range(args.warmup):
            seq()
        stream.synchronize()
        seq_steps = max(3, args.steps // 4)
        t_seq = timed(seq, seq_steps)
        # end to end: pinned H2D of every state and u_nom, the batched
        # iteration, D2H of every u_nom'
        xh = [torch.tensor(m.home()).pin_memory() for m in models]
        uh = [torch.zeros((sc.H, sc.nu)).pin_memory() for sc in pool]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(args.steps):
            for a, c in zip(xs, xh):
                a.copy_(c, non_blocking=True)
            for a, c in zip(us, uh):
                a.copy_(c, non_blocking=True)
            b.step(xs, us, stream=stream, graph=True)
            for a, c in zip(uh, us):
                a.copy_(c, non_blocking=True)
            stream.synchronize()
        e1.record(stream)
        stream.synchronize()
        e2e_ms = _max_over_ranks(e0.elapsed_time(e1), world)
    total = _max_over_ranks(sum(t_batch), world)
    value = units * args.steps * world / (total * 1e-3)
    seq_value = units * seq_steps / (sum(t_seq) * 1e-3)
    if rank != 0:
        return 0
    props = torch.cuda.get_device_properties(dev)
    clocks = clk.summary()
    sm_mhz = clocks["sm_mhz"] or 1477.0
    peak = props.multi_processor_count * 128 * 2 * sm_mhz * 1e6 / 1e12
    fl = sum(flops.per_sample_step(sc, 1.0, 0.0, 1.0) * sc.K * sc.H for sc in pool)
    ms = total / args.steps
    hb = sum(4 * (sc.nq + sc.nv + sc.H * sc.nu) for sc in pool)
    line = {
        "metric": METRIC.replace("MPPI iteration", "MPPI iteration of 64 batched controllers"),
        "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "64 independent 7-DoF controllers, K in {256..4096}, H in {16..64}, "
                               "0..16 boxes (seeded), one persistent launch + update, graph replay",
                   "instances": 64, "sample_steps_per_iteration": units, "autotuned_samples_per_cta": spc,
                   "autotuned_order": "longest first" if order == 1 else "as given",
                   "autotuned_lanes_per_sample": lps,
                   "autotuned_placement": "fused" if place == 0 else "after the factor",
                   "autotune_ms": tune_ms, "parallelism": f"replicas x{world}",
                   "l2": "flushed between timed steps (256 MiB write)"},
        "iters_per_s": 64 * args.steps * world / (total * 1e-3),
        "sequential_plain": {"value": seq_value, "unit": UNIT, "ms_per_step": sum(t_seq) / seq_steps,
                             "launches_per_step": 128},
        "speedup_vs_sequential": value / world / seq_value,
        "e2e": {"value": units * args.steps * world / (e2e_ms * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": hb, "d2h_bytes_per_step": sum(4 * sc.H * sc.nu for sc in pool)},
        "gpu_launches": 2 * args.steps,
        "roofline": {"bound": "alu", "kernel": "batch_rollout_kernel<7> + batch_update_kernel<14>",
                     "achieved": fl / (ms * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                     "frac": fl / (ms * 1e-3) / 1e12 / peak, "traffic": None,
                     "flops_basis": "lower bound (one lone ball contact, no capsule-box test per step) over "
                                    "the whole iteration time"},
        "clocks": clocks,
    }
    if full:
        line["config"]["update"] = {"n_elite": args.elite or "K", "eta": args.eta, "covariance": bool(args.cov),
                                    "projection_iters": args.qp}
        line["metric"] = line["metric"].replace("controllers", "controllers, full Eq. 8" +
                                                (" + QP projection" if args.qp else ""))
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """Continuous-batching replan server: Poisson arrivals at each rate over
    a pool of 256 scenes (7-DoF arms, 0-16 boxes, K in {512..4096}, H in
    {16..64}), M = 10 MPPI iterations per request, warm-started resident
    state per scene.  The batched server (64 slots, 256 MiB budget) against a
    server that runs one request at a time on the same arrival trace."""
    import torch
    from paper_2511_21264_gb300 import native
    rank, world, local = _dist_setup(args.gpus)
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    native.build() if rank == 0 and world == 1 else None
    native.lib()
    pool = scenes.served_pool(256, seed=0)
    models = [native.Model(sc.to_blob()) for sc in pool]
    rates = [float(r) for r in args.serve_rates.split(",")]
    M = 10

    def serve(max_active, rate, seconds):
        srv = native.Server(256 << 20, max_active, M, lanes_per_sample=args.lps, size_classes=args.serve_classes)
        for m, sc in zip(models, pool):
            srv.add_scene(m, sc.K, sc.H, sc.lam, sc.sigma_vec(), scenes.controller_key(sc.seed, rank))
        srv.start()
        t0 = time.perf_counter()
        srv.run_load(rate, seconds, seed=int(rate), drain_ms=600000)
        wall = time.perf_counter() - t0
        st = srv.stats()
        rc = srv.stop()
        if rc != 0:
            raise RuntimeError(f"server error {rc}")
        srv.close()
        st["wall_s"] = wall
        return st

    out = {}
    with ClockSampler(local) as clk:
        for r in rates:
            b = serve(64, r, args.serve_seconds)
            entry = {"batched": {k: b[k] for k in ("p50_ms", "p99_ms", "mean_ms", "sample_steps_per_s", "completed",
                                                   "mean_active", "admission_waits", "wall_s")}}
            # the one-request-at-a-time server on the same kind of trace and
            # window; above 200 req/s, where it saturates and its backlog
            # would drain long after the window, a 5 s window (its throughput
            # is then its capacity)
            short = args.serve_seconds if r <= 200 else min(args.serve_seconds, 5.0)
            p = serve(1, r, short)
            entry["one_at_a_time"] = {k: p[k] for k in ("p50_ms", "p99_ms", "mean_ms", "sample_steps_per_s",
                                                        "completed", "wall_s")}
            entry["one_at_a_time"]["arrival_window_s"] = short
            if short < args.serve_seconds:
                # saturated: latency grows with the window (the backlog), so
                # the batched server also runs the one-at-a-time window
                bs = serve(64, r, short)
                entry["batched_same_window"] = {k: bs[k] for k in ("p50_ms", "p99_ms", "mean_ms",
                                                                   "sample_steps_per_s", "completed", "wall_s")}
                entry["batched_same_window"]["arrival_window_s"] = short
                b = bs
            entry["p99_one_at_a_time_over_batched"] = p["p99_ms"] / max(b["p99_ms"], 1e-9)
            entry["throughput_batched_over_one_at_a_time"] = b["sample_steps_per_s"] / max(p["sample_steps_per_s"], 1e-9)
            out[f"{r:g}_req_per_s"] = entry
    if rank != 0:
        return 0
    top = out[f"{max(rates):g}_req_per_s"]["batched"]
    line = {
        "metric": "replan server: simulated sample-steps/s and p50/p99 replan latency (ms) under Poisson load",
        "value": top["sample_steps_per_s"], "unit": UNIT, "n_gpus": world, "steps": None, "warmup": 0,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "256 scenes (7-DoF arms, 0-16 boxes, K 512..4096, H 16..64), M=10 iterations per "
                               "request, Poisson arrivals", "rates_req_per_s": rates,
                   "arrival_window_s": args.serve_seconds, "max_active": 64, "budget_bytes": 256 << 20,
                   "size_classes": args.serve_classes or 6, "lanes_per_sample": args.lps or 16},
        "latency": out,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_closed_loop(args):
    """Closed-loop receding horizon as the paper evaluates it (Sec. IV-A):
    N_runs = args.runs episodes of the planar ball lift with randomised
    goals (ball start + (U(-0.1, 0.1), 0, U(0.15, 0.3)) m), K = args.k
    samples, H = args.cl_h, M = 10 iterations per planning step, the first 4
    steps of the best sequence averaged and executed, 8 s of simulated time
    per run.  Cost: the paper's ball-task suite (Sec. IV-B), pick phase then
    move phase (switched when the end effectors' midpoint reaches the pick
    point), end effectors l_ball apart and the pick point eps below the
    ball's centre; --task -1 uses the scene's stage cost instead.  Reports
    the success rate, task time (mean and standard deviation over
    successful runs) and planning compute time (mean and standard deviation
    over every planning step)."""
    import numpy as np
    import torch
    from paper_2511_21264_gb300 import native
    rank, world, local = _dist_setup(args.gpus)
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    native.build() if rank == 0 and world == 1 else None
    native.lib()
    rng = np.random.default_rng(1000 + rank)
    K, H, M, n_avg, max_steps = args.k, args.cl_h, 10, 4, 800
    task = 0 if args.task is None else args.task
    task = None if task < 0 else task
    results = []
    stream = torch.cuda.Stream(device=dev)
    with ClockSampler(local) as clk:
        for run in range(args.runs):
            sc = scenes.config(1, seed=run)
            start = np.array(sc.x0[sc.nu:sc.nu + 3])
            sc.goal = tuple(start + np.array([rng.uniform(-0.1, 0.1), 0.0, rng.uniform(0.15, 0.3)]))
            m = native.Model(sc.to_blob())
            ctl = native.Controller(m, K, H, sc.lam, sc.sigma_vec(), scenes.controller_key(run, rank))
            if args.elite or args.eta != 1.0 or args.cov:
                ctl.set_update(args.elite or K, args.eta, args.cov, 1e-6)
            if args.qp:
                ctl.set_projection(scenes.projection_bounds(sc), iters=args.qp)
            if task is not None:
                ctl.set_task_cost(scenes.ball_task(sc, phase=task, eps=args.eps, l_ball=args.l_ball))
            u = torch.zeros((H, sc.nu), device=dev)
            with torch.cuda.stream(stream):
                ep = ctl.run_episode(sc.x0, u, iters=M, n_avg=n_avg, max_steps=max_steps, goal_tol=0.03,
                                     lift_dz=0.05, drop_dz=0.05, pick_tol=0.03 if task == 0 else 0.0,
                                     record=True, stream=stream)
            results.append(ep)
            ctl.close()
            m.close()
    if rank != 0:
        return 0
    ok = [r for r in results if r["outcome_name"] == "success"]
    comp = np.concatenate([r["comp_ms"] for r in results])
    tt = np.array([r["task_time_s"] for r in ok]) if ok else np.zeros(0)
    outcomes = {}
    for r in results:
        outcomes[r["outcome_name"]] = outcomes.get(r["outcome_name"], 0) + 1
    line = {
        "metric": "closed-loop success rate (%) of the planar ball lift, receding horizon (Sec. IV-A metrics)",
        "value": 100.0 * len(ok) / len(results), "unit": "%", "n_gpus": world, "steps": None, "warmup": 0,
        "ms_per_step": float(comp.mean()), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"planar 3-link bimanual ball lift, {args.runs} runs with randomised goals, K={K}, "
                               f"H={H}, M={M} iterations per plan, first {n_avg} steps averaged and executed, "
                               f"{max_steps} world steps ({max_steps * 0.01:g} s) per run",
                   "update": {"n_elite": args.elite or K, "eta": args.eta, "covariance": bool(args.cov)},
                   "projection_iters": args.qp,
                   "cost": (f"ball-task suite (Sec. IV-B), pick then move, l_ball={args.l_ball} m, eps={args.eps} m"
                            if task == 0 else ("ball-task suite, move" if task == 1 else "scene stage cost"))},
        "task_time_s": {"mean": float(tt.mean()) if tt.size else None, "std": float(tt.std()) if tt.size else None,
                        "n_success": len(ok)},
        "comp_time_ms": {"mean": float(comp.mean()), "std": float(comp.std()), "n_plans": int(comp.size)},
        "outcomes": outcomes,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=("lift", "transfer", "batched", "serve", "closed_loop"),
                    default="transfer",
                    help="transfer: 8-box transfer K=4096 H=64 (default; the line also carries the lift); "
                         "lift: 7-DoF ball lift K=1024 H=32; batched: 64 instances (K 256..4096, H 16..64, 0..16 boxes) in one "
                         "persistent launch vs 64 sequential plain launches; serve: Poisson replan "
                         "requests over 256 scenes, batched server vs one-at-a-time server; closed_loop: "
                         "receding-horizon episodes with the paper's success / task-time / compute-time metrics")
    ap.add_argument("--runs", type=int, default=20, help="closed_loop: episodes (the paper's N_runs = 20)")
    ap.add_argument("--k", type=int, default=1024, help="closed_loop: samples per iteration")
    ap.add_argument("--elite", type=int, default=0, help="elite set size (0 = all samples: the plain update)")
    ap.add_argument("--eta", type=float, default=1.0, help="learning rate of Eq. 8 (elite mode)")
    ap.add_argument("--cov", action="store_true", help="update the per-step covariance blocks (Eq. 8b/8c)")
    ap.add_argument("--qp", type=int, default=0, help="QP smoothing projection (Eq. 5) iterations (0 = off)")
    ap.add_argument("--task", type=int, choices=(-1, 0, 1), default=None,
                    help="the paper's ball-task cost suite in the given phase (0 pick, 1 move); closed_loop: "
                         "default 0 (pick, then move), -1 = the scene's stage cost")
    ap.add_argument("--cl-h", type=int, default=48, help="closed_loop: horizon (steps of 10 ms)")
    ap.add_argument("--l-ball", type=float, default=0.25, help="closed_loop: end-effector distance of the grasp (m)")
    ap.add_argument("--eps", type=float, default=0.02, help="closed_loop: pick point below the ball's centre (m)")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="arrival window per rate (serve)")
    ap.add_argument("--serve-classes", type=int, default=0,
                    help="serve: size classes of the batched server (0 = 6; 1 = one batch of all requests)")
    ap.add_argument("--serve-rates", type=str, default="50,200,1000")
    ap.add_argument("--spc", type=int, default=0, help="samples per CTA (0 = library default)")
    ap.add_argument("--lps", type=int, default=0, help="lanes per sample: 32, 16 (0 = library default)")
    ap.add_argument("--place", type=int, default=0, help="lone ball contact solve: 0 fused, 1 after the factor")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-lift", action="store_true", help="transfer: skip the extra lift measurement")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "closed_loop":
        return run_closed_loop(args)
    if args.task is not None and args.task < 0:
        args.task = None
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
