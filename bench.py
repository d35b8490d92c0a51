"""Throughput benchmark of the MPPI + contact-rollout hot path.

A step is one MPPI iteration (Alg. 1 loop body: Philox sampling, H-step
contact rollouts of K samples, stage costs, softmax weights, weighted-mean
update) of the two 7-DoF arms / 0.12 m ball lift scene with K = 1024
samples and H = 32 steps (dt = 0.01 s, 4 PGS sweeps), on synthetic seeded
inputs.  value = simulated sample-steps/s = K * H * steps / time over all
ranks (each rank runs its own independent controller: weak scaling).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

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


def _config_json(sc, n_gpus):
    return {"workload": WORKLOAD, "scene": sc.name, "K": sc.K, "H": sc.H, "nv": sc.nv, "n_boxes": sc.n_boxes,
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
    return {"value": done / el, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "sample": f"{it} MPPI iterations of K'={Kp} samples (of K={sc.K}), H={sc.H}, same scene; "
                      f"{el:.1f} s of FP64 work on {nthreads} threads"}


def run_reference(args):
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return 0
    sc = scenes.config(2)
    nthreads = os.cpu_count() or 1
    import oracle
    om = oracle.Model(sc.to_blob())
    x = sc.x0.astype(np.float32).astype(np.float64)
    u = np.zeros((sc.H, sc.nu))
    Kp = max(2 * nthreads, 16)   # bounded sample per step
    for w in range(args.warmup):
        om.mppi_iteration(x, u, Kp, sc.lam, sc.sigma_vec(), 1, w, nthreads=nthreads)
    t0 = time.perf_counter()
    for s in range(args.steps):
        om.mppi_iteration(x, u, Kp, sc.lam, sc.sigma_vec(), 1, args.warmup + s, nthreads=nthreads)
    el = time.perf_counter() - t0
    value = Kp * sc.H * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config_json(sc, args.gpus),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                             "sample": f"each step: one MPPI iteration with K'={Kp} of K={sc.K} samples"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    from paper_2511_21264_gb300 import native

    rank, world, local = _dist_setup(args.gpus)
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    native.build() if rank == 0 and world == 1 else None
    native.lib()
    sc = scenes.config(2)
    K, H = sc.K, sc.H
    model = native.Model(sc.to_blob())
    ctl = native.Controller(model, K, H, sc.lam, sc.sigma_vec(), scenes.controller_key(sc.seed, rank))
    if args.spc:
        ctl.set_launch(args.spc)
    stream = torch.cuda.Stream(device=dev)
    x = torch.tensor(model.home(), device=dev)
    u = torch.zeros((H, sc.nu), device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            ctl.step(x, u, u, stream=stream)
        stream.synchronize()
        _barrier(world)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        ctl.profile(args.steps)
        with ClockSampler(local) as clk:
            time.sleep(0.3)
            for i in range(args.steps):
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
        ctl.profile(0)

        # end to end through the public API with host buffers: pinned H2D
        # copy of (state, u_nom), the iteration, D2H read of u_nom'
        xh = torch.tensor(model.home()).pin_memory()
        uh = torch.zeros((H, sc.nu)).pin_memory()
        uo = torch.empty((H, sc.nu)).pin_memory()
        xd, ud = torch.empty_like(x), torch.empty_like(u)
        _barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(args.steps):
            xd.copy_(xh, non_blocking=True)
            ud.copy_(uh, non_blocking=True)
            ctl.step(xd, ud, ud, stream=stream)
            uo.copy_(ud, non_blocking=True)
            stream.synchronize()
            uh.copy_(uo)
        e1.record(stream)
        stream.synchronize()
        e2e_ms = _max_over_ranks(e0.elapsed_time(e1), world)

    units = K * H * args.steps * world
    value = units / (total_ms * 1e-3)
    e2e = units / (e2e_ms * 1e-3)
    clocks = clk.summary()
    if rank != 0:
        return 0
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_mhz = clocks["sm_mhz"] or 1477.0
    peak = sms * 128 * 2 * sm_mhz * 1e6 / 1e12
    fl = flops.per_sample_step(sc, kt["contacts_per_step"], kt["box_tests_per_step"])
    roll_ms = kt["rollout_ms"] / max(1, kt["iterations"])
    achieved = fl * K * H / (roll_ms * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": _config_json(sc, world),
        "iters_per_s": args.steps * world / (total_ms * 1e-3),
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": int(4 * (x.numel() + u.numel())),
                "d2h_bytes_per_step": int(4 * u.numel())},
        "gpu_launches": 2 * args.steps,
        "roofline": {"bound": "alu", "kernel": "rollout_kernel<7,1>", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak, "traffic": args.traffic,
                     "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz (median SM clock "
                                   f"sampled during the timed steps)",
                     "flops_per_sample_step": fl, "rollout_ms": roll_ms,
                     "update_ms": kt["update_ms"] / max(1, kt["iterations"]),
                     "contacts_per_step": kt["contacts_per_step"],
                     "box_tests_per_step": kt["box_tests_per_step"]},
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(sc, seconds=args.cpu_seconds)
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--spc", type=int, default=0, help="samples per CTA (0 = library default)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per rollout launch from an ncu capture (else null)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
