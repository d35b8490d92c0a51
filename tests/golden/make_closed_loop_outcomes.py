"""Writes closed_loop_outcomes_config1.json: the FP64 oracle's closed-loop
receding-horizon runs (Sec. III-A; outcome metrics of Sec. IV-A) on the
planar ball lift with the ball-task cost suite (Sec. IV-B), for the GPU
closed-loop tests to compare against.  Calls only the oracle and the seeded
scene generator.

Two parts:
- "runs": 100 episodes (seed s: scene config 1 with lift_goal(s), noise key
  controller_key(s, 1)), outcome and step counts of each;
- "first_plan": 12 single-plan episodes with noise key controller_key(s, 0),
  the executed control, the index of the lowest-cost sample and all sample
  costs of the plan's last iteration.

Run from the repository root:  python tests/golden/make_closed_loop_outcomes.py
(about half an hour on 8 cores; --keep-runs rewrites the first-plan part
only, keeping the stored runs when their setting is unchanged)."""
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.abspath(os.path.join(os.path.dirname(__file__), "..", "..")))
import oracle  # noqa: E402
from paper_2511_21264_gb300 import scenes  # noqa: E402

SETTING = dict(K=256, H=48, iters=5, n_avg=4, max_steps=300, goal_tol=0.03, lift_dz=0.05, drop_dz=0.05,
               pick_tol=0.03, eps=0.02, l_ball=0.25)
N_RUNS, N_FIRST = 100, 12
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "closed_loop_outcomes_config1.json")


def episode(seed, key_instance, max_steps, nthreads):
    s = SETTING
    sc = scenes.config(1, seed=seed)
    sc.goal = scenes.lift_goal(sc, seed)
    om = oracle.Model(sc.to_blob())
    task = scenes.ball_task(sc, phase=0, eps=s["eps"], l_ball=s["l_ball"])
    return oracle.run_episode(om, sc.x0, s["K"], s["H"], sc.lam, sc.sigma_vec(),
                              scenes.controller_key(seed, key_instance), s["iters"], s["n_avg"], max_steps,
                              s["goal_tol"], s["lift_dz"], s["drop_dz"], pick_tol=s["pick_tol"], task=task,
                              nthreads=nthreads)


def first_plan(seed, nthreads):
    # the same single plan, with its last iteration's costs for the gap
    s = SETTING
    sc = scenes.config(1, seed=seed)
    sc.goal = scenes.lift_goal(sc, seed)
    om = oracle.Model(sc.to_blob())
    task = scenes.ball_task(sc, phase=0, eps=s["eps"], l_ball=s["l_ball"])
    key = scenes.controller_key(seed, 0)
    u = np.zeros((s["H"], sc.nu))
    for it in range(s["iters"]):
        r = om.mppi_iteration(sc.x0, u, s["K"], sc.lam, sc.sigma_vec(), key, it, nthreads=nthreads,
                              want_samples=True, task=task)
        u = r["u_nom"]
    costs = np.where(np.isfinite(r["costs"]), r["costs"], np.inf)
    ep = episode(seed, 0, s["n_avg"], nthreads)
    return dict(seed=seed, u_exec0=ep["u_exec"][0].tolist(), best=int(np.argmin(costs)),
                costs=[float(c) for c in r["costs"]])


def main():
    nthreads = os.cpu_count() or 1
    t0 = time.time()
    runs = []
    if "--keep-runs" in sys.argv and os.path.exists(OUT):
        old = json.load(open(OUT))
        if old["setting"] == SETTING and len(old["runs"]) == N_RUNS:
            runs = old["runs"]
    for seed in range(len(runs), N_RUNS):
        ep = episode(seed, 1, SETTING["max_steps"], nthreads)
        runs.append(dict(seed=seed, outcome=ep["outcome"], steps=ep["steps"], plans=ep["plans"],
                         switch_step=ep["switch_step"]))
        print(seed, ep["outcome"], ep["steps"], f"{time.time() - t0:.0f}s", flush=True)
    first = [first_plan(seed, nthreads) for seed in range(N_FIRST)]
    counts = {}
    for r in runs:
        counts[r["outcome"]] = counts.get(r["outcome"], 0) + 1
    doc = dict(
        source="oracle.run_episode (FP64), written by tests/golden/make_closed_loop_outcomes.py",
        passage="Sec. III-A receding horizon; Sec. IV-A outcome metrics; Sec. IV-B ball-task cost suite",
        scene="config 1 (planar 3-link arms, ball lift), goal scenes.lift_goal(seed)",
        setting=SETTING, runs_key_instance=1, first_plan_key_instance=0, counts=counts, runs=runs,
        first_plan=first)
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
    print("counts", counts, f"{time.time() - t0:.0f}s")


if __name__ == "__main__":
    main()
