"""Pins of the oracle's closed-loop receding-horizon driver (Sec. III-A; the
outcome metrics of Sec. IV-A): each outcome on a scene built so that the
outcome and its world step follow from elementary kinematics, the pick ->
move switch, the timeout count, and the warm-start shift."""
import numpy as np
import pytest

import oracle
from paper_2511_21264_gb300 import scenes

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

K, H = 8, 4


def _run(sc, task=None, goal=None, **kw):
    om = oracle.Model(sc.to_blob())
    args = dict(iters=1, n_avg=2, max_steps=6, goal_tol=0.03, lift_dz=0.05, drop_dz=0.05)
    args.update(kw)
    return om, oracle.run_episode(om, sc.x0, K, H, sc.lam, sc.sigma_vec(), scenes.controller_key(1, 0),
                                  task=task, goal=goal if goal is not None else sc.goal, **args)


def _ball(sc):
    return 2 * sc.n_a


def test_success_on_the_first_world_step_when_the_ball_starts_at_the_goal():
    sc = scenes.config(1)
    b = _ball(sc)
    sc.goal = tuple(sc.x0[b:b + 3] + np.array([0.0, 0.0, 0.01]))
    om, ep = _run(sc)
    assert ep["outcome"] == "success" and ep["steps"] == 1 and ep["plans"] == 1
    # the task suite's target is the goal when the suite is on
    task = scenes.ball_task(sc, phase=1)
    om, ep = _run(sc, task=task, goal=np.array([5.0, 5.0, 5.0]))
    assert ep["outcome"] == "success" and ep["steps"] == 1


def test_timeout_counts_world_steps_and_plans():
    sc = scenes.config(1)
    om, ep = _run(sc, max_steps=7, n_avg=3)
    assert ep["outcome"] == "timeout" and ep["steps"] == 7 and ep["plans"] == 3
    assert ep["traj"].shape == (8, sc.nq + sc.nv) and ep["u_exec"].shape == (7, sc.nu)
    # the executed control is held for n_avg world steps
    np.testing.assert_array_equal(ep["u_exec"][0], ep["u_exec"][2])
    assert np.abs(ep["u_exec"][3] - ep["u_exec"][2]).max() > 0


def test_collision_when_a_link_starts_inside_a_box():
    sc = scenes.config(1)
    om = oracle.Model(sc.to_blob())
    a0 = om.fk(sc.x0[:sc.nq])["a0"][0][1]          # the left arm's second link
    sc.boxes_c = a0[None, :].copy()
    sc.boxes_h = np.array([[0.05, 0.05, 0.05]])
    om, ep = _run(sc)
    assert ep["outcome"] == "collision" and ep["steps"] == 1


def test_drop_step_of_a_ball_thrown_upwards_away_from_the_arms():
    # The ball starts 1.5 m to the side and 1 m up with v_z = 1 m/s: it
    # rises, peaks and falls freely (the arms cannot reach it).  With
    # lift_dz = 0 it counts as lifted after the first step, and the drop is
    # reported on the first step whose height is more than drop_dz below
    # the highest so far, under semi-implicit Euler (v += g dt, z += v dt).
    sc = scenes.config(1)
    b = _ball(sc)
    x0 = sc.x0.copy()
    x0[b:b + 3] = [1.5, 0.0, 1.0]
    x0[sc.nq + b + 2] = 1.0
    sc.x0 = x0
    drop_dz, dt, g = 0.02, sc.dt, 9.81
    z, v, zmax, n = 1.0, 1.0, 1.0, 0
    while True:
        v -= g * dt
        z += v * dt
        n += 1
        zmax = max(zmax, z)
        if z < zmax - drop_dz:
            break
    om, ep = _run(sc, max_steps=200, lift_dz=0.0, drop_dz=drop_dz)
    assert ep["outcome"] == "dropped" and ep["steps"] == n


def test_pick_switch_and_its_tolerance():
    sc = scenes.config(1)
    task = scenes.ball_task(sc, phase=0)
    om = oracle.Model(sc.to_blob())
    mid = om.ee_state(sc.x0)["p"].mean(axis=0)
    pick = task[12:15] - np.array([0.0, 0.0, task[11]])
    d0 = np.linalg.norm(mid - pick)
    _, ep = _run(sc, task=task, goal=None, pick_tol=d0 + 0.5)
    assert ep["switch_step"] == 1
    _, ep = _run(sc, task=task, goal=None, pick_tol=0.0)
    assert ep["switch_step"] == -1
    # the switch changes the cost of later plans: the same run with the
    # move phase from the start differs from the first plan on only
    _, e0 = _run(sc, task=task, goal=None, pick_tol=d0 + 0.5, n_avg=1, max_steps=3)
    t1 = task.copy()
    t1[0] = 1.0
    _, e1 = _run(sc, task=t1, goal=None, n_avg=1, max_steps=3)
    assert np.abs(e0["u_exec"][0] - e1["u_exec"][0]).max() > 0


def test_warm_start_shift_and_iteration_counter():
    # Two plans of n_avg = 2 with 2 iterations each: the second plan starts
    # from the first plan's nominal sequence shifted by two steps (the last
    # step repeated) and draws noise blocks 2 and 3.
    sc = scenes.config(1)
    om = oracle.Model(sc.to_blob())
    seed, sig = scenes.controller_key(1, 0), sc.sigma_vec()
    ep = oracle.run_episode(om, sc.x0, K, H, sc.lam, sig, seed, iters=2, n_avg=2, max_steps=4, goal_tol=0.03,
                            lift_dz=0.05, drop_dz=0.05, goal=sc.goal)
    x, u = sc.x0.astype(np.float64), np.zeros((H, sc.nu))
    for it in (0, 1):
        r = om.mppi_iteration(x, u, K, sc.lam, sig, seed, it, want_samples=True)
        u = r["u_nom"]
    x2 = ep["traj"][2]
    u_shift = np.vstack([u[2:], u[3:4], u[3:4]])
    for it in (2, 3):
        r = om.mppi_iteration(x2, u_shift, K, sc.lam, sig, seed, it, want_samples=True)
        u_shift = r["u_nom"]
    k = int(np.argmin(r["costs"]))
    np.testing.assert_array_equal(ep["u_exec"][2], r["U"][k, :2].mean(axis=0))


def test_stored_closed_loop_outcomes_reproduce():
    # The stored FP64 closed-loop outcomes (tests/golden, written by
    # make_closed_loop_outcomes.py from the oracle alone): the shortest
    # stored run and the first single-plan record, re-run here.
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "closed_loop_outcomes_config1.json")
    doc = json.load(open(path))
    s = doc["setting"]

    def run(seed, inst, max_steps):
        sc = scenes.config(1, seed=seed)
        sc.goal = scenes.lift_goal(sc, seed)
        om = oracle.Model(sc.to_blob())
        task = scenes.ball_task(sc, phase=0, eps=s["eps"], l_ball=s["l_ball"])
        return oracle.run_episode(om, sc.x0, s["K"], s["H"], sc.lam, sc.sigma_vec(),
                                  scenes.controller_key(seed, inst), s["iters"], s["n_avg"], max_steps,
                                  s["goal_tol"], s["lift_dz"], s["drop_dz"], pick_tol=s["pick_tol"], task=task,
                                  nthreads=os.cpu_count() or 1)
    r = min(doc["runs"], key=lambda r: r["steps"])
    ep = run(r["seed"], doc["runs_key_instance"], s["max_steps"])
    assert (ep["outcome"], ep["steps"], ep["plans"]) == (r["outcome"], r["steps"], r["plans"])
    f = doc["first_plan"][0]
    ep = run(f["seed"], doc["first_plan_key_instance"], s["n_avg"])
    np.testing.assert_allclose(ep["u_exec"][0], f["u_exec0"], rtol=0, atol=1e-12)
    assert len(doc["runs"]) == 100 and doc["counts"] == {o: sum(1 for q in doc["runs"] if q["outcome"] == o)
                                                        for o in doc["counts"]}
