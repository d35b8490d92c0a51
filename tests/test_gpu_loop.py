"""Closed-loop receding horizon (mppi_run_episode) on the GPU: the driver's
steps against the same steps made through the C ABI by hand (bitwise), the
world steps against the FP64 oracle's simulator (single-step tolerance
1e-4 max(1, |x|)), outcomes, statistics and determinism; the first planning
step's executed control and the outcome rates of 100 runs against the
oracle's closed loop."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2511_21264_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


@pytest.fixture(scope="module")
def native():
    from paper_2511_21264_gb300 import native as nat
    nat.build()
    nat.lib()
    return nat


def _ctl(native, sc, K=64, H=16, key=9):
    gm = native.Model(sc.to_blob())
    return gm, native.Controller(gm, K, H, sc.lam, sc.sigma_vec(), key)


def test_episode_equals_the_steps_made_by_hand(native):
    sc = scenes.config(1)
    K, H, iters, n_avg = 64, 16, 3, 4
    gm, ctl = _ctl(native, sc, K, H)
    u = torch.zeros((H, sc.nu), device=DEV)
    ep = ctl.run_episode(sc.x0, u, iters=iters, n_avg=n_avg, max_steps=8, goal_tol=1e-6)
    assert ep["outcome_name"] == "timeout" and ep["steps"] == 8 and ep["plans"] == 2
    # by hand, on a second controller with the same key
    gm2, c2 = _ctl(native, sc, K, H)
    u2 = torch.zeros((H, sc.nu), device=DEV)
    world = torch.tensor(sc.x0, dtype=torch.float32, device=DEV)
    best = torch.zeros(2, device=DEV)
    S = torch.empty((H, K, sc.nu), device=DEV)
    states, execs = [world.cpu().numpy()], []
    for plan in range(2):
        c2.solve(world, u2, iters, best=best)
        c2.samples(S)
        k = int(best[1].item())
        acc = S[0, k, :].clone()
        for h in range(1, n_avg):  # the driver's summation order
            acc = acc + S[h, k, :]
        u1 = acc / n_avg
        for _ in range(n_avg):
            c2.sim_step(world.view(1, -1), u1.view(1, -1).contiguous())
            states.append(world.cpu().numpy())
            execs.append(u1.cpu().numpy())
        u2 = torch.cat([u2[n_avg:], u2[-1:].expand(n_avg, sc.nu)]).contiguous()
    assert c2.sync() == 0
    np.testing.assert_array_equal(ep["traj"], np.array(states))
    np.testing.assert_array_equal(ep["u_exec"], np.array(execs))


def test_world_steps_match_the_oracle_simulator(native):
    sc = scenes.config(1)
    gm, ctl = _ctl(native, sc, K=128, H=16)
    om = oracle.Model(sc.to_blob())
    u = torch.zeros((16, sc.nu), device=DEV)
    ep = ctl.run_episode(sc.x0, u, iters=4, n_avg=4, max_steps=40, goal_tol=1e-6)
    traj, uex = ep["traj"].astype(np.float64), ep["u_exec"].astype(np.float64)
    checked = 0
    for m in range(ep["steps"]):
        if om.min_abs_dist(traj[m]) < 1e-4:
            continue
        xo, _ = om.step(traj[m], uex[m])
        tol = 1e-4 * max(1.0, np.abs(xo).max())
        assert np.abs(xo - traj[m + 1]).max() <= tol, m
        checked += 1
    assert checked >= ep["steps"] // 2


def test_outcomes_and_statistics(native):
    sc = scenes.config(1)
    gm, ctl = _ctl(native, sc)
    u = torch.zeros((16, sc.nu), device=DEV)
    ok = ctl.run_episode(sc.x0, u, iters=2, n_avg=2, max_steps=10, goal_tol=10.0)
    assert ok["outcome_name"] == "success" and ok["steps"] == 1 and ok["plans"] == 1
    assert ok["task_time_s"] == pytest.approx(sc.dt)
    to = ctl.run_episode(sc.x0, u, iters=2, n_avg=3, max_steps=7, goal_tol=1e-6)
    assert to["outcome_name"] == "timeout" and to["steps"] == 7 and to["plans"] == 3
    c = to["comp_ms"].astype(np.float64)
    assert np.all(c > 0)
    assert to["comp_mean_ms"] == pytest.approx(c.mean(), rel=1e-5)
    assert to["comp_std_ms"] == pytest.approx(c.std(), rel=1e-3, abs=1e-6)
    # a box through a link at the start: a collision on the first step
    sc2 = scenes.dh_scene(seed=3, n_boxes=1, K=64, H=8)
    om = oracle.Model(sc2.to_blob())
    fk = om.fk(sc2.x0[:om.nq])
    mid = 0.5 * (fk["a0"][0][2] + fk["a1"][0][2])
    sc2.boxes_c = mid[None, :].copy()
    sc2.boxes_h = np.array([[0.05, 0.05, 0.05]])
    gm2 = native.Model(sc2.to_blob())
    c2 = native.Controller(gm2, 64, 8, sc2.lam, sc2.sigma_vec(), 1)
    col = c2.run_episode(sc2.x0, torch.zeros((8, sc2.nu), device=DEV), iters=1, n_avg=1, max_steps=5)
    assert col["outcome_name"] == "collision" and col["steps"] == 1


def test_phase_switch_and_determinism(native):
    sc = scenes.config(1)
    runs = []
    for _ in range(2):
        gm, ctl = _ctl(native, sc, K=64, H=16, key=21)
        ctl.set_task_cost(scenes.ball_task(sc, phase=0))
        u = torch.zeros((16, sc.nu), device=DEV)
        runs.append(ctl.run_episode(sc.x0, u, iters=2, n_avg=4, max_steps=12, goal_tol=1e-6, pick_tol=10.0))
    a, b = runs
    assert a["switch_step"] == 1
    np.testing.assert_array_equal(a["traj"], b["traj"])
    np.testing.assert_array_equal(a["u_exec"], b["u_exec"])


def test_episode_with_projection_and_full_update(native):
    sc = scenes.config(2)
    gm, ctl = _ctl(native, sc, K=128, H=16)
    ctl.set_projection(scenes.projection_bounds(sc), iters=20)
    ctl.set_update(16, 0.7, True, 1e-6)
    u = torch.zeros((16, sc.nu), device=DEV)
    ep = ctl.run_episode(sc.x0, u, iters=2, n_avg=4, max_steps=8, goal_tol=1e-6)
    assert ep["steps"] == 8 and ep["plans"] == 2
    assert np.all(np.isfinite(ep["traj"]))
    # executed controls respect the projection's velocity bounds (to the ADMM tolerance)
    assert np.abs(ep["u_exec"]).max() <= np.pi * 1.05


# -- closed-loop outcomes against the oracle's (Sec. IV-A metrics) ---------
GOLDEN_CL = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                         "closed_loop_outcomes_config1.json")


def _cl_controller(native, s, seed, key_instance):
    sc = scenes.config(1, seed=seed)
    sc.goal = scenes.lift_goal(sc, seed)
    gm = native.Model(sc.to_blob())
    ctl = native.Controller(gm, s["K"], s["H"], sc.lam, sc.sigma_vec(), scenes.controller_key(seed, key_instance))
    ctl.set_task_cost(scenes.ball_task(sc, phase=0, eps=s["eps"], l_ball=s["l_ball"]))
    return sc, gm, ctl


def _cl_episode(native, s, seed, key_instance, max_steps):
    sc, gm, ctl = _cl_controller(native, s, seed, key_instance)
    u = torch.zeros((s["H"], sc.nu), device=DEV)
    ep = ctl.run_episode(sc.x0, u, iters=s["iters"], n_avg=s["n_avg"], max_steps=max_steps,
                         goal_tol=s["goal_tol"], lift_dz=s["lift_dz"], drop_dz=s["drop_dz"],
                         pick_tol=s["pick_tol"], record=True)
    ctl.close()
    gm.close()
    return ep


def test_first_plan_executes_the_oracles_control(native):
    # Same noise key as the oracle's stored single plans.  The lowest-cost
    # sample of the plan's last iteration is unique unless two costs are
    # within the FP32 rollouts' tolerance (1e-3 relative): where the GPU
    # picks the oracle's sample, the executed control (mean of its first
    # n_avg rows) must match; where it picks another, that sample's oracle
    # cost must tie with the lowest.
    doc = json.load(open(GOLDEN_CL))
    s = doc["setting"]
    same = 0
    for rec in doc["first_plan"]:
        sc, gm, ctl = _cl_controller(native, s, rec["seed"], doc["first_plan_key_instance"])
        u = torch.zeros((s["H"], sc.nu), device=DEV)
        best = torch.zeros(2, device=DEV)
        ctl.solve(torch.tensor(_f32(sc.x0), device=DEV), u, s["iters"], best=best)
        assert ctl.sync() == 0
        k = int(best[1].item())
        ctl.close()
        gm.close()
        costs = np.array(rec["costs"])
        if k == rec["best"]:
            ep = _cl_episode(native, s, rec["seed"], doc["first_plan_key_instance"], s["n_avg"])
            np.testing.assert_allclose(ep["u_exec"][0], np.array(rec["u_exec0"]), atol=1e-3, rtol=0)
            same += 1
        else:
            cmin = costs[rec["best"]]
            assert costs[k] - cmin <= 1e-3 * abs(cmin), (rec["seed"], k, rec["best"])
    assert same >= len(doc["first_plan"]) // 2


def test_closed_loop_outcome_rates_match_the_oracle(native):
    # 100 closed-loop runs of the planar ball lift on the GPU against the
    # oracle's 100 (same scenes and goals, independent noise keys): for each
    # outcome a two-proportion z test, |z| < 2.576 (two-sided, alpha = 0.01).
    doc = json.load(open(GOLDEN_CL))
    s = doc["setting"]
    n = len(doc["runs"])
    gpu = [_cl_episode(native, s, r["seed"], 0, s["max_steps"])["outcome_name"] for r in doc["runs"]]
    ora = [r["outcome"] for r in doc["runs"]]
    for outcome in oracle.EPISODE_OUTCOMES:
        x1, x2 = gpu.count(outcome), ora.count(outcome)
        p = (x1 + x2) / (2 * n)
        if p in (0.0, 1.0):
            continue
        z = (x1 / n - x2 / n) / math.sqrt(p * (1 - p) * 2 / n)
        assert abs(z) < 2.576, (outcome, x1, x2, z)
    # the comparison has power only if some outcome is neither rare nor certain
    assert any(10 <= ora.count(o) <= n - 10 for o in oracle.EPISODE_OUTCOMES)
