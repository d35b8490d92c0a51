"""Closed-form pins for the oracle's stage cost, its time indexing and the
ball's orientation step.

- stage cost: every term of the workloads' cost (goal distance, control
  effort, penetration depth, obstacle penetration, grasp maintenance) on
  hand-placed states whose values are known in closed form, with the weights
  the workloads state (10, 0.01, 100, 50, 1);
- penetration sums: a ball pressed a known depth into the floor or a box,
  and arm links pressed a known depth into a box face;
- indexing (reading A6): position terms on x_{h+1}, effort on u_h and the
  penetration found while stepping from x_h, over a two-step rollout;
- orientation: with no contact and no gravity a constant world-frame spin
  w turns the ball by |w| n dt about w/|w| after n steps, composed on the
  left of the start orientation.
"""
import copy
import math

import numpy as np
import pytest

import oracle
from paper_2511_21264_gb300 import scenes
from tests import helpers


def _dh_home_ee(sc):
    """Distal capsule ends of the straight, tilted DH home arms in closed form."""
    t = scenes.DH_HOME_TILT
    out = []
    for a, sx in ((0, 1.0), (1, -1.0)):
        L = sum(ln.F_p[0] for ln in sc.links[a])
        out.append(sc.base_p[a] + L * np.array([sx * math.sin(t), 0.0, math.cos(t)]))
    return out


def test_transfer_weights_are_the_stated_ones():
    sc = scenes.config(3)
    assert (sc.w_goal, sc.w_u, sc.w_pen, sc.w_obst, sc.w_grasp) == (10.0, 0.01, 100.0, 50.0, 1.0)
    sc1 = scenes.config(1)
    assert (sc1.w_goal, sc1.w_u, sc1.w_pen, sc1.w_obst, sc1.w_grasp) == (10.0, 0.01, 100.0, 0.0, 0.0)


def test_stage_cost_terms_closed_form():
    sc = scenes.config(3)
    m = oracle.Model(sc.to_blob())
    b0 = 2 * sc.n_a
    goal = np.array(sc.goal)
    pL, pR = _dh_home_ee(sc)
    rng = np.random.default_rng(11)
    for _ in range(6):
        d = rng.normal(size=3) * 0.2
        u = rng.normal(size=sc.nu)
        pen_all, pen_box = rng.uniform(0, 0.01), rng.uniform(0, 0.005)
        x = sc.x0.copy()
        x[b0:b0 + 3] = goal + d
        info = oracle.StepInfo(0, 0, pen_all, pen_box, 0)
        grasp = np.sum((pL + pR - 2.0 * (goal + d)) ** 2)
        want = 10.0 * d @ d + 0.01 * u @ u + 100.0 * pen_all + 50.0 * pen_box + 1.0 * grasp
        assert m.stage_cost(x, u, info) == pytest.approx(want, rel=1e-13, abs=1e-13)
        # one term at a time: the ball at the goal, no control, no penetration
        # leaves the grasp term alone; each further term adds its own value
        x[b0:b0 + 3] = goal
        z = np.zeros(sc.nu)
        g0 = np.sum((pL + pR - 2.0 * goal) ** 2)
        none = oracle.StepInfo(0, 0, 0.0, 0.0, 0)
        assert m.stage_cost(x, z, none) == pytest.approx(g0, rel=1e-13)
        assert m.stage_cost(x, u, none) - g0 == pytest.approx(0.01 * u @ u, rel=1e-12)
        assert (m.stage_cost(x, z, oracle.StepInfo(0, 0, pen_all, 0.0, 0)) - g0
                == pytest.approx(100.0 * pen_all, rel=1e-12))
        assert (m.stage_cost(x, z, oracle.StepInfo(0, 0, 0.0, pen_box, 0)) - g0
                == pytest.approx(50.0 * pen_box, rel=1e-12))


def test_goal_term_alone_on_the_planar_lift():
    # config 1 has no grasp term: the cost of a displaced ball is 10 |d|^2
    sc = scenes.config(1)
    m = oracle.Model(sc.to_blob())
    b0 = 2 * sc.n_a
    none = oracle.StepInfo(0, 0, 0.0, 0.0, 0)
    for d in ((0.1, 0.0, 0.0), (0.0, -0.3, 0.0), (0.05, 0.02, -0.3)):
        x = sc.x0.copy()
        x[b0:b0 + 3] = np.array(sc.goal) + np.array(d)
        assert m.stage_cost(x, np.zeros(sc.nu), none) == pytest.approx(10.0 * np.dot(d, d), rel=1e-13)


def _one_box(sc, c, h):
    sc = copy.deepcopy(sc)
    sc.boxes_c = np.array([c], dtype=float)
    sc.boxes_h = np.array([h], dtype=float)
    return sc


def test_penetration_of_ball_into_floor_and_box():
    base = scenes.config(3)
    b0 = 2 * base.n_a
    r = base.ball_r
    for delta in (1e-4, 3e-3, 2e-2):
        # ball pressed into the floor, far from arms and boxes
        sc = _one_box(base, (0.0, 3.0, 0.5), (0.1, 0.1, 0.1))
        m = oracle.Model(sc.to_blob())
        x = sc.x0.copy()
        x[b0:b0 + 3] = (0.0, -2.0, r - delta)
        _, info = m.step(x, np.zeros(sc.nu))
        assert info.pen_all == pytest.approx(delta, abs=1e-14)
        assert info.pen_box == 0.0
        # ball pressed into the top face of a box, clear of the floor
        x[b0:b0 + 3] = (0.0, 3.0, 0.6 + r - delta)
        _, info = m.step(x, np.zeros(sc.nu))
        assert info.pen_all == pytest.approx(delta, abs=1e-14)
        assert info.pen_box == pytest.approx(delta, abs=1e-14)
        # both at once: a box resting on the floor, the ball in its side face
        sc2 = _one_box(base, (0.0, 3.0, 0.2), (0.2, 0.2, 0.2))
        m2 = oracle.Model(sc2.to_blob())
        x[b0:b0 + 3] = (0.0, 3.0 - 0.2 - r + 2 * delta, r - delta)
        _, info = m2.step(x, np.zeros(sc.nu))
        assert info.pen_all == pytest.approx(3 * delta, abs=1e-14)
        assert info.pen_box == pytest.approx(2 * delta, abs=1e-14)


def test_penetration_of_links_into_a_box_face():
    # The home arms lie in the plane y = 0.  A large box whose -y face sits at
    # y = r_cap - delta covers the projection of every link: each of the 14
    # capsules then penetrates it by exactly delta.
    base = scenes.config(3)
    b0 = 2 * base.n_a
    rc = base.links[0][0].radius
    for delta in (1e-3, 1e-2):
        hy = 0.5
        sc = _one_box(base, (0.0, rc - delta + hy, 0.5), (2.0, hy, 2.0))
        m = oracle.Model(sc.to_blob())
        x = sc.x0.copy()
        x[b0:b0 + 3] = (0.0, -3.0, 1.0)    # ball clear of everything
        _, info = m.step(x, np.zeros(sc.nu))
        assert info.nactive == 14
        assert info.pen_box == pytest.approx(14 * delta, abs=1e-10)
        assert info.pen_all == pytest.approx(14 * delta, abs=1e-10)


def test_stage_cost_indexing_over_two_steps():
    # Reading A6: c_h = w_g |p_ball(x_{h+1}) - goal|^2 + w_u |u_h|^2
    #                  + w_p * (depth found at x_h), summed over h = 0, 1.
    # The ball sinks into the floor, so every term differs between the
    # candidate indexings.
    sc = scenes.config(1)
    m = oracle.Model(sc.to_blob())
    b0, nq = 2 * sc.n_a, sc.nq
    r = sc.ball_r
    x = sc.x0.copy()
    x[b0:b0 + 3] = (0.0, 2.0, r - 0.004)
    x[nq + b0 + 2] = -0.3
    U = np.array([[0.5, -1.0, 0.2, 0.0, 0.3, 0.7], [-0.4, 0.1, 0.9, 1.2, -0.8, 0.05]])
    total, traj = m.rollout(x, U, traj=True)
    goal = np.array(sc.goal)
    want = 0.0
    for h in range(2):
        pb_next = traj[h + 1, b0:b0 + 3]
        depth_h = max(0.0, r - traj[h, b0 + 2])
        want += 10.0 * np.sum((pb_next - goal) ** 2) + 0.01 * U[h] @ U[h] + 100.0 * depth_h
    assert total == pytest.approx(want, rel=1e-13)
    # the alternative readings give clearly different totals
    alt_pos = sum(10.0 * np.sum((traj[h, b0:b0 + 3] - goal) ** 2) + 0.01 * U[h] @ U[h]
                  + 100.0 * max(0.0, r - traj[h, b0 + 2]) for h in range(2))
    alt_pen = sum(10.0 * np.sum((traj[h + 1, b0:b0 + 3] - goal) ** 2) + 0.01 * U[h] @ U[h]
                  + 100.0 * max(0.0, r - traj[h + 1, b0 + 2]) for h in range(2))
    assert abs(alt_pos - want) > 1e-3 and abs(alt_pen - want) > 1e-3


def _qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def _axis_angle(axis, angle):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    return np.concatenate([[math.cos(angle / 2)], math.sin(angle / 2) * axis])


def _rotate(q, v):
    p = _qmul(_qmul(q, np.concatenate([[0.0], v])), q * np.array([1, -1, -1, -1]))
    return p[1:]


@pytest.mark.parametrize("w", [(0.0, 0.0, 3.0), (0.3, -1.1, 2.0), (25.0, 10.0, -40.0)])
def test_ball_orientation_under_constant_world_spin(w):
    sc = helpers.ball_far(scenes.config(1), pos=(0.0, 5.0, 2.0))
    sc = copy.deepcopy(sc)
    sc.gravity = (0.0, 0.0, 0.0)
    m = oracle.Model(sc.to_blob())
    b0, nq = 2 * sc.n_a, sc.nq
    q0 = _qmul(_axis_angle((1.0, 0.2, 0.0), 1.0), _axis_angle((0.0, 0.0, 1.0), 0.4))
    x = sc.x0.copy()
    x[b0 + 3:b0 + 7] = q0
    x[nq + b0 + 3:nq + b0 + 6] = w
    wv = np.array(w)
    n_steps = 60
    for n in range(1, n_steps + 1):
        x, info = m.step(x, np.zeros(sc.nu))
        assert info.ncon == 0
        np.testing.assert_array_equal(x[nq + b0 + 3:nq + b0 + 6], wv)
        qn = _qmul(_axis_angle(wv, np.linalg.norm(wv) * n * sc.dt), q0)
        got = x[b0 + 3:b0 + 7]
        assert min(np.abs(got - qn).max(), np.abs(got + qn).max()) < 1e-12
    # the body-frame composition q0 * dq gives another orientation here
    body = _qmul(q0, _axis_angle(wv, np.linalg.norm(wv) * n_steps * sc.dt))
    assert min(np.abs(got - body).max(), np.abs(got + body).max()) > 1e-3
    # a point fixed on the ball moves by the world-frame rotation
    v_body = np.array([0.3, -0.5, 0.8])
    turned = _rotate(_axis_angle(wv, np.linalg.norm(wv) * n_steps * sc.dt), _rotate(q0, v_body))
    np.testing.assert_allclose(_rotate(got, v_body), turned, atol=1e-12)
