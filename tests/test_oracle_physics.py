"""Closed-form pins for the oracle's time stepping and soft contact model.

- free fall: the discrete closed form of semi-implicit Euler, exactly;
- physical pendulum period 2 pi sqrt(I_pivot / (m g l_c));
- energy with contacts off and no damping: the error vanishes at first
  order in dt;
- resting ball on a soft contact: depth g dt^2 (1-d)/(d ERP), zero
  velocity, normal impulse m g dt;
- a sliding ball starts rolling at 5/7 of its initial speed after
  2 v0 / (7 mu g);
- the implicit velocity servo settles at gear*u / (kv + damping).
"""
import copy
import math

import numpy as np
import pytest

import oracle
from paper_2511_21264_gb300 import scenes
from tests import helpers


def test_free_fall_discrete_closed_form():
    sc = helpers.ball_far(scenes.config(1), pos=(0.0, 5.0, 3.0))
    m = oracle.Model(sc.to_blob())
    b = 2 * sc.n_a
    x = sc.x0.copy()
    v0 = 0.7
    x[sc.nq + b + 2] = v0
    x[sc.nq + b + 0] = -0.2
    z0, dt, g = x[b + 2], sc.dt, -9.81
    for n in range(1, 51):
        x, info = m.step(x, np.zeros(sc.nu))
        assert info.ncon == 0
        zn = z0 + v0 * n * dt + g * dt * dt * n * (n + 1) / 2
        assert x[b + 2] == pytest.approx(zn, abs=1e-12)
        assert x[sc.nq + b + 2] == pytest.approx(v0 + n * g * dt, abs=1e-12)
    # horizontal motion is uniform
    assert x[b + 0] == pytest.approx(0.0 + (-0.2) * 50 * dt, abs=1e-12)


def test_pendulum_period():
    sc = helpers.planar_single_link(length=0.3, radius=0.01, mass=1.0, dt=1e-3)
    m = oracle.Model(sc.to_blob())
    x = sc.x0.copy()
    amp = 0.02
    x[0] = x[1] = math.pi / 2 + amp    # hanging straight down is q = pi/2
    ln = sc.links[0][0]
    lc = 0.15
    I_pivot = ln.inertia[1, 1] + ln.mass * lc ** 2    # transverse moment
    T = 2 * math.pi * math.sqrt(I_pivot / (ln.mass * 9.81 * lc))
    prev = x[0] - math.pi / 2
    crossings = []
    t = 0.0
    for n in range(int(3.2 * T / sc.dt)):
        x, _ = m.step(x, np.zeros(sc.nu))
        t += sc.dt
        cur = x[0] - math.pi / 2
        if prev > 0 >= cur:
            crossings.append(t - sc.dt * cur / (cur - prev))
        prev = cur
        assert x[1] == x[0]   # mirrored arms behave identically
    period = np.diff(crossings).mean()
    assert period == pytest.approx(T, rel=5e-3)


def _arm_energy(m, sc, x):
    nq = sc.nq
    q, qd = x[:nq], x[nq:]
    M = m.mass_matrix(q)
    na2 = 2 * sc.n_a
    ke = 0.5 * qd[:na2] @ M[:na2, :na2] @ qd[:na2]
    f = m.fk(q)
    pe = sum(ln.mass * 9.81 * f["c"][a, i][2] for a in range(2) for i, ln in enumerate(sc.links[a]))
    return ke + pe


def _energy_error(dt, t_end=0.25):
    sc = helpers.ball_far(helpers.torque_mode(scenes.config(1)))
    sc.dt = dt
    m = oracle.Model(sc.to_blob())
    x = sc.x0.copy()
    x[:3] = (0.3, -0.5, 0.8)
    x[3:6] = (-0.2, 0.6, -0.4)
    E0 = _arm_energy(m, sc, x)
    for _ in range(int(round(t_end / dt))):
        x, _ = m.step(x, np.zeros(sc.nu))
    return _arm_energy(m, sc, x) - E0


def test_energy_error_vanishes_at_first_order():
    """Contacts off, no damping, no actuation.  Semi-implicit Euler is not
    symplectic when M depends on q, so energy is not conserved exactly at
    finite dt; the error must halve with dt (first order) and extrapolate
    to zero.  A wrong bias or mass term leaves an O(1) residual."""
    e1 = _energy_error(2e-4)
    e2 = _energy_error(1e-4)
    assert e1 / e2 == pytest.approx(2.0, rel=0.02)
    assert abs(2 * e2 - e1) < 0.02 * abs(e1)
    assert abs(e2) < 3e-3 * (1.0 * 9.81 * 0.3)


def test_resting_ball_soft_contact():
    sc = scenes.config(1)
    m = oracle.Model(sc.to_blob())
    x = sc.x0.copy()
    b = 2 * sc.n_a
    delta = 9.81 * sc.dt ** 2 * (1 - sc.impedance) / (sc.impedance * sc.erp)
    assert delta == pytest.approx(5.45e-4, rel=1e-3)
    assert sc.ball_r - x[b + 2] == pytest.approx(delta, rel=1e-12)
    for _ in range(20):
        x, info, lam, cons = m.step(x, np.zeros(sc.nu), want_contacts=True)
        assert info.ncon == 1 and cons[0]["bodyA"] == b and cons[0]["bodyB"] == -1
        assert lam[0] == pytest.approx(sc.ball_m * 9.81 * sc.dt, rel=1e-10)
        assert abs(lam[1]) < 1e-15 and abs(lam[2]) < 1e-15
        assert np.abs(x[sc.nq + b:sc.nq + b + 6]).max() < 1e-13
    assert sc.ball_r - x[b + 2] == pytest.approx(delta, rel=1e-9)


def test_ball_settles_to_resting_depth_from_above():
    sc = scenes.config(1)
    m = oracle.Model(sc.to_blob())
    x = sc.x0.copy()
    b = 2 * sc.n_a
    x[b + 2] = sc.ball_r + 0.002
    for _ in range(400):
        x, info = m.step(x, np.zeros(sc.nu))
    delta = 9.81 * sc.dt ** 2 * (1 - sc.impedance) / (sc.impedance * sc.erp)
    assert sc.ball_r - x[b + 2] == pytest.approx(delta, rel=1e-3)


def test_sliding_ball_starts_rolling_at_five_sevenths():
    sc = helpers.ball_far(scenes.config(1), pos=(0.0, 3.0, 0.1))
    sc.dt = 1e-3
    sc.mu = 0.2
    m = oracle.Model(sc.to_blob())
    b = 2 * sc.n_a
    x = sc.x0.copy()
    delta = 9.81 * sc.dt ** 2 * (1 - sc.impedance) / (sc.impedance * sc.erp)
    x[b + 2] = sc.ball_r - delta
    v0 = 1.0
    x[sc.nq + b] = v0
    t_roll = 2 * v0 / (7 * sc.mu * 9.81)
    t = 0.0
    slip_t = None
    vx_hist = []
    for _ in range(int(2 * t_roll / sc.dt)):
        x, _ = m.step(x, np.zeros(sc.nu))
        t += sc.dt
        vx = x[sc.nq + b]
        wy = x[sc.nq + b + 4]
        vx_hist.append(vx)
        if slip_t is None and vx - sc.ball_r * wy < 1e-3 * v0:
            slip_t = t
    assert slip_t == pytest.approx(t_roll, rel=0.03)
    assert vx_hist[-1] == pytest.approx(5 / 7 * v0, rel=0.02)


def test_velocity_servo_settles_at_commanded_rate():
    # one gravity-compensated link per arm: M qdd = clamp(gear u) - D qd
    sc = helpers.planar_single_link(length=0.3, radius=0.04, dt=0.01)
    for arm in sc.links:
        arm[0].gear, arm[0].kv, arm[0].gravcomp, arm[0].damping, arm[0].tau_max = 10.0, 10.0, 1.0, 0.1, 10.0
    m = oracle.Model(sc.to_blob())
    x = sc.x0.copy()
    ln = sc.links[0][0]
    for u0, expect in ((0.4, ln.gear * 0.4 / (ln.kv + ln.damping)),
                       (50.0, ln.tau_max / (ln.kv + ln.damping))):   # saturated drive
        u = np.array([u0, -u0])
        for _ in range(300):
            x, _ = m.step(x, u)
        assert x[sc.nq + 0] == pytest.approx(expect, rel=1e-9)
        assert x[sc.nq + 1] == pytest.approx(-expect, rel=1e-9)


def _sweep_pair(sc):
    one, four = copy.deepcopy(sc), copy.deepcopy(sc)
    one.sweeps, four.sweeps = 1, 4
    return oracle.Model(one.to_blob()), oracle.Model(four.to_blob())


def _first_box_at(sc, c, h):
    sc = copy.deepcopy(sc)
    bc, bh = np.array(sc.boxes_c), np.array(sc.boxes_h)
    bc[0], bh[0] = c, h
    sc.boxes_c, sc.boxes_h = bc, bh
    return sc


def test_lone_ball_contact_is_solved_by_one_sweep():
    """A lone contact of the ball with the floor or a box has its point on
    the normal through the ball's centre, so its Delassus block is diagonal
    and projected Gauss-Seidel stops moving after the first sweep: one sweep
    and four give the same step (the reading behind the rollout's one-sweep
    solve of this case).  Two coupled contacts (the ball pressed into the
    floor and a box side) do depend on the sweep count."""
    rng = np.random.default_rng(11)
    worst = 0.0
    # the floor, the ball sliding and spinning in any direction
    sc = helpers.ball_far(scenes.config(1), pos=(0.0, 3.0, 0.1))
    m1, m4 = _sweep_pair(sc)
    b = 2 * sc.n_a
    for _ in range(20):
        x = sc.x0.copy()
        x[b + 2] = sc.ball_r - 1e-3 * rng.uniform()
        x[sc.nq + b:sc.nq + b + 6] = rng.normal(size=6)
        x1, i1, _, c1 = m1.step(x, np.zeros(sc.nu), want_contacts=True)
        x4, _ = m4.step(x, np.zeros(sc.nu))
        assert i1.ncon == 1 and c1[0]["bodyB"] == -1 and c1[0]["box"] == -1
        worst = max(worst, np.abs(x1 - x4).max())
    # a box face from outside, and the centre inside the box
    base = helpers.ball_far(scenes.config(3), pos=(0.0, 3.0, 1.0))
    b, r = 2 * base.n_a, base.ball_r
    c, h = np.array((0.0, 3.0, 1.0)), np.array((0.1, 0.08, 0.12))
    sc = _first_box_at(base, c, h)
    m1, m4 = _sweep_pair(sc)
    for t in range(30):
        x = sc.x0.copy()
        off = rng.uniform(-0.5, 0.5, size=3) * h
        if t % 5 != 4:
            ax = t % 3
            off[ax] = (1 if t % 2 == 0 else -1) * (h[ax] + r - 1e-3 * rng.uniform())
        x[b:b + 3] = c + off
        x[sc.nq + b:sc.nq + b + 6] = rng.normal(size=6)
        x1, i1, _, c1 = m1.step(x, np.zeros(sc.nu), want_contacts=True)
        x4, _ = m4.step(x, np.zeros(sc.nu))
        assert i1.ncon == 1 and c1[0]["bodyB"] == -1 and c1[0]["box"] == 0
        worst = max(worst, np.abs(x1 - x4).max())
    assert worst < 1e-12, worst
    # control: floor and a box side together
    sc = _first_box_at(base, (0.0, 3.0, h[2] + 0.05), h)
    m1, m4 = _sweep_pair(sc)
    gap = 0.0
    for _ in range(5):
        x = sc.x0.copy()
        x[b:b + 3] = (h[0] + r - 1e-3, 3.0, r - 1e-3)
        v = rng.normal(size=6)
        v[0], v[2] = -abs(v[0]) - 0.5, -abs(v[2]) - 0.5
        x[sc.nq + b:sc.nq + b + 6] = v
        x1, i1 = m1.step(x, np.zeros(sc.nu))
        x4, _ = m4.step(x, np.zeros(sc.nu))
        assert i1.ncon == 2
        gap = max(gap, np.abs(x1 - x4).max())
    assert gap > 1e-2, gap
