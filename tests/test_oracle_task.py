"""Pins of the oracle's ball-task cost suite (Sec. IV-B): the features it
reads off a state (capsule-capsule distances, end-effector orientation and
velocity, the collision pairs) and the cost terms, each against something
other than the oracle's own formula -- brute force, closed forms of
constructed inputs, finite differences, invariants of the barrier."""
import math

import numpy as np
import pytest

import oracle
from paper_2511_21264_gb300 import scenes


def _rodrigues(axis, ang):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def _quat_to_rot(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


# ----------------------------------------------------------------- features
def test_capsule_capsule_against_brute_force():
    rng = np.random.default_rng(0)
    g = np.linspace(0.0, 1.0, 401)
    for trial in range(40):
        a0, a1, b0, b1 = rng.normal(scale=0.3, size=(4, 3))
        if trial % 5 == 0:
            b1 = b0 + (a1 - a0) * rng.uniform(0.3, 2.0)  # parallel
        if trial % 7 == 0:
            a1 = a0.copy()                               # a point
        ra, rb = rng.uniform(0.0, 0.05, 2)
        P = a0[None, :] + g[:, None] * (a1 - a0)[None, :]
        Q = b0[None, :] + g[:, None] * (b1 - b0)[None, :]
        brute = np.sqrt(((P[:, None, :] - Q[None, :, :]) ** 2).sum(-1)).min() - ra - rb
        d = oracle.capsule_capsule(a0, a1, ra, b0, b1, rb)
        lip = (np.linalg.norm(a1 - a0) + np.linalg.norm(b1 - b0)) * 0.5 * (g[1] - g[0])
        assert d <= brute + 1e-12
        assert brute - d <= lip + 1e-12


def test_capsule_capsule_special_cases():
    # crossing segments touch: distance = - radii
    d = oracle.capsule_capsule([-1, 0, 0], [1, 0, 0], 0.1, [0, -1, 0], [0, 1, 0], 0.05)
    assert d == pytest.approx(-0.15, abs=1e-15)
    # parallel, overlapping in x, 0.3 apart in z
    d = oracle.capsule_capsule([0, 0, 0], [1, 0, 0], 0.0, [0.5, 0, 0.3], [2, 0, 0.3], 0.0)
    assert d == pytest.approx(0.3, abs=1e-15)
    # collinear and disjoint: end to end
    d = oracle.capsule_capsule([0, 0, 0], [1, 0, 0], 0.0, [1.5, 0, 0], [3, 0, 0], 0.0)
    assert d == pytest.approx(0.5, abs=1e-15)
    # skew lines, closest points interior: x axis and the line y = 1 along z
    d = oracle.capsule_capsule([-1, 0, 0], [1, 0, 0], 0.0, [0, 1, -1], [0, 1, 1], 0.0)
    assert d == pytest.approx(1.0, abs=1e-15)


@pytest.mark.parametrize("ang", [0.0, 0.3, 1.5, 2.9, math.pi - 1e-9, math.pi])
def test_rotation_to_quaternion(ang):
    rng = np.random.default_rng(int(ang * 1000))
    for _ in range(5):
        axis = rng.normal(size=3)
        R = _rodrigues(axis, ang)
        q = oracle.rot_to_quat(R)
        assert np.linalg.norm(q) == pytest.approx(1.0, abs=1e-12)
        a = axis / np.linalg.norm(axis)
        expect = np.concatenate([[math.cos(ang / 2)], a * math.sin(ang / 2)])
        assert abs(np.dot(q, expect)) == pytest.approx(1.0, abs=1e-9)
        np.testing.assert_allclose(_quat_to_rot(q), R, atol=1e-12)


def test_end_effector_velocity_is_the_time_derivative_of_its_position():
    for cfg in (1, 2):
        sc = scenes.config(cfg)
        om = oracle.Model(sc.to_blob())
        x = scenes.random_states(sc, 3, 5)[1]
        nq = om.nq
        qd = x[nq:nq + sc.nu]
        h = 1e-6
        xp, xm = x.copy(), x.copy()
        xp[:sc.nu] += h * qd
        xm[:sc.nu] -= h * qd
        fd = (om.ee_state(xp)["p"] - om.ee_state(xm)["p"]) / (2 * h)
        np.testing.assert_allclose(om.ee_state(x)["v"], fd, atol=1e-7)


def test_planar_end_effector_orientation_turns_by_the_joint_angle_sum():
    # all joint axes of the planar arms are parallel (world y): the last
    # frame's rotation between two poses is the sum of the joint changes
    sc = scenes.config(1)
    om = oracle.Model(sc.to_blob())
    rng = np.random.default_rng(2)
    for _ in range(10):
        x = sc.x0.copy()
        x2 = x.copy()
        dq = rng.uniform(-0.5, 0.5, sc.nu)
        x2[:sc.nu] += dq
        qa, qb = om.ee_state(x)["quat"], om.ee_state(x2)["quat"]
        for a in range(2):
            ang = 2 * math.acos(min(1.0, abs(np.dot(qa[a], qb[a]))))
            assert ang == pytest.approx(abs(dq[3 * a:3 * a + 3].sum()), abs=1e-9)


def test_end_effector_position_is_the_distal_capsule_end_planar_closed_form():
    sc = scenes.config(1)
    om = oracle.Model(sc.to_blob())
    x = sc.x0.copy()
    p = om.ee_state(x)["p"]
    # planar arms: base + sum of link vectors at absolute angles in the x-z plane
    fk = om.fk(x[:om.nq])
    for a in range(2):
        np.testing.assert_allclose(p[a], fk["a1"][a][sc.n_a - 1], atol=1e-15)
    assert p[0][1] == pytest.approx(0.0, abs=1e-12) and p[1][1] == pytest.approx(0.0, abs=1e-12)


def test_pair_set_by_phase():
    sc = scenes.config(3)
    om = oracle.Model(sc.to_blob())
    na, nb = sc.n_a, sc.n_boxes
    x = sc.x0
    d_pick = om.pair_distances(x, 0)
    d_move = om.pair_distances(x, 1)
    assert len(d_pick) == 2 * na * nb + 2 * na + na * na
    assert len(d_move) == 2 * na * nb + na * na
    # move drops exactly the ball-link block
    np.testing.assert_array_equal(d_move[:2 * na * nb], d_pick[:2 * na * nb])
    np.testing.assert_array_equal(d_move[2 * na * nb:], d_pick[2 * na * nb + 2 * na:])
    # ball-link entries: the ball centre's distance to the link segment minus both radii
    fk = om.fk(x[:om.nq])
    c = x[2 * na:2 * na + 3]
    g = np.linspace(0, 1, 20001)
    for a in range(2):
        for i in range(na):
            seg = fk["a0"][a][i][None] + g[:, None] * (fk["a1"][a][i] - fk["a0"][a][i])[None]
            brute = np.sqrt(((seg - c) ** 2).sum(1)).min() - sc.ball_r - sc.links[a][i].radius
            assert d_pick[2 * na * nb + a * na + i] == pytest.approx(brute, abs=1e-7)


# ------------------------------------------------------------------- terms
def _features(H, B, nu):
    return np.zeros((H + 1, B)), np.zeros((H + 1, nu)), np.zeros((H + 1, 20))


def _task(nu, **kw):
    t = np.zeros(oracle.TASK_N + nu)
    t[2] = 0.2  # gamma
    t[18] = t[22] = 1.0  # identity target orientations
    for k, v in kw.items():
        t[{"phase": 0, "w_c": 1, "gamma": 2, "w_theta": 3, "w_yz": 4, "w_v": 5, "w_r": 6, "w_l": 7, "l_ball": 8,
           "w_eo": 9, "w_ot": 10, "eps": 11}[k]] = v
    return t


def _set_ee(EE, k, p1, p2, v1=(0, 0, 0), v2=(0, 0, 0), q1=(1, 0, 0, 0), q2=(1, 0, 0, 0)):
    EE[k] = np.concatenate([p1, p2, v1, v2, q1, q2])


def test_barrier_is_zero_on_its_boundary_and_grows_past_it():
    # d_{k+1} = (1 - gamma) d_k is the fastest approach the barrier allows
    H, B, nu, gam = 10, 3, 2, 0.2
    D, TH, EE = _features(H, B, nu)
    for k in range(H + 1):
        _set_ee(EE, k, [0, 0, 0], [0, 0, 0])
        D[k] = np.array([0.5, 1.0, 2.0]) * (1 - gam) ** k
    t = _task(nu, w_c=1.0, gamma=gam)
    c, terms = oracle.task_cost_features(t, D, TH, EE)
    assert terms[0] == pytest.approx(0.0, abs=1e-15)
    # a pair standing still costs nothing; one closing faster than the barrier costs
    D2 = D.copy()
    D2[:, 0] = 0.5
    D2[:, 1] = 1.0 * (0.5 ** np.arange(H + 1))
    c2, terms2 = oracle.task_cost_features(t, D2, TH, EE)
    expect = sum(max(-D2[k + 1, 1] + (1 - gam) * D2[k, 1], 0.0) for k in range(H))
    assert terms2[0] == pytest.approx(expect, rel=1e-14)
    assert expect == pytest.approx(sum(1.0 * 0.5 ** k * (0.5 - gam) for k in range(H)), rel=1e-14)


def test_penetration_indicator_counts_states_after_the_controls():
    H, B, nu = 4, 2, 2
    D, TH, EE = _features(H, B, nu)
    D[:] = 1.0
    D[0, 0] = -0.1          # the present state does not count
    D[2, 1] = -0.01         # one penetrating state ...
    D[3, 1] = -0.01         # ... and another
    t = _task(nu, w_c=1.0, gamma=0.0)
    # gamma = 0: the barrier is the total decrease of each distance
    _, terms = oracle.task_cost_features(t, D, TH, EE)
    assert terms[0] == pytest.approx(2 + 1.01, abs=1e-15)


def test_end_effector_terms_on_constructed_poses():
    H, B, nu = 5, 1, 2
    D, TH, EE = _features(H, B, nu)
    D[:] = 1.0
    rng = np.random.default_rng(0)
    lb, eps = 0.2, 0.03
    pb0, ptg = np.array([0.1, 0.2, 0.3]), np.array([-0.4, 0.5, 0.6])
    exp = dict(yz=0.0, v2=0.0, l=0.0, eo=0.0, ot=0.0, r=0.0)
    for k in range(H + 1):
        c = rng.normal(scale=0.3, size=3)
        half = rng.normal(scale=0.1, size=3)
        p1, p2 = c + half, c - half
        rel = p1 - p2
        perp = np.cross(rel, rng.normal(size=3))
        vpar = 0.7 * rel / np.linalg.norm(rel)
        ang = rng.uniform(0, 2.5)
        q1 = np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * np.array([0, 0, 1.0])])
        _set_ee(EE, k, p1, p2, v1=perp + vpar, v2=0 * perp, q1=q1, q2=(1, 0, 0, 0))
        if k >= 1:
            exp["yz"] += math.hypot(rel[1], rel[2])
            exp["v2"] += (np.linalg.norm(rel) * 0.7) ** 2    # only the parallel part counts
            exp["l"] += (np.linalg.norm(rel) - lb) ** 2
            exp["eo"] += np.linalg.norm(c - (pb0 - [0, 0, eps]))
            exp["ot"] += np.linalg.norm(c + [0, 0, eps] - ptg)
            exp["r"] += 0.5 * ang
    t = _task(nu, l_ball=lb, eps=eps)
    t[12:15], t[15:18] = pb0, ptg
    _, terms = oracle.task_cost_features(t, D, TH, EE)
    np.testing.assert_allclose(terms[2:], [exp["yz"], math.sqrt(exp["v2"]), exp["r"], exp["l"], exp["eo"], exp["ot"]],
                               rtol=1e-12)


def test_joint_deviation_and_phase_weights():
    H, B, nu = 3, 1, 4
    D, TH, EE = _features(H, B, nu)
    D[:] = 1.0
    D[1:, 0] = -1.0  # 3 penetrating states, no barrier decrease after k = 1
    home = np.array([0.1, -0.2, 0.3, 0.0])
    TH[:] = home
    TH[2] += [0.0, 0.3, 0.0, 0.4]  # |.| = 0.5 at one state
    for k in range(H + 1):
        _set_ee(EE, k, [0, 0, 0], [0, 0, 0])
    base = dict(w_c=2.0, w_theta=3.0, w_eo=5.0, w_ot=7.0, eps=0.0)
    tp = _task(nu, phase=0, **base)
    tm = _task(nu, phase=1, **base)
    for t in (tp, tm):
        t[oracle.TASK_N:] = home
        t[12:15] = [1.0, 0, 0]   # |c - p_ball0| = 1 at every state
        t[15:18] = [0, 2.0, 0]   # |c - p_target| = 2 at every state
    cp, terms = oracle.task_cost_features(tp, D, TH, EE)
    cm, _ = oracle.task_cost_features(tm, D, TH, EE)
    assert terms[1] == pytest.approx(0.5, abs=1e-15)
    Cc = terms[0]
    # 3 indicators; the drop 1 -> -1 costs 1 + 0.8; a distance held at -1
    # keeps costing gamma |d| = 0.2 per step (the barrier pushes out of contact)
    assert Cc == pytest.approx(3 + (1 + 0.8) + 2 * 0.2, abs=1e-12)
    assert cp == pytest.approx(2.0 * Cc + 5.0 * 3 * 1.0 + 3.0 * 0.5, rel=1e-13)
    assert cm == pytest.approx(2.0 * Cc + 7.0 * 3 * 2.0 + 3.0 * 0.5, rel=1e-13)


def test_trajectory_cost_composes_the_features_of_each_state():
    sc = scenes.config(3)
    om = oracle.Model(sc.to_blob())
    task = scenes.ball_task(sc, phase=0)
    rng = np.random.default_rng(4)
    U = 0.2 * rng.normal(size=(6, sc.nu))
    c, terms, traj = om.rollout_task(sc.x0, U, task)
    assert np.isfinite(c) and np.all(np.isfinite(terms))
    D = np.stack([om.pair_distances(x, 0) for x in traj])
    TH = traj[:, :sc.nu]
    EE = np.stack([np.concatenate([(e := om.ee_state(x))["p"].ravel(), e["v"].ravel(), e["quat"].ravel()])
                   for x in traj])
    c2, terms2 = oracle.task_cost_features(task, D, TH, EE)
    assert c2 == pytest.approx(c, rel=1e-14)
    np.testing.assert_allclose(terms2, terms, rtol=1e-14)
    c3, _ = om.task_cost(task, traj)
    assert c3 == pytest.approx(c, rel=1e-14)
