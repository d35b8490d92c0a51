"""Pins for the oracle's kinematics, mass matrix and bias forces.

M and c are computed in the oracle from their Jacobian definitions; these
tests check them against quantities fixed independently: closed-form
kinematics, the Lagrangian identity by finite differences, the skew
property, a textbook recursive Newton-Euler route, and numerical
quadrature of the link inertia."""
import copy
import math

import numpy as np
import pytest

import oracle
from paper_2511_21264_gb300 import scenes
from tests import helpers


def _scenes():
    return [helpers.torque_mode(scenes.config(1)), helpers.torque_mode(scenes.config(2)),
            helpers.torque_mode(scenes.config(3), gravcomp=0.0)]


def _rand_q(sc, rng):
    q = sc.x0[:sc.nq].copy()
    q[:2 * sc.n_a] = rng.uniform(-np.pi, np.pi, 2 * sc.n_a)
    return q


def test_planar_fk_closed_form():
    sc = scenes.config(1)
    m = oracle.Model(sc.to_blob())
    rng = np.random.default_rng(3)
    for _ in range(5):
        q = _rand_q(sc, rng)
        f = m.fk(q)
        for a, sx in ((0, 1.0), (1, -1.0)):
            base = sc.base_p[a]
            phi = np.cumsum(q[3 * a:3 * a + 3])
            # link vectors in the x-z plane: (cos, -sin) for the left arm,
            # mirrored in x for the right arm
            pts = base + np.cumsum(0.3 * np.stack([sx * np.cos(phi), 0 * phi, -np.sin(phi)], 1), 0)
            np.testing.assert_allclose(f["a1"][a], pts, atol=1e-14)
            np.testing.assert_allclose(f["a0"][a][1:], pts[:-1], atol=1e-14)
            np.testing.assert_allclose(f["z"][a], np.tile([0.0, sx, 0.0], (3, 1)), atol=1e-15)


def test_planar_home_touches_ball_side():
    sc = scenes.config(1)
    f = oracle.Model(sc.to_blob()).fk(sc.x0[:sc.nq])
    ball = sc.x0[6:9]
    for a in range(2):
        ee = f["a1"][a, -1]
        gap = np.linalg.norm(ee - ball) - sc.ball_r
        assert abs(gap - 0.05) < 1e-3
        assert abs(ee[2] - ball[2]) < 1e-3


def test_dh_straight_home_closed_form():
    sc = scenes.config(2)
    f = oracle.Model(sc.to_blob()).fk(sc.x0[:sc.nq])
    t = scenes.DH_HOME_TILT
    for a, sx in ((0, 1.0), (1, -1.0)):
        L = np.array([ln.F_p[0] for ln in sc.links[a]])
        d = np.array([sx * math.sin(t), 0.0, math.cos(t)])
        np.testing.assert_allclose(f["a1"][a], sc.base_p[a] + np.cumsum(L)[:, None] * d, atol=1e-13)


def test_link_inertia_against_quadrature():
    # capsule of length 0.3, radius 0.05, mass 1: integrate on a grid
    L, r, m = 0.3, 0.05, 1.0
    ln = scenes.dh_link(L, 0.0, 0.0, 0.0, m, r)
    n = 240
    xs = np.linspace(-L / 2 - r, L / 2 + r, n)
    ys = np.linspace(-r, r, n // 3)
    X, Y, Z = np.meshgrid(xs, ys, ys, indexing="ij")
    ax = np.clip(X, -L / 2, L / 2)
    inside = (X - ax) ** 2 + Y ** 2 + Z ** 2 <= r * r
    w = inside.astype(float)
    w *= m / w.sum()
    Ixx = np.sum(w * (Y ** 2 + Z ** 2))
    Iyy = np.sum(w * (X ** 2 + Z ** 2))
    assert ln.inertia[0, 0] == pytest.approx(Ixx, rel=2e-2)
    assert ln.inertia[1, 1] == pytest.approx(Iyy, rel=2e-2)
    assert ln.inertia[2, 2] == pytest.approx(Iyy, rel=2e-2)


@pytest.mark.parametrize("si", [0, 1, 2])
def test_mass_matrix_symmetric_positive_definite(si):
    sc = _scenes()[si]
    m = oracle.Model(sc.to_blob())
    rng = np.random.default_rng(si)
    for _ in range(10):
        M = m.mass_matrix(_rand_q(sc, rng))
        assert np.abs(M - M.T).max() < 1e-13
        assert np.linalg.eigvalsh(M).min() > 0


@pytest.mark.parametrize("si", [0, 1, 2])
def test_mass_and_bias_against_recursive_newton_euler(si):
    sc = _scenes()[si]
    m = oracle.Model(sc.to_blob())
    rng = np.random.default_rng(10 + si)
    nv = sc.nv
    for _ in range(5):
        q = _rand_q(sc, rng)
        qd = rng.normal(size=nv)
        qdd = rng.normal(size=nv)
        M = m.mass_matrix(q)
        c = m.bias(q, qd)
        np.testing.assert_allclose(m.rnea(q, qd, qdd), M @ qdd + c, atol=1e-11)


def _potential(m, sc, q):
    f = m.fk(q)
    V = 0.0
    g = np.asarray(sc.gravity)
    for a in range(2):
        for i, ln in enumerate(sc.links[a]):
            V -= (1.0 - ln.gravcomp) * ln.mass * g @ f["c"][a, i]
    return V


@pytest.mark.parametrize("si", [0, 1])
def test_bias_lagrangian_identity(si):
    """c = dM/dt qd - 1/2 d/dq (qd^T M qd) + dV/dq, central differences."""
    sc = _scenes()[si]
    m = oracle.Model(sc.to_blob())
    rng = np.random.default_rng(20 + si)
    na2 = 2 * sc.n_a
    h = 1e-6
    for _ in range(3):
        q = _rand_q(sc, rng)
        qd = np.zeros(sc.nv)
        qd[:na2] = rng.normal(size=na2)
        c = m.bias(q, qd)
        Mdot = np.zeros((sc.nv, sc.nv))
        dT = np.zeros(na2)
        dV = np.zeros(na2)
        for k in range(na2):
            e = np.zeros(sc.nq)
            e[k] = h
            Mp, Mm = m.mass_matrix(q + e), m.mass_matrix(q - e)
            Mdot += (Mp - Mm) / (2 * h) * qd[k]
            dT[k] = 0.5 * (qd @ Mp @ qd - qd @ Mm @ qd) / (2 * h)
            dV[k] = (_potential(m, sc, q + e) - _potential(m, sc, q - e)) / (2 * h)
        lag = (Mdot @ qd)[:na2] - dT + dV
        np.testing.assert_allclose(c[:na2], lag, atol=2e-7 * max(1.0, np.abs(lag).max()))


@pytest.mark.parametrize("si", [0, 1])
def test_skew_property(si):
    """qd^T (dM/dt - 2C) qd = 0 with C qd = c(q, qd) - c(q, 0)."""
    sc = _scenes()[si]
    m = oracle.Model(sc.to_blob())
    rng = np.random.default_rng(30 + si)
    h = 1e-6
    for _ in range(3):
        q = _rand_q(sc, rng)
        qd = rng.normal(size=sc.nv)
        qd[2 * sc.n_a:] = 0.0
        qdot_q = np.zeros(sc.nq)
        qdot_q[:2 * sc.n_a] = qd[:2 * sc.n_a]
        Mdot = (m.mass_matrix(q + h * qdot_q) - m.mass_matrix(q - h * qdot_q)) / (2 * h)
        Cqd = m.bias(q, qd) - m.bias(q, np.zeros(sc.nv))
        assert abs(qd @ Mdot @ qd - 2 * qd @ Cqd) < 1e-6 * max(1.0, abs(qd @ Mdot @ qd))


def test_gravity_compensation_removes_link_gravity():
    sc = scenes.config(2)
    m = oracle.Model(sc.to_blob())
    q = _rand_q(sc, np.random.default_rng(4))
    c = m.bias(q, np.zeros(sc.nv))
    assert np.abs(c[:14]).max() < 1e-14
    np.testing.assert_allclose(c[14:17], [0, 0, sc.ball_m * 9.81], atol=1e-14)


def test_ball_block_is_diagonal():
    sc = scenes.config(1)
    M = oracle.Model(sc.to_blob()).mass_matrix(sc.x0[:sc.nq])
    b = 2 * sc.n_a
    np.testing.assert_allclose(M[b:, b:], np.diag([sc.ball_m] * 3 + [sc.ball_I] * 3), atol=0)
    assert np.all(M[:b, b:] == 0) and np.all(M[0:3, 3:6] == 0)
