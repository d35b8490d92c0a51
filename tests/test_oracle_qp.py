"""Pins of the oracle's QP smoothing projection (Eq. 5): each check comes from
the problem statement itself (bounds on the joint trajectory and its first
three derivatives), not from the ADMM iteration the oracle runs.

- closed forms: velocity bounds alone reduce to a clamp; a position bound
  alone on a constant target gives the uniform sequence that just reaches
  it; acceleration bounds alone on a constant target give the ramp from the
  present velocity;
- a feasible sample is returned unchanged after any number of iterations;
- at convergence the result satisfies the KKT conditions of the QP, with the
  constraint rows built here from finite differences of the trajectory;
- on tiny horizons, enumeration of active sets finds the same minimiser.
"""
import itertools
import zlib

import numpy as np
import pytest

import oracle

DT = 0.01
INF = np.inf


def derivs(v, q, qd, dt=DT):
    """Position after each step, velocity, acceleration and jerk of the
    commanded sequence v, in the order the bounds list them (jerk from t=1)."""
    v = np.asarray(v, dtype=float)
    th = q + dt * np.cumsum(v)
    ext = np.concatenate([[qd], v])
    acc = np.diff(ext) / dt
    jerk = np.diff(ext, 2) / dt ** 2
    return np.concatenate([th, v, acc, jerk])


def bound_vectors(b, H):
    lo = np.concatenate([np.full(H, b[0]), np.full(H, b[2]), np.full(H, b[4]), np.full(H - 1, b[6])])
    hi = np.concatenate([np.full(H, b[1]), np.full(H, b[3]), np.full(H, b[5]), np.full(H - 1, b[7])])
    return lo, hi


def jacobian(H, q, qd):
    f0 = derivs(np.zeros(H), q, qd)
    return np.stack([derivs(np.eye(H)[i], q, qd) - f0 for i in range(H)], axis=1), f0


def kkt_residual(v, vt, b, q, qd, rtol=1e-7):
    """Largest violation of primal feasibility and of stationarity with
    non-negative multipliers on the active rows (found by NNLS)."""
    from scipy.optimize import nnls
    H = len(v)
    G, _ = jacobian(H, q, qd)
    lo, hi = bound_vectors(b, H)
    f = derivs(v, q, qd)
    scale = np.maximum(1.0, np.where(np.isfinite(hi), np.abs(hi), 0.0) + np.where(np.isfinite(lo), np.abs(lo), 0.0))
    viol = np.max(np.maximum(0.0, np.maximum(lo - f, f - hi)) / scale)
    up = f >= hi - rtol * scale
    dn = f <= lo + rtol * scale
    A = np.concatenate([G[up].T, -G[dn].T], axis=1)
    # rows are scaled to unit norm so that NNLS is well conditioned
    if A.shape[1] == 0:
        stat = np.max(np.abs(vt - v))
    else:
        nrm = np.linalg.norm(A, axis=0)
        mu, res = nnls(A / nrm, vt - v, maxiter=5000)
        stat = res
    return viol, stat


REGIMES = {
    "ur5e-like": np.array([-2.0, 2.0, -np.pi, np.pi, -10.0, 10.0, -300.0, 300.0]),
    "tight jerk": np.array([-2.0, 2.0, -np.pi, np.pi, -10.0, 10.0, -50.0, 50.0]),
    "tight position": np.array([-0.25, 0.25, -1.0, 1.0, -10.0, 10.0, -300.0, 300.0]),
    "velocity only": np.array([-INF, INF, -0.5, 0.5, -INF, INF, -INF, INF]),
}


def test_velocity_bounds_alone_reduce_to_a_clamp():
    rng = np.random.default_rng(1)
    b = REGIMES["velocity only"]
    vt = 0.6 * rng.normal(size=24)
    v, _, viol = oracle.qp_project(vt, b, 0.3, 0.2, DT, rho=1.0, iters=3000)
    np.testing.assert_allclose(v, np.clip(vt, -0.5, 0.5), atol=1e-9)
    assert viol < 1e-9


def test_position_bound_alone_gives_the_uniform_sequence_that_reaches_it():
    # min sum (v - c)^2 s.t. every prefix sum <= P: the last prefix binds and
    # the uniform v = P / H satisfies all the others
    H, c, q, th_hi = 20, 1.5, 0.1, 0.2
    b = np.array([-INF, th_hi, -INF, INF, -INF, INF, -INF, INF])
    v, _, _ = oracle.qp_project(np.full(H, c), b, q, 0.0, DT, rho=1.0, iters=4000)
    np.testing.assert_allclose(v, np.full(H, (th_hi - q) / (H * DT)), atol=1e-8)


def test_acceleration_bounds_alone_give_the_ramp_from_the_present_velocity():
    # every v_t <= qd + (t+1) a dt is implied by the bounds and the componentwise
    # minimiser min(c, qd + (t+1) a dt) is feasible, hence optimal
    H, c, qd, a = 16, 0.8, 0.1, 3.0
    b = np.array([-INF, INF, -INF, INF, -a, a, -INF, INF])
    v, _, _ = oracle.qp_project(np.full(H, c), b, 0.0, qd, DT, rho=1.0, iters=4000)
    np.testing.assert_allclose(v, np.minimum(c, qd + (np.arange(H) + 1) * a * DT), atol=1e-8)


@pytest.mark.parametrize("iters", [1, 7, 100])
def test_feasible_sample_is_a_fixed_point(iters):
    H = 32
    t = np.arange(H) * DT
    vt = 0.3 + 0.2 * np.sin(2.0 * t)        # accel <= 0.4, jerk <= 0.8
    b = REGIMES["ur5e-like"]
    v, y, viol = oracle.qp_project(vt, b, 0.0, 0.3, DT, rho=1.0, iters=iters)
    np.testing.assert_allclose(v, vt, atol=1e-12)
    assert viol == 0.0 and np.all(y == 0.0)


@pytest.mark.parametrize("regime", sorted(REGIMES))
@pytest.mark.parametrize("H", [8, 20])
def test_converged_projection_satisfies_kkt(regime, H):
    rng = np.random.default_rng(zlib.crc32(f"{regime} {H}".encode()))
    b = REGIMES[regime]
    for trial in range(3):
        vt = 0.1 + 0.4 * rng.normal(size=H)
        # a state the bounds can hold (the QP is feasible)
        q, qd = rng.uniform(-0.1, 0.1), rng.uniform(-0.3, 0.3)
        v, _, viol = oracle.qp_project(vt, b, q, qd, DT, rho=1.0, iters=30000)
        pv, stat = kkt_residual(v, vt, b, q, qd)
        assert pv < 1e-7, (regime, trial, pv)
        assert stat < 1e-6, (regime, trial, stat)
        assert np.max(np.abs(v - vt)) > 1e-3 or regime == "velocity only"


def test_kkt_check_rejects_a_planted_sign_error():
    # the same problem solved with the jerk rows' v_{-1} term dropped: the
    # check built from the trajectory's derivatives must flag it
    H = 8
    rng = np.random.default_rng(3)
    b = REGIMES["tight jerk"]
    vt = 0.4 * rng.normal(size=H)
    v_ok, _, _ = oracle.qp_project(vt, b, 0.0, 0.3, DT, iters=30000)
    v_bad, _, _ = oracle.qp_project(vt, b, 0.0, 0.0, DT, iters=30000)  # qd ignored
    assert max(kkt_residual(v_ok, vt, b, 0.0, 0.3)) < 1e-6
    assert max(kkt_residual(v_bad, vt, b, 0.0, 0.3)) > 1e-4


def brute_force(vt, b, q, qd, max_active):
    """Minimiser by enumeration of active sets (rows at a lower or upper
    bound) with equality-constrained KKT solves."""
    H = len(vt)
    G, f0 = jacobian(H, q, qd)
    lo, hi = bound_vectors(b, H)
    m = G.shape[0]
    best = None
    for na in range(max_active + 1):
        for rows in itertools.combinations(range(m), na):
            for sides in itertools.product((0, 1), repeat=na):
                tgt = np.array([hi[r] if s else lo[r] for r, s in zip(rows, sides)])
                if not np.all(np.isfinite(tgt)):
                    continue
                GA = G[list(rows)]
                K = np.block([[np.eye(H), GA.T], [GA, np.zeros((na, na))]])
                rhs = np.concatenate([vt, tgt - f0[list(rows)]])
                try:
                    sol = np.linalg.solve(K, rhs)
                except np.linalg.LinAlgError:
                    continue
                v, lam = sol[:H], sol[H:]
                f = derivs(v, q, qd)
                if np.any(f < lo - 1e-9 * np.maximum(1, np.abs(lo))) or np.any(f > hi + 1e-9 * np.maximum(1, np.abs(hi))):
                    continue
                # lam is the multiplier of G v = target in L = 1/2|v-vt|^2 + lam^T (G v - t):
                # upper bounds need lam >= 0, lower bounds lam <= 0
                sgn = np.array([1.0 if s else -1.0 for s in sides])
                if np.any(sgn * lam < -1e-9):
                    continue
                obj = 0.5 * np.sum((v - vt) ** 2)
                if best is None or obj < best[0] - 1e-12:
                    best = (obj, v)
    return best[1]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tiny_horizon_matches_active_set_enumeration(seed):
    rng = np.random.default_rng(10 + seed)
    H = 3
    b = np.array([-0.004, 0.006, -0.5, 0.5, -20.0, 20.0, -2000.0, 2000.0])
    vt = 0.6 * rng.normal(size=H)
    q, qd = 0.0, 0.1 * rng.normal()
    v_bf = brute_force(vt, b, q, qd, max_active=H)
    v, _, _ = oracle.qp_project(vt, b, q, qd, DT, rho=1.0, iters=40000)
    np.testing.assert_allclose(v, v_bf, atol=1e-8)
    assert np.max(np.abs(v - vt)) > 1e-3
