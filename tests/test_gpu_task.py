"""The ball-task cost suite (Sec. IV-B) inside the GPU rollout against the
FP64 oracle, through the C ABI.

Tolerance: per-sample cost |c_gpu - c_oracle| <= 1e-3 |c_oracle| + 1e-3
(the existing bound for 8-step rollout costs).  The suite's non-smooth
parts are kept away from their kinks: parity states keep every collision
pair's distance at least 1e-4 from zero along the oracle's trajectory (the
penetration count is a step function of it), and the target orientations
are 90 degrees from the end effectors' (acos is steep near 1)."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2511_21264_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"


@pytest.fixture(scope="module")
def native():
    from paper_2511_21264_gb300 import native as nat
    nat.build()
    nat.lib()
    return nat


def _t(a):
    return torch.tensor(np.ascontiguousarray(np.asarray(a, np.float32)), device=DEV)


def _f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def _cases(sc, om, task, n, H, seed, **spread):
    """States and controls whose oracle trajectories keep every pair
    distance at least 1e-4 from zero."""
    rng = np.random.default_rng(seed)
    X, U, ref = [], [], []
    s = seed
    while len(X) < n:
        for x in _f32(scenes.random_states(sc, 2 * n, s, **spread)):
            u = _f32(0.3 * rng.normal(size=(H, sc.nu)))
            c, terms, traj = om.rollout_task(x, u, task)
            if not np.isfinite(c):
                continue
            dmin = min(np.abs(om.pair_distances(xk, int(task[0]))).min() for xk in traj)
            if dmin < 1e-4 or min(om.min_abs_dist(xk) for xk in traj[:-1]) < 1e-5:
                continue
            X.append(x)
            U.append(u)
            ref.append(c)
            if len(X) == n:
                break
        s += 1000
    return np.array(X), np.array(U), np.array(ref)


@pytest.mark.parametrize("cfg,phase", [(1, 0), (2, 0), (2, 1), (3, 0), (3, 1)])
def test_rollout_task_cost_matches_oracle(native, cfg, phase):
    K, H = 48, 8
    sc = scenes.config(cfg)
    blob = sc.to_blob()
    gm, om = native.Model(blob), oracle.Model(blob)
    task = _f32(scenes.ball_task(sc, phase=phase))
    ctl = native.Controller(gm, K, H, sc.lam, sc.sigma_vec(), 3)
    ctl.set_task_cost(task)
    X, U, ref = _cases(sc, om, task, K, H, 100 + cfg)
    costs = torch.empty(K, device=DEV)
    ctl.rollout_batch(_t(X), _t(U), costs)
    assert ctl.sync() == 0
    c = costs.cpu().numpy().astype(np.float64)
    err = np.abs(c - ref) - (1e-3 * np.abs(ref) + 1e-3)
    assert err.max() <= 0.0, (err.argmax(), c[err.argmax()], ref[err.argmax()])
    # off again: the scene's own stage cost
    ctl.set_task_cost(None)
    ctl.rollout_batch(_t(X), _t(U), costs)
    assert ctl.sync() == 0
    plain = np.array([om.rollout(x, u) for x, u in zip(X, U)])
    np.testing.assert_allclose(costs.cpu().numpy(), plain, rtol=1e-3, atol=1e-3)


def test_mppi_step_with_task_cost_matches_oracle(native):
    K, H = 64, 8
    sc = scenes.config(1)
    blob = sc.to_blob()
    gm, om = native.Model(blob), oracle.Model(blob)
    task = _f32(scenes.ball_task(sc, phase=0))
    key = scenes.controller_key(1, 7)
    ctl = native.Controller(gm, K, H, sc.lam, sc.sigma_vec(), key)
    ctl.set_task_cost(task)
    x = _f32(sc.x0)
    u0 = np.zeros((H, sc.nu))
    out = torch.empty((H, sc.nu), device=DEV)
    ctl.step(_t(x), _t(u0), out)
    assert ctl.sync() == 0
    U = u0[None] + oracle.noise(key, 0, K, H, sc.nu, _f32(sc.sigma_vec()))
    costs = np.array([om.rollout_task(x, U[k], task)[0] for k in range(K)])
    u_ref, _, st = oracle.mppi_update(costs, U, sc.lam, u0)
    assert st == 0
    np.testing.assert_allclose(out.cpu().numpy(), u_ref, atol=1e-3, rtol=0)


def test_task_cost_argument_errors(native):
    from paper_2511_21264_gb300.native import MPPIError
    sc = scenes.config(2)
    gm = native.Model(sc.to_blob())
    ctl = native.Controller(gm, 8, 4, sc.lam, sc.sigma_vec(), 1)
    good = scenes.ball_task(sc)
    for bad in (good[:-1], np.where(np.arange(good.size) == 0, 2.0, good),
                np.where(np.arange(good.size) == 2, 1.0, good), np.where(np.arange(good.size) == 18, 0.5, good),
                np.where(np.arange(good.size) == 5, np.nan, good)):
        with pytest.raises(MPPIError):
            ctl.set_task_cost(bad)
    ctl.set_task_cost(good)
    ctl.set_task_cost(None)


def _boxes_across_links(sc, links, half=0.04):
    """The scene with its first boxes moved onto the midpoints of the given
    (arm, link) segments at the home pose (cubes of half extent `half`)."""
    f = oracle.Model(sc.to_blob()).fk(sc.x0[:sc.nq])
    bc, bh = np.array(sc.boxes_c), np.array(sc.boxes_h)
    for j, (a, i) in enumerate(links):
        bc[j] = 0.5 * (f["a0"][a, i] + f["a1"][a, i])
        bh[j] = half
    return dataclasses.replace(sc, boxes_c=bc, boxes_h=bh)


def test_task_cost_with_link_segments_through_boxes(native):
    """Link segments that meet a box take the capsule-box distance's other
    branch (the piece walk through the box); random states rarely produce
    them.  Two of the config-3 boxes sit across links of the home pose and
    the states stay near it, so that many pairs along the trajectories have
    a segment inside a box (at least 50, counted by the oracle).  More boxes
    across links make the oracle's own rollouts fail (deep contacts)."""
    K, H = 48, 3
    sc = _boxes_across_links(scenes.config(3), [(0, 3), (1, 5)])
    blob = sc.to_blob()
    gm, om = native.Model(blob), oracle.Model(blob)
    task = _f32(scenes.ball_task(sc, phase=1))
    X, U, ref = _cases(sc, om, task, K, H, 7, q_spread=0.1, v_spread=0.1)
    na, nb = sc.n_a, sc.n_boxes
    rc = np.repeat([sc.links[a][i].radius for a in range(2) for i in range(na)], nb)
    inside = sum(int((om.pair_distances(xk, 1)[:2 * na * nb] + rc <= 0.0).sum())
                 for x, u in zip(X, U) for xk in om.rollout_task(x, u, task)[2])
    assert inside >= 50, inside
    ctl = native.Controller(gm, K, H, sc.lam, sc.sigma_vec(), 3)
    ctl.set_task_cost(task)
    costs = torch.empty(K, device=DEV)
    ctl.rollout_batch(_t(X), _t(U), costs)
    assert ctl.sync() == 0
    c = costs.cpu().numpy().astype(np.float64)
    err = np.abs(c - ref) - (1e-3 * np.abs(ref) + 1e-3)
    assert err.max() <= 0.0, (err.argmax(), c[err.argmax()], ref[err.argmax()])
