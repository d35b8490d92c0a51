"""The rows beyond the hot path at the benchmark's full sizes, on sampled
outputs the oracle computes one by one:

- the QP projection inside the 8-box transfer controller (K = 4096, H = 64:
  the one-thread-per-sequence kernel), sampled sequences against the
  oracle's projection within 2e-4 + 1e-4 |v|;
- the ball-task cost suite at the same size, sampled per-sample costs over
  8 steps within 1e-3 relative (states kept 1e-4 away from every
  penetration threshold);
- the full Eq. 8 update on the 1024-sample lift (test-drawn costs, the
  Philox samples of iteration 0): mean and covariance blocks against the
  oracle's elite update within 1e-3, the best sequence within 2e-6."""
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


def test_projection_full_size_transfer_sampled(native):
    sc = scenes.config(3)
    K, H, iters = sc.K, sc.H, 30
    gm = native.Model(sc.to_blob())
    key = scenes.controller_key(3, 2)
    ctl = native.Controller(gm, K, H, sc.lam, sc.sigma_vec(), key)
    bounds = _f32(scenes.projection_bounds(sc))
    ctl.set_projection(bounds, iters=iters)
    x = _f32(sc.x0)
    u0 = np.zeros((H, sc.nu))
    out = torch.empty((H, sc.nu), device=DEV)
    ctl.step(_t(x), _t(u0), out)
    assert ctl.sync() == 0
    S = torch.empty((H, K, sc.nu), device=DEV)
    ctl.samples(S)
    torch.cuda.synchronize()
    S = S.cpu().numpy()
    assert np.all(np.isfinite(S))
    rng = np.random.default_rng(3)
    ks = rng.choice(K, 5, replace=False)
    raw = oracle.noise(key, 0, K, H, sc.nu, _f32(sc.sigma_vec()))  # unclamped: the projection replaces the clamp
    for k in ks:
        for j in range(sc.nu):
            ref = oracle.qp_project(raw[k, :, j], bounds[j], x[j], x[sc.nq + j], sc.dt, 1.0, iters)[0]
            err = np.abs(S[:, k, j] - ref) - (2e-4 + 1e-4 * np.abs(ref))
            assert err.max() <= 0.0, (k, j, err.max())


def test_task_suite_full_size_transfer_sampled(native):
    sc = scenes.config(3)
    K, H = sc.K, 8
    blob = sc.to_blob()
    gm, om = native.Model(blob), oracle.Model(blob)
    task = _f32(scenes.ball_task(sc, phase=1))
    ctl = native.Controller(gm, K, H, sc.lam, sc.sigma_vec(), 4)
    ctl.set_task_cost(task)
    rng = np.random.default_rng(8)
    X = _f32(scenes.random_states(sc, K, 31))
    U = _f32(0.3 * rng.normal(size=(K, H, sc.nu)))
    costs = torch.empty(K, device=DEV)
    ctl.rollout_batch(_t(X), _t(U), costs)
    assert ctl.sync() == 0
    c = costs.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(c))
    checked = 0
    for k in rng.permutation(K)[:40]:
        ref, _, traj = om.rollout_task(X[k], U[k], task)
        if not np.isfinite(ref):
            continue
        if min(np.abs(om.pair_distances(xk, 1)).min() for xk in traj) < 1e-4:
            continue
        if min(om.min_abs_dist(xk) for xk in traj[:-1]) < 1e-5:
            continue
        assert abs(c[k] - ref) <= 1e-3 * abs(ref) + 1e-3, (k, c[k], ref)
        checked += 1
        if checked == 8:
            break
    assert checked >= 6


def test_elite_update_full_size_lift(native):
    sc = scenes.config(2)
    K, H = sc.K, sc.H
    gm = native.Model(sc.to_blob())
    key = 12
    ctl = native.Controller(gm, K, H, sc.lam, sc.sigma_vec(), key)
    ctl.set_update(64, 0.7, True, 1e-6)
    rng = np.random.default_rng(21)
    costs = _f32(rng.uniform(100.0, 110.0, K))
    u0 = _f32(rng.normal(scale=0.1, size=(H, sc.nu)))
    out = torch.empty((H, sc.nu), device=DEV)
    ctl.update(_t(costs), _t(u0), out)  # the samples of iteration 0, regenerated from Philox
    assert ctl.sync() == 0
    sig = _f32(sc.sigma_vec())
    U = u0[None] + oracle.noise(key, 0, K, H, sc.nu, sig)
    S0 = np.stack([np.diag(sig ** 2)] * H)
    nu1, S1, elite, st = oracle.elite_update(costs, U, 64, sc.lam, 0.7, u0, S0, update_cov=True, cov_floor=1e-6)
    assert st == 0
    np.testing.assert_allclose(out.cpu().numpy(), nu1, atol=1e-3, rtol=0)
    Sg = torch.empty((H, sc.nu, sc.nu), device=DEV)
    ctl.covariance(Sg)
    torch.cuda.synchronize()
    assert np.abs(Sg.cpu().numpy() - S1).max() <= 1e-3 * np.abs(S1).max()
    best = torch.empty((H, sc.nu), device=DEV)
    ctl.best_controls(best)
    np.testing.assert_allclose(best.cpu().numpy(), U[elite[0]], atol=2e-6)
