"""The paper's full Eq. 8 on the GPU (elite set, learning rate, covariance
blocks) against the FP64 oracle.  Tolerances: nominal update <= 1e-3
(absolute), covariance blocks <= 1e-3 relative to their largest entry."""
import numpy as np
import pytest

import oracle
from paper_2511_21264_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"


def _t(a):
    return torch.tensor(np.ascontiguousarray(np.asarray(a, np.float32)), device=DEV)


def _f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def native():
    from paper_2511_21264_gb300 import native as nat
    nat.build()
    return nat


def _ctl(native, cfg, K, H, key=5):
    sc = scenes.config(cfg)
    blob = sc.to_blob()
    gm = native.Model(blob)
    ctl = native.Controller(gm, K, H, sc.lam, sc.sigma_vec(), key)
    return sc, gm, oracle.Model(blob), ctl


@pytest.mark.parametrize("n_elite,eta,cov", [(32, 1.0, False), (20, 0.7, True), (257, 0.5, True)])
def test_elite_update_matches_oracle(native, n_elite, eta, cov):
    K, H = 257, 5
    sc, gm, om, ctl = _ctl(native, 2, K, H)
    ctl.set_update(n_elite, eta, cov, 1e-6)
    rng = np.random.default_rng(n_elite)
    costs = _f32(rng.uniform(3.0, 4.0, K))
    u_nom = _f32(rng.normal(scale=0.1, size=(H, sc.nu)))
    out = torch.empty((H, sc.nu), device=DEV)
    ctl.update(_t(costs), _t(u_nom), out)
    assert ctl.sync() == 0
    sig = _f32(sc.sigma_vec())
    S0 = np.stack([np.diag(sig ** 2)] * H)
    U = u_nom[None] + oracle.noise(5, 0, K, H, sc.nu, sig)
    nu1, S1, elite, st = oracle.elite_update(costs, U, n_elite, sc.lam, eta, u_nom, S0, update_cov=cov,
                                             cov_floor=1e-6)
    np.testing.assert_allclose(out.cpu().numpy(), nu1, atol=1e-3, rtol=0)
    assert np.abs(out.cpu().numpy() - nu1).max() < 2e-5
    S = torch.empty((H, sc.nu, sc.nu), device=DEV)
    ctl.covariance(S)
    torch.cuda.synchronize()
    Sg = S.cpu().numpy()
    assert np.abs(Sg - S1).max() <= 1e-3 * np.abs(S1).max()
    # the optimiser's output: controls of the lowest-cost sample
    best = torch.empty((H, sc.nu), device=DEV)
    ctl.best_controls(best)
    np.testing.assert_allclose(best.cpu().numpy(), U[elite[0]], atol=2e-6)


def test_two_iterations_with_covariance_adaptation(native):
    """mppi_step twice with the elite set and the covariance update: the
    second iteration samples through the adapted blocks' factors."""
    K, H = 64, 8
    sc, gm, om, ctl = _ctl(native, 1, K, H, key=9)
    n_e, eta = 16, 0.6
    ctl.set_update(n_e, eta, True, 1e-6)
    x = _f32(sc.x0)
    u = torch.zeros((H, sc.nu), device=DEV)
    sig = _f32(sc.sigma_vec())
    nu_o = np.zeros((H, sc.nu))
    S_o = np.stack([np.diag(sig ** 2)] * H)
    for it in range(2):
        ctl.step(_t(x), u, u)
        assert ctl.sync() == 0
        U = om.sample_cov(9, it, K, nu_o, S_o)
        costs = om.rollout_many(x, U, nthreads=4)
        nu_o, S_o, elite, st = oracle.elite_update(costs, U, n_e, sc.lam, eta, nu_o, S_o, True, 1e-6)
        S_o = S_o.copy()
        np.testing.assert_allclose(u.cpu().numpy(), nu_o, atol=1e-3, rtol=0)
        S = torch.empty((H, sc.nu, sc.nu), device=DEV)
        ctl.covariance(S)
        torch.cuda.synchronize()
        assert np.abs(S.cpu().numpy() - S_o).max() <= 1e-3 * np.abs(S_o).max()
        # keep the oracle on the GPU's FP32 state so the next samples agree
        nu_o = _f32(u.cpu().numpy())
        S_o = _f32(S.cpu().numpy())


def test_diagonal_covariance_samples_like_the_plain_path(native):
    K, H = 96, 6
    sc, gm, om, ctl_a = _ctl(native, 2, K, H, key=3)
    _, _, _, ctl_b = _ctl(native, 2, K, H, key=3)
    sig = sc.sigma_vec().astype(np.float32)
    ctl_b.set_covariance(_t(np.stack([np.diag(sig ** 2)] * H)))
    x = _t(_f32(sc.x0))
    ua = torch.zeros((H, sc.nu), device=DEV)
    ub = torch.zeros((H, sc.nu), device=DEV)
    ctl_a.step(x, ua, ua)
    ctl_b.step(x, ub, ub)
    assert ctl_a.sync() == 0 and ctl_b.sync() == 0
    np.testing.assert_allclose(ub.cpu().numpy(), ua.cpu().numpy(), atol=1e-6, rtol=0)


def test_set_update_validation(native):
    sc, gm, om, ctl = _ctl(native, 1, 64, 4)
    from paper_2511_21264_gb300.native import MPPIError
    for args in ((0, 1.0, False), (65, 1.0, False), (8, 0.0, False), (8, 1.5, False)):
        with pytest.raises(MPPIError):
            ctl.set_update(*args)
