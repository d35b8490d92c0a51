"""Pins for the oracle's full Eq. 8 update (elite set, learning rate eta,
per-step covariance blocks) and for sampling from those blocks."""
import numpy as np
import pytest

import oracle
from paper_2511_21264_gb300 import scenes


def _data(K=40, H=3, nu=4, seed=0):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(K, H, nu)), rng.uniform(1.0, 2.0, K), rng.normal(size=(H, nu))


def _spd(H, nu, rng):
    A = rng.normal(size=(H, nu, nu))
    return np.einsum("hij,hkj->hik", A, A) + 0.5 * np.eye(nu)


def test_reduces_to_the_softmax_mean():
    U, c, nu0 = _data()
    S0 = _spd(3, 4, np.random.default_rng(1))
    nu1, S1, elite, st = oracle.elite_update(c, U, n_elite=40, beta=0.3, eta=1.0, nu_in=nu0, Sigma_in=S0,
                                             update_cov=False)
    ref, w, _ = oracle.mppi_update(c, U, 0.3, nu0)
    np.testing.assert_allclose(nu1, ref, rtol=1e-13, atol=1e-14)
    np.testing.assert_array_equal(S1, S0)


def test_zero_learning_rate_keeps_the_distribution():
    U, c, nu0 = _data()
    S0 = _spd(3, 4, np.random.default_rng(2))
    nu1, S1, _, _ = oracle.elite_update(c, U, 10, 0.3, 0.0, nu0, S0, update_cov=True, cov_floor=0.0)
    np.testing.assert_array_equal(nu1, nu0)
    np.testing.assert_allclose(S1, S0, rtol=0, atol=0)


def test_elite_set_is_the_lowest_costs_with_index_ties():
    U, c, nu0 = _data(K=50)
    c[[3, 17, 40]] = 0.5          # exact ties at the bottom
    c[7] = np.nan                 # non-finite costs are never elite
    nu1, S1, elite, st = oracle.elite_update(c, U, 8, 0.3, 1.0, nu0, _spd(3, 4, np.random.default_rng(3)))
    order = sorted(range(50), key=lambda k: (np.inf if np.isnan(c[k]) else c[k], k))[:8]
    assert list(elite) == order and 7 not in elite


def test_weighted_covariance_equals_covariance_of_a_population_with_multiplicities():
    """With s_j = exp(-(c_j - c_min)/beta) set to integers 1..3, dSigma is the
    covariance (about nu') of the population in which sample j appears s_j
    times; with eta = 1 nu' is that population's mean."""
    rng = np.random.default_rng(4)
    K, H, nu, beta = 12, 2, 3, 0.7
    U = rng.normal(size=(K, H, nu))
    mult = rng.integers(1, 4, K)
    mult[0] = 1
    costs = 5.0 - beta * np.log(mult / mult.max())
    nu1, S1, elite, st = oracle.elite_update(costs, U, K, beta, 1.0, np.zeros((H, nu)), np.zeros((H, nu, nu)),
                                             update_cov=True, cov_floor=0.0)
    pop = np.repeat(U, mult, axis=0)
    np.testing.assert_allclose(nu1, pop.mean(0), rtol=1e-12, atol=1e-13)
    for h in range(H):
        np.testing.assert_allclose(S1[h], np.cov(pop[:, h, :].T, bias=True), rtol=1e-11, atol=1e-13)


def test_learning_rate_blends_and_floor_is_added():
    rng = np.random.default_rng(5)
    U = rng.normal(size=(20, 2, 3))
    c = np.full(20, 3.0)          # equal weights
    S0 = _spd(2, 3, rng)
    eta, floor = 0.3, 1e-4
    nu0 = rng.normal(size=(2, 3))
    nu1, S1, _, _ = oracle.elite_update(c, U, 20, 1.0, eta, nu0, S0, update_cov=True, cov_floor=floor)
    np.testing.assert_allclose(nu1, (1 - eta) * nu0 + eta * U.mean(0), rtol=1e-13)
    for h in range(2):
        d = U[:, h, :] - nu1[h]
        dS = d.T @ d / 20
        np.testing.assert_allclose(S1[h], (1 - eta) * S0[h] + eta * dS + floor * np.eye(3), rtol=1e-12)
        assert np.linalg.eigvalsh(S1[h]).min() > 0


def test_covariance_sampling():
    sc = scenes.config(1)
    m = oracle.Model(sc.to_blob())
    H, nu = 3, sc.nu
    sig = sc.sigma_vec()
    nu0 = np.random.default_rng(6).normal(scale=0.1, size=(H, nu))
    # diagonal blocks reproduce the plain sampler exactly
    S = np.stack([np.diag(sig ** 2)] * H)
    U = m.sample_cov(11, 2, 50, nu0, S)
    eps = oracle.noise(11, 2, 50, H, nu, sig)
    np.testing.assert_allclose(U, nu0[None] + eps, rtol=1e-14, atol=1e-15)
    # a full block: the empirical covariance matches
    rng = np.random.default_rng(7)
    A = rng.normal(scale=0.2, size=(nu, nu))
    Sf = np.stack([A @ A.T + 0.01 * np.eye(nu)] * H)
    U = m.sample_cov(3, 0, 20000, nu0, Sf)
    emp = np.cov(U[:, 1, :].T)
    se = np.sqrt((Sf[1] ** 2 + np.outer(np.diag(Sf[1]), np.diag(Sf[1]))) / 20000)
    assert np.all(np.abs(emp - Sf[1]) < 5 * se + 1e-12)
    np.testing.assert_allclose(U.mean(0), nu0, atol=5 * np.sqrt(np.diag(Sf[1]).max() / 20000))
