"""Pins for the oracle's MPPI update (Eq. 8a/8d with eta = 1, all samples in
the elite set, beta = lambda).

For a linear-quadratic cost J(U) = U^T Q U + 2 b^T U + c and Gaussian
samples U ~ N(u, Sigma), the exponentially weighted mean converges (as the
sample count grows) to the mean of the Gaussian tilted by exp(-J/lambda):
    (Sigma^-1 + 2Q/lambda)^-1 (Sigma^-1 u - 2b/lambda)
whose fixed point under iteration is the optimum -Q^-1 b.
The LQ system is x_{h+1} = x_h + dt u_h, J = sum_h q x_{h+1}^2 + r u_h^2."""
import numpy as np
import pytest

import oracle


def _lq(H, dt=0.1, q=1.0, r=0.1, x0=1.0):
    # x_{h+1} = x0 + dt * sum_{i<=h} u_i = x0 + (S U)_h
    S = dt * np.tril(np.ones((H, H)))
    Q = q * S.T @ S + r * np.eye(H)
    b = q * S.T @ (x0 * np.ones(H))
    c = q * H * x0 * x0
    return Q, b, c


def _costs(U, Q, b, c):
    return np.einsum("ki,ij,kj->k", U, Q, U) + 2 * U @ b + c


def test_update_matches_tilted_gaussian_mean():
    H, sigma, lam = 4, 0.5, 2.0
    Q, b, c = _lq(H)
    u_nom = np.array([0.2, -0.1, 0.0, 0.3])
    K = 200_000
    eps = oracle.noise(seed=11, iteration=3, K=K, H=H, nu=1, sigma=np.array([sigma]))[..., 0]
    U = u_nom[None, :] + eps
    out, w, st = oracle.mppi_update(_costs(U, Q, b, c), U[..., None], lam, u_nom[:, None])
    assert st == 0
    Si = np.eye(H) / sigma ** 2
    expect = np.linalg.solve(Si + 2 * Q / lam, Si @ u_nom - 2 * b / lam)
    cov = np.linalg.inv(Si + 2 * Q / lam)
    k_eff = 1.0 / np.sum(w ** 2)
    se = np.sqrt(np.diag(cov) / k_eff)
    assert np.all(np.abs(out[:, 0] - expect) < 5 * se + 1e-12)
    assert w.sum() == pytest.approx(1.0, abs=1e-12)


def test_iterated_update_converges_to_lq_optimum():
    H, sigma, lam = 4, 0.5, 1.0
    Q, b, c = _lq(H)
    u = np.zeros(H)
    opt = -np.linalg.solve(Q, b)
    Si = np.eye(H) / sigma ** 2
    contraction = np.linalg.solve(Si + 2 * Q / lam, Si)
    err0 = np.linalg.norm(u - opt)
    for it in range(40):
        eps = oracle.noise(seed=5, iteration=it, K=50_000, H=H, nu=1, sigma=np.array([sigma]))[..., 0]
        U = u[None, :] + eps
        out, w, st = oracle.mppi_update(_costs(U, Q, b, c), U[..., None], lam, u[:, None])
        u = out[:, 0]
    rho = np.abs(np.linalg.eigvals(contraction)).max()
    assert np.linalg.norm(u - opt) < max(rho ** 40 * err0, 0.02)


def test_weights_are_softmax_of_negative_costs():
    rng = np.random.default_rng(0)
    K, H = 64, 3
    costs = rng.uniform(0, 50, K)
    U = rng.normal(size=(K, H, 2))
    lam = 0.7
    out, w, st = oracle.mppi_update(costs, U, lam, np.zeros((H, 2)))
    z = -costs / lam
    soft = np.exp(z - z.max()) / np.exp(z - z.max()).sum()
    np.testing.assert_allclose(w, soft, rtol=1e-12)
    np.testing.assert_allclose(out, np.einsum("k,khj->hj", soft, U), rtol=1e-12, atol=1e-14)


def test_nonfinite_costs_get_zero_weight_and_all_nonfinite_keeps_nominal():
    K, H = 8, 2
    U = np.arange(K * H * 1, dtype=float).reshape(K, H, 1)
    costs = np.array([np.nan, 1.0, np.inf, 2.0, -np.inf, 3.0, 1.0, np.nan])
    out, w, st = oracle.mppi_update(costs, U, 1.0, np.zeros((H, 1)))
    assert st == 0 and w[0] == w[2] == w[4] == w[7] == 0.0
    u_nom = np.array([[5.0], [6.0]])
    out, w, st = oracle.mppi_update(np.full(K, np.nan), U, 1.0, u_nom)
    assert st == 1
    np.testing.assert_array_equal(out, u_nom)


def test_equal_costs_give_the_sample_mean():
    rng = np.random.default_rng(1)
    U = rng.normal(size=(16, 5, 3))
    out, w, st = oracle.mppi_update(np.full(16, 4.2), U, 0.05, np.zeros((5, 3)))
    np.testing.assert_allclose(out, U.mean(0), rtol=1e-13, atol=1e-15)
