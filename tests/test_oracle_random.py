"""Pins for the oracle's Philox4x32-10 generator, Box-Muller normals and
noise layout (sampling step of Alg. 1: draws from N(nu_m, Sigma_m))."""
import os

import numpy as np
import pytest
from scipy import stats

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(t, 16) for t in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat())
def test_philox_known_answers(ctr, key, expect):
    assert oracle.philox4x32_10(ctr, key) == expect


def test_uniform_mapping_bounds():
    # ((x >> 9) + 1/2) 2^-23 never reaches 0 or 1: the extreme words give
    # finite normals
    z = oracle.normals4([0, 0, 0xFFFFFFFF, 0xFFFFFFFF])
    assert np.all(np.isfinite(z))
    # word 0 = 0 -> u = 2^-24 -> r = sqrt(2 * 24 ln 2)
    r = np.sqrt(-2.0 * np.log(0.5 / 8388608.0))
    assert z[0] == pytest.approx(r * np.cos(2 * np.pi * 0.5 / 8388608.0), rel=1e-15)
    # every uniform is exactly representable in FP32 (24-bit significand)
    xs = np.array([0, 1, 511, 512, 0x7FFFFFFF, 0xFFFFFE00, 0xFFFFFFFF], dtype=np.uint64)
    u = ((xs >> 9).astype(np.float64) + 0.5) / 2 ** 23
    assert np.all(u.astype(np.float32).astype(np.float64) == u)
    assert np.all((u > 0) & (u < 1))


def test_box_muller_pairs_closed_form():
    # u0 = 1/2 + 1/2^25 (x = 0x80000000), u1 = 1/4 + ... : angle 90 degrees
    w = [0x80000000, 0x40000000, 0x80000000, 0x00000000]
    z = oracle.normals4(w)
    u0 = ((0x80000000 >> 9) + 0.5) / 2 ** 23
    u1 = ((0x40000000 >> 9) + 0.5) / 2 ** 23
    r = np.sqrt(-2 * np.log(u0))
    assert z[0] == pytest.approx(r * np.cos(2 * np.pi * u1), abs=1e-15)
    assert z[1] == pytest.approx(r * np.sin(2 * np.pi * u1), rel=1e-14)


def test_noise_layout_and_counter_mapping():
    sigma = np.array([0.5, 1.0, 2.0, 3.0, 4.0, 5.0])
    eps = oracle.noise(seed=0x1234_5678_9ABC_DEF0, iteration=7, K=3, H=2, nu=6, sigma=sigma)
    key = [0x9ABCDEF0, 0x12345678]
    for k in range(3):
        for h in range(2):
            for jb in range(2):
                w = oracle.philox4x32_10([jb, h, k, 7], key)
                z = oracle.normals4(w)
                for t in range(4):
                    j = 4 * jb + t
                    if j < 6:
                        assert eps[k, h, j] == pytest.approx(sigma[j] * z[t], rel=1e-15, abs=1e-300)


def test_normals_distribution():
    eps = oracle.noise(seed=42, iteration=0, K=4096, H=16, nu=4, sigma=np.ones(4)).ravel()
    n = eps.size
    assert abs(eps.mean()) < 5 / np.sqrt(n)
    assert abs(eps.var() - 1) < 5 * np.sqrt(2 / n)
    assert abs(stats.skew(eps)) < 5 * np.sqrt(6 / n)
    assert abs(stats.kurtosis(eps)) < 5 * np.sqrt(24 / n)
    assert stats.kstest(eps, "norm").pvalue > 1e-3
    # cos/sin partners are uncorrelated
    e = oracle.noise(seed=9, iteration=1, K=8192, H=4, nu=4, sigma=np.ones(4))
    r = np.corrcoef(e[..., 0].ravel(), e[..., 1].ravel())[0, 1]
    assert abs(r) < 5 / np.sqrt(e[..., 0].size)


def test_streams_differ_by_iteration_and_seed():
    a = oracle.noise(1, 0, 64, 4, 4, np.ones(4))
    b = oracle.noise(1, 1, 64, 4, 4, np.ones(4))
    c = oracle.noise(2, 0, 64, 4, 4, np.ones(4))
    assert np.abs(a - b).max() > 0.1 and np.abs(a - c).max() > 0.1
