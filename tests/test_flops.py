"""The algorithmic FLOP model behind the bench line's roofline fraction:
totals quoted for the three configurations, the charge of one exact
capsule-box test, and the Cholesky part against a direct count of the
operations of an n x n factor and two triangular solves."""
import pytest

from paper_2511_21264_gb300 import flops, scenes


@pytest.mark.parametrize("cfg,one,lone", [(1, 4364.0, 3824.0), (2, 10478.0, 9216.0), (3, 13826.0, 12564.0)])
def test_totals_per_configuration(cfg, one, lone):
    sc = scenes.config(cfg)
    assert flops.per_sample_step(sc, 1.0, 0.0, 0.0) == one
    assert flops.per_sample_step(sc, 1.0, 0.0, 1.0) == lone


def test_parts_sum_and_exact_test_charge():
    sc = scenes.config(3)
    total, parts = flops.per_sample_step(sc, 1.0, 0.2, 0.9, breakdown=True)
    assert total == pytest.approx(sum(parts.values()))
    step = flops.per_sample_step(sc, 1.0, 1.0, 0.0) - flops.per_sample_step(sc, 1.0, 0.0, 0.0)
    assert step == 1919.0
    # more contacts never cost less
    assert flops.per_sample_step(sc, 2.0, 0.0, 0.0) > flops.per_sample_step(sc, 1.0, 0.0, 0.0)


def _cholesky_ops(n):
    # right-hand count: for column j the pivot takes j multiply-adds (2 each)
    # and a square root; each of the n-1-j entries below it takes j
    # multiply-adds and one scaling multiply
    ops = 0
    for j in range(n):
        ops += 2 * j
        ops += (n - 1 - j) * (2 * j + 1)
    return ops


def test_cholesky_part_counts_two_arm_factors_and_solves():
    for cfg in (1, 3):
        sc = scenes.config(cfg)
        n = sc.n_a
        _, parts = flops.per_sample_step(sc, 1.0, 0.0, 0.0, breakdown=True)
        solves = 2 * (n * (n - 1) + n)   # forward and back substitution: n(n-1)/2 multiply-adds and n scalings each
        assert parts["cholesky"] == 2 * (_cholesky_ops(n) + solves) + 6
