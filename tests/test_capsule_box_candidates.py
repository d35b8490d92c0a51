"""The kernels' closed candidate set for the capsule-box minimum (the table
of 43 candidates in csrc/mppi_device.cuh, read from the source here): the
smallest box SDF over the candidates' clamped parameters equals the FP64
oracle's exact minimum of the SDF along the segment, on random segments
and boxes (outside, crossing and inside the box) and on degenerate
directions (segments parallel to faces and axes)."""
import os
import re

import numpy as np
import pytest

import oracle

SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", "paper_2511_21264_gb300", "csrc",
                   "mppi_device.cuh")


def _table():
    text = open(SRC).read()
    body = text[text.index("CB_TABLE[CB_CANDIDATES][3] = {"):]
    body = body[:body.index("};")]
    rows = re.findall(r"\{\{([^}]*)\},\s*\{([^}]*)\},\s*\{([^}]*)\}\}", body)
    return np.array([[[float(v.strip().rstrip("f")) for v in axis.split(",")] for axis in row] for row in rows])


def _sdf(x, c, h):
    q = np.abs(x - c) - h
    return np.linalg.norm(np.maximum(q, 0.0)) + min(q.max(), 0.0)


def _candidates(T, a, d, c, h):
    ts = []
    for i in range(len(T)):
        num = 1.0 if i == 1 else 0.0
        den = 1.0 if i < 2 else 0.0
        for k in range(3):
            s, Z, p, b = T[i, k]
            al = s * (a[k] - c[k]) - Z * h[k]
            be = s * d[k]
            t1 = b - p * be
            num += al * t1
            den -= be * t1
        with np.errstate(divide="ignore", invalid="ignore"):
            t = num / den
        t = 0.0 if not (t >= 0.0) else min(t, 1.0)
        ts.append(t)
    return np.array(ts)


def test_table_shape():
    T = _table()
    assert T.shape == (43, 3, 4)
    assert set(np.unique(T[:, :, 0])) <= {-1.0, 1.0} and set(np.unique(T[:, :, 1])) <= {0.0, 1.0}


@pytest.mark.parametrize("seed", range(4))
def test_candidate_minimum_is_the_exact_minimum(seed):
    T = _table()
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(300):
        c = rng.normal(scale=0.3, size=3)
        h = rng.uniform(0.03, 0.3, size=3)
        a0 = c + rng.normal(scale=0.4, size=3)
        a1 = a0 + rng.normal(scale=0.4, size=3)
        if rng.random() < 0.3:            # axis-parallel or face-parallel directions
            a1 = a0.copy()
            a1[rng.integers(3)] += rng.normal(scale=0.5)
        d = a1 - a0
        ts = _candidates(T, a0, d, c, h)
        fmin = min(_sdf(a0 + t * d, c, h) for t in ts)
        ref = oracle.capsule_box(a0, a1, 0.0, c, h)[0]
        worst = max(worst, abs(fmin - ref))
    assert worst < 1e-9
