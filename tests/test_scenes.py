"""The seeded scene generator and the blob format."""
import struct

import numpy as np
import pytest

import oracle
from paper_2511_21264_gb300 import scenes


@pytest.mark.parametrize("n", [1, 2, 3])
def test_blob_round_trip(n):
    sc = scenes.config(n)
    blob = sc.to_blob()
    magic, ver, count, _ = struct.unpack("<IIII", blob[:16])
    assert (magic, ver) == (scenes.MAGIC, scenes.VERSION)
    assert len(blob) == 16 + 8 * count
    vals = np.frombuffer(blob[16:], dtype="<f8")
    assert vals[0] == sc.n_a and vals[1] == sc.n_boxes
    np.testing.assert_array_equal(vals[-(sc.nq + sc.nv):], sc.x0)
    m = oracle.Model(blob)
    assert (m.nq, m.nv, m.nu) == (sc.nq, sc.nv, sc.nu)


def test_malformed_blob_rejected():
    blob = bytearray(scenes.config(1).to_blob())
    blob[0] ^= 1
    with pytest.raises(ValueError):
        oracle.Model(bytes(blob))
    with pytest.raises(ValueError):
        oracle.Model(scenes.config(1).to_blob()[:-8])


def test_seeded_and_reproducible():
    a, b = scenes.config(3, seed=4), scenes.config(3, seed=4)
    assert a.to_blob() == b.to_blob()
    assert scenes.config(3, seed=5).to_blob() != a.to_blob()


def test_obstacle_layout_constraints():
    sc = scenes.config(3, seed=0)
    assert sc.n_boxes == 8
    assert np.all(sc.boxes_h >= 0.03) and np.all(sc.boxes_h <= 0.15)
    start = sc.x0[14:17]
    for c, h in zip(sc.boxes_c, sc.boxes_h):
        assert not np.all(np.abs(start - c) <= h + sc.ball_r)
        assert not np.all(np.abs(np.asarray(sc.goal) - c) <= h + sc.ball_r)


def test_home_state_has_only_floor_contact():
    for sc in (scenes.config(1), scenes.config(2), scenes.config(3)):
        m = oracle.Model(sc.to_blob())
        _, info, _, cons = m.step(sc.x0, np.zeros(sc.nu), want_contacts=True)
        assert info.nactive == 1 and cons[0]["bodyB"] == -1 and cons[0]["box"] == -1


def test_batched_pool_draws_from_the_sets():
    pool = scenes.batched_pool(12)
    assert {s.K for s in pool} <= set(scenes.K_CHOICES)
    assert {s.H for s in pool} <= set(scenes.H_CHOICES)
    assert all(0 <= s.n_boxes <= 16 for s in pool)


def test_controller_keys_distinct():
    keys = {scenes.controller_key(s, i) for s in range(10) for i in range(64)}
    assert len(keys) == 640
