"""Scene variants used by the closed-form tests (test-only)."""
import copy

import numpy as np

from paper_2511_21264_gb300 import scenes


def torque_mode(sc, gravcomp=0.0, damping=0.0):
    """Actuators as plain torque sources (gear 1, no servo gain), optional
    gravity compensation and joint damping."""
    sc = copy.deepcopy(sc)
    for arm in sc.links:
        for ln in arm:
            ln.gear, ln.kv, ln.gravcomp, ln.damping = 1.0, 0.0, gravcomp, damping
            ln.tau_max = 1e9
    return sc


def ball_far(sc, pos=(0.0, 5.0, 2.0)):
    """Move the ball far from the arms and the floor."""
    sc = copy.deepcopy(sc)
    b0 = 2 * sc.n_a
    sc.x0 = sc.x0.copy()
    sc.x0[b0:b0 + 3] = pos
    return sc


def planar_single_link(length=0.3, radius=0.01, mass=1.0, dt=1e-3):
    """One-link planar arms (a physical pendulum on each side)."""
    sc = scenes.planar_scene()
    sc = copy.deepcopy(sc)
    sc.n_a = 1
    sc.links = [[scenes.dh_link(length, 0.0, 0.0, 0.0, mass, radius)] for _ in range(2)]
    nq, nv, _ = scenes.dims(1)
    x0 = np.zeros(nq + nv)
    x0[2:5] = (0.0, 5.0, 2.0)
    x0[5] = 1.0
    sc.x0 = x0
    sc.dt = dt
    return torque_mode(sc)
