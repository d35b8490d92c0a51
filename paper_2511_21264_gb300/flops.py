"""Algorithmic FP32 operation count of one simulated sample-step.

Counts what the method must compute per sample and per time step in this
formulation (add, sub, mul = 1 FLOP, fused multiply-add = 2), with the
recursive algorithms' O(n) prefix/suffix sums, the Cholesky factor of each
arm's (M + dt D) block, and contact rows restricted to the degrees of
freedom they touch.  Work the kernels do redundantly (several lanes drawing
the same Philox block, zero blocks of contact rows, per-lane suffix sums)
is not counted, so the figure cannot be inflated by waste.  Square roots,
divisions, trigonometric, exponential and logarithmic functions run on the
special-function units and are not FP32 FLOPs; Philox is integer work.

The data-dependent terms (active contacts per step, capsule-box pairs that
pass the separating-axis cull, steps whose only contact is the ball against
static geometry) are measured on the device during the timed run
(mppi_profile_read, mppi_profile_lone_contacts).
"""
from __future__ import annotations


def per_sample_step(scene, contacts: float, box_tests: float, lone: float = 0.0, breakdown: bool = False):
    """lone: the sample-steps (per sample-step) whose only contact is the ball
    against the floor or a box.  Such a contact touches the ball's six
    coordinates alone and its Delassus block is diagonal, so it costs its
    three rows and one projected sweep; the other contacts are charged as
    rows over the ball and one arm chain with `sweeps` sweeps."""
    na = scene.n_a
    nl, nv, nu, nb = 2 * na, 2 * na + 6, 2 * na, scene.n_boxes
    sweeps = scene.sweeps
    parts = {}
    # a1 sampling: uniform mapping (2 x 2), -2 log(u), r * trig, sigma z + u
    parts["sample"] = 8 * nu
    # a2 kinematics per link: R Rz (6 x 3), p += Rj Fp (18), R Fp (9 x 5),
    #    three points (COM, capsule ends) 3 x 18
    parts["fk"] = nl * (18 + 18 + 45 + 54)
    # a3 broad + narrow phase
    sphere_capsule = 53
    sphere_box = 25
    cull = 28  # segment against the inflated box: centre offset, three box axes, three cross axes
    # exact capsule-box distance of a pair that passes the cull: the 43
    # candidate parameters along the segment (the two ends 0, the nine slab
    # and centre crossings 3 each, the twelve edge-region stationary points
    # 18, the eight vertex-region ones 22, the twelve face-distance crossings
    # 14), each clamped (2), the box SDF there (26: the point 6, per axis 6,
    # root and sum 2) and the running minimum (2); at the minimiser the SDF
    # with normal and surface point (30) and the contact point (12)
    exact = (3 * 9 + 18 * 12 + 22 * 8 + 14 * 12) + 43 * (2 + 26 + 2) + 30 + 12
    parts["collide"] = 4 + sphere_capsule * nl + sphere_box * nb + cull * nl * nb + exact * box_tests
    # a4/a5 per link: world inertia (R I R^T 75, params 26), axis 6, composite 10,
    #    F = I^c S 42, velocity 12, velocity-product acceleration 42, gravity 6,
    #    I a and I v 84, force cross product 36, subtree force 6, S.F 11, drive 7
    per_link = 75 + 26 + 6 + 10 + 42 + 12 + 42 + 6 + 84 + 36 + 6 + 11 + 7
    mass_cols = 11 * na * (na + 1) // 2          # S_r . F_i for r <= i, per arm
    parts["crba_rnea"] = nl * per_link + 2 * mass_cols + 12
    # a6 Cholesky of each arm block, two triangular solves, free velocity
    chol = sum(2 * j + (na - 1 - j) * (2 * j + 1) for j in range(na))
    solve = 2 * na * (na - 1) + 2 * na
    parts["cholesky"] = 2 * (chol + solve) + 6
    # a7 contact rows: frame, Jacobian of the touched bodies (ball + one
    #    link chain), half-solve with one arm factor, diagonal, reference
    general = max(contacts - lone, 0.0)
    touched = na + 6
    row = 12 + 18 + 19 * (na + 1) // 2 + na * (na - 1) + 2 * touched + 4
    zf = 2 * na * (na + 1) + 6 if general > 0 else 0
    back = 2 * na * (na - 1) if general > 0 else 0
    # a lone ball contact: frame (t1 10, t2 = n x t1 6), lever arm 3, Baumgarte
    #    term 2, per row the lever-arm cross product 9, b = e.v + (d x e).w with
    #    the side sign 12, the diagonal entry, regularisation and sum 9; the
    #    impulse on the ball M^-1 J^T lambda 39
    ball_rows = 16 + 3 + 2 + 3 * (9 + 12 + 9) + 39
    parts["contact_rows"] = zf + 3 * row * general + back + ball_rows * lone
    # a8 PGS: per contact and sweep, normal (dot, update) and tangent pair; a
    #    lone ball contact's one sweep: normal 2, tangents 2, friction disk 8
    parts["pgs"] = sweeps * general * (12 * touched + 16) + 12 * lone
    # a9 integration (coordinates, quaternion)
    parts["integrate"] = 2 * (2 * na + 3) + 50
    # a10 stage cost
    parts["cost"] = 8 + 2 * nu + 8 + (12 if scene.w_grasp else 0)
    total = float(sum(parts.values()))
    if breakdown:
        return total, parts
    return total


def update_flops(K: int, H: int, nu: int) -> float:
    """a11/a12 per iteration: weights (sub, mul) and the weighted sums, with
    the samples regenerated (sampling counted as in per_sample_step)."""
    return K * (2 + 1) * H + K * H * nu * (8 + 2)


def qp_flops(H: int, iters: int) -> float:
    """Algorithmic FP32 operations of the QP smoothing projection (Eq. 5) of
    one sequence: `iters` ADMM iterations in the banded form.  Per horizon
    step and iteration: the four row values (11), clip, dual and scaled
    residual of each row (4 x 5 = 20), the right-hand side scatter (14) and
    one row each of the forward and backward band substitutions (7 + 7);
    FMA = 2, min/max = 1 each.  The start point (prefix sums, B^T vt) adds
    3 per step; sampling is not counted."""
    return float(iters) * 59.0 * H + 3.0 * H


def task_flops(scene, phase: int) -> float:
    """Algorithmic FP32 operations of the ball-task cost suite (Sec. IV-B)
    per state: every collision pair's signed distance -- capsule-box for a
    segment that misses the box (the slab intervals, 21; the squared
    distance's derivative at the six crossings and both ends, 8 x 15; the
    interpolated minimiser, 6; the distance there, 17: 165 in all; segments
    that meet the box take the longer piece walk, not counted),
    sphere-capsule 25, capsule-capsule 90 -- plus 4 for the barrier per
    pair, the end effectors' velocities (6 per joint) and quaternions (25
    each), and the per-state terms (about 80)."""
    na, nb = scene.n_a, scene.n_boxes
    pairs_box = 2 * na * nb
    pairs_ball = 2 * na if phase == 0 else 0
    pairs_arm = na * na
    dist = pairs_box * 165 + pairs_ball * 25 + pairs_arm * 90
    return float(dist + 4 * (pairs_box + pairs_ball + pairs_arm) + 2 * na * 6 + 2 * 25 + 80)
