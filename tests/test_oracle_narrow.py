"""Brute-force pins for the oracle's narrow phase.

Distances between a sphere, a capsule and an axis-aligned box are checked
against dense sampling of the shapes in FP64: for separated shapes the
surface distance is the minimum over sampled points; for penetrating shapes
the depth is checked against the minimum of the box's signed distance over
densely sampled segment points, or against hand-derived special cases."""
import numpy as np
import pytest

import oracle


def _seg_pts(a, b, n=20001):
    t = np.linspace(0.0, 1.0, n)[:, None]
    return a[None, :] + t * (b - a)[None, :]


def _box_dist_points(P, bc, bh):
    """Unsigned distance from points to a box, by sampling its surface."""
    n = 161
    u = np.linspace(-1, 1, n)
    U, V = np.meshgrid(u, u, indexing="ij")
    faces = []
    for ax in range(3):
        o1, o2 = [k for k in range(3) if k != ax]
        for s in (-1.0, 1.0):
            F = np.zeros((n * n, 3))
            F[:, ax] = bc[ax] + s * bh[ax]
            F[:, o1] = bc[o1] + U.ravel() * bh[o1]
            F[:, o2] = bc[o2] + V.ravel() * bh[o2]
            faces.append(F)
    S = np.concatenate(faces)
    d = np.full(P.shape[0], np.inf)
    for i in range(0, S.shape[0], 20000):
        blk = S[i:i + 20000]
        d = np.minimum(d, np.sqrt(((P[:, None, :] - blk[None, :, :]) ** 2).sum(-1)).min(1))
    return d


def test_sphere_capsule_brute_force():
    rng = np.random.default_rng(0)
    for _ in range(40):
        c = rng.uniform(-0.5, 0.5, 3)
        a, b = rng.uniform(-0.5, 0.5, 3), rng.uniform(-0.5, 0.5, 3)
        r, rc = rng.uniform(0.02, 0.15), rng.uniform(0.02, 0.08)
        d, p, n = oracle.sphere_capsule(c, r, a, b, rc)
        P = _seg_pts(a, b)
        dist_axis = np.sqrt(((P - c) ** 2).sum(1)).min()
        assert d == pytest.approx(dist_axis - r - rc, abs=1e-8)
        assert np.linalg.norm(n) == pytest.approx(1.0, abs=1e-14)
        # the contact point lies halfway between the two witness points
        assert np.linalg.norm(p - (c - (r + 0.5 * d) * n)) < 1e-12


def test_sphere_box_outside_brute_force_and_inside_closed_form():
    rng = np.random.default_rng(1)
    bc, bh = np.array([0.1, -0.2, 0.3]), np.array([0.1, 0.15, 0.05])
    C = rng.uniform(-0.6, 0.6, (30, 3)) + bc
    dist_surf = _box_dist_points(C, bc, bh)
    for c, ds in zip(C, dist_surf):
        inside = np.all(np.abs(c - bc) <= bh)
        d, p, n = oracle.sphere_box(c, 0.07, bc, bh)
        if inside:
            continue
        assert d == pytest.approx(ds - 0.07, abs=2e-3 * max(bh))
        exact = np.linalg.norm(c - np.clip(c, bc - bh, bc + bh)) - 0.07
        assert d == pytest.approx(exact, abs=1e-14)
    # centre inside: nearest face, depth = face distance + r
    c = bc + np.array([0.0, 0.1, 0.0])       # 0.05 from the +y face
    d, p, n = oracle.sphere_box(c, 0.07, bc, bh)
    # z faces are nearer (0.05 as well): tie -> lowest axis among equals
    assert d == pytest.approx(-(0.05) - 0.07, abs=1e-14)
    c = bc + np.array([0.0, 0.12, 0.0])      # 0.03 from +y face, 0.05 from z faces
    d, p, n = oracle.sphere_box(c, 0.07, bc, bh)
    assert d == pytest.approx(-0.03 - 0.07, abs=1e-14)
    np.testing.assert_array_equal(n, [0.0, 1.0, 0.0])
    # exact ties (dyadic values): lowest axis wins, + face before - face
    bc2, bh2 = np.zeros(3), np.array([0.25, 0.5, 0.125])
    d, p, n = oracle.sphere_box(np.array([0.125, 0.0, 0.0]), 0.0625, bc2, bh2)
    np.testing.assert_array_equal(n, [1.0, 0.0, 0.0])      # +x and +-z tie at 0.125
    assert d == -0.125 - 0.0625
    d, p, n = oracle.sphere_box(np.array([0.0, 0.0, 0.0]), 0.0625, bc2, bh2)
    np.testing.assert_array_equal(n, [0.0, 0.0, 1.0])      # +z and -z tie
    d, p, n = oracle.sphere_box(np.array([0.0, -0.375, 0.0]), 0.0625, bc2, bh2)
    np.testing.assert_array_equal(n, [0.0, -1.0, 0.0])     # -y (0.125) vs z (0.125): y is lower axis


def test_box_sdf_sign_and_gradient():
    bc, bh = np.zeros(3), np.array([0.2, 0.1, 0.3])
    rng = np.random.default_rng(2)
    for _ in range(50):
        x = rng.uniform(-0.5, 0.5, 3)
        s, n, surf = oracle.box_sdf(x, bc, bh)
        inside = np.all(np.abs(x) < bh)
        assert (s < 0) == inside
        h = 1e-7
        # gradient of the SDF equals the normal where it is differentiable
        g = np.array([(oracle.box_sdf(x + h * e, bc, bh)[0] - oracle.box_sdf(x - h * e, bc, bh)[0]) / (2 * h)
                      for e in np.eye(3)])
        if np.abs(np.sort(np.abs(np.abs(x) - bh))[:2]).min() > 1e-3:
            np.testing.assert_allclose(g, n, atol=1e-5)


def test_capsule_box_brute_force():
    rng = np.random.default_rng(3)
    bc, bh = np.array([0.0, 0.0, 0.2]), np.array([0.12, 0.08, 0.1])
    for trial in range(40):
        a = rng.uniform(-0.5, 0.5, 3) + bc
        b = rng.uniform(-0.5, 0.5, 3) + bc
        rc = 0.05
        d, p, n, t = oracle.capsule_box(a, b, rc, bc, bh)
        P = _seg_pts(a, b, 4001)
        sdf = np.array([oracle.box_sdf(x, bc, bh)[0] for x in P])
        # the SDF is 1-Lipschitz, so the true minimum lies within half a
        # sample spacing below the sampled one, and never above it
        spacing = np.linalg.norm(b - a) / (P.shape[0] - 1)
        assert d + rc <= sdf.min() + 1e-12
        assert d + rc >= sdf.min() - 0.5 * spacing - 1e-12
        if sdf.min() > 0:
            ds = _box_dist_points(P[np.argsort(sdf)[:3]], bc, bh).min()
            assert d == pytest.approx(ds - rc, abs=2e-3 * bh.max())


def test_capsule_box_flat_minimum_takes_interval_midpoint():
    # segment parallel to the top face, partly over the box: every point
    # over the face is equally close; the contact is the middle of that set
    bc, bh = np.zeros(3), np.array([0.2, 0.2, 0.1])
    a, b = np.array([-0.1, 0.0, 0.15]), np.array([0.5, 0.0, 0.15])
    d, p, n, t = oracle.capsule_box(a, b, 0.08, bc, bh)
    assert d == pytest.approx(0.05 - 0.08, abs=1e-14)
    # flat set: x in [-0.1, 0.2] -> t in [0, 0.5]
    assert t == pytest.approx(0.25, abs=1e-6)
    np.testing.assert_allclose(n, [0, 0, 1], atol=1e-12)


def test_canonical_pair_order_and_cap():
    from paper_2511_21264_gb300 import scenes
    sc = scenes.config(3)
    m = oracle.Model(sc.to_blob())
    x = sc.x0.copy()
    xo, info, lam, cons = m.step(x, np.zeros(sc.nu), want_contacts=True)
    assert info.ncon == info.nactive == 1       # only the ball on the floor
    assert cons[0]["bodyA"] == 2 * sc.n_a and cons[0]["box"] == -1
