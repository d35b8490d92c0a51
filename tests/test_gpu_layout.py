"""Rollout layouts: 32, 16 or 8 lanes per sample (one, two or four samples
per warp) and the two placements of a lone ball contact's solve give the
same bits, and each matches the FP64 oracle within the parity bounds.

- single simulator steps from states with up to several contacts (boxes,
  links and the floor), 101 samples (a ragged last warp);
- 8-step rollouts of explicit controls: costs and final states;
- MPPI iterations on the K=256 / H=16 transfer scene (8 boxes) for every
  layout, samples per CTA, eagerly and from the captured graph.
"""
import numpy as np
import pytest

import oracle
from paper_2511_21264_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"


@pytest.fixture(scope="module")
def native():
    from paper_2511_21264_gb300 import native as nat
    nat.build()
    nat.lib()
    return nat


def _layouts(cfg):
    lps = (32, 16, 8) if cfg == 1 else (32, 16)
    return [(l, p) for l in lps for p in (0, 1)]


def _f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def _t(a):
    return torch.tensor(np.ascontiguousarray(np.asarray(a, np.float32)), device=DEV)


def _states(sc, om, n, seed, min_gap=1e-4, **kw):
    out, s = [], seed
    while len(out) < n:
        for x in _f32(scenes.random_states(sc, 2 * n, s, **kw)):
            if om.min_abs_dist(x) > min_gap:
                out.append(x)
                if len(out) == n:
                    break
        s += 1000
    return np.array(out)


def _controller(native, cfg, K, H):
    sc = scenes.config(cfg)
    blob = sc.to_blob()
    gm = native.Model(blob)
    ctl = native.Controller(gm, K, H, sc.lam, sc.sigma_vec(), scenes.controller_key(cfg, 5))
    return sc, gm, oracle.Model(blob), ctl


@pytest.mark.parametrize("cfg", [1, 2, 3])
def test_single_step_same_bits_in_every_layout(native, cfg):
    n = 101
    sc, gm, om, ctl = _controller(native, cfg, K=n, H=1)
    X = _states(sc, om, n, seed=40 + cfg)
    U1 = _f32(np.random.default_rng(cfg).normal(scale=0.5, size=(n, sc.nu)))
    outs = []
    for lps, place in _layouts(cfg):
        for spc in (1, 4):
            ctl.set_layout(lps, place)
            ctl.set_launch(spc)
            xs = _t(X)
            ctl.sim_step(xs, _t(U1))
            assert ctl.sync() == 0
            outs.append(((lps, place, spc), xs.cpu().numpy()))
    ref = outs[0][1]
    for tag, g in outs[1:]:
        np.testing.assert_array_equal(g, ref, err_msg=str(tag))
    ncon = []
    for i in range(n):
        xo, info = om.step(X[i], U1[i])
        ncon.append(info.ncon)
        assert np.abs(ref[i] - xo).max() <= 1e-4 * max(1.0, np.abs(xo).max()), i
    assert max(ncon) >= 2


@pytest.mark.parametrize("cfg", [1, 2, 3])
def test_rollout_costs_same_bits_in_every_layout(native, cfg):
    n, H = 67, 8
    sc, gm, om, ctl = _controller(native, cfg, K=n, H=H)
    X = _states(sc, om, n, seed=60 + cfg, q_spread=0.2, v_spread=0.2)
    U = _f32(np.random.default_rng(70 + cfg).normal(scale=sc.sigma, size=(n, H, sc.nu)))
    outs = []
    for lps, place in _layouts(cfg):
        ctl.set_layout(lps, place)
        costs = torch.empty(n, device=DEV)
        xo = torch.empty((n, sc.nq + sc.nv), device=DEV)
        ctl.rollout_batch(_t(X), _t(U), costs, xo)
        assert ctl.sync() == 0
        outs.append(((lps, place), costs.cpu().numpy(), xo.cpu().numpy()))
    for tag, c, x in outs[1:]:
        np.testing.assert_array_equal(c, outs[0][1], err_msg=str(tag))
        np.testing.assert_array_equal(x, outs[0][2], err_msg=str(tag))
    gc = outs[0][1]
    checked = 0
    for i in range(n):
        c, T = om.rollout(X[i], U[i], traj=True)
        if all(om.min_abs_dist(T[h]) > 1e-5 for h in range(H)):
            checked += 1
            assert abs(gc[i] - c) <= 1e-3 * abs(c), i
    assert checked >= 0.8 * n


def test_iterations_same_bits_in_every_layout_transfer(native):
    K, H = 256, 16
    sc, gm, om, ctl = _controller(native, 3, K=K, H=H)
    x = _t(sc.x0)
    s = torch.cuda.Stream()
    outs = []
    with torch.cuda.stream(s):
        for lps, place in _layouts(3):
            for spc in (2, 8):
                ctl.set_layout(lps, place)
                ctl.set_launch(spc)
                for graph in (False, True):
                    ctl.set_iteration(0, stream=s)
                    u = torch.zeros((H, sc.nu), device=DEV)
                    if graph:
                        ctl.solve(x, u, 4, stream=s)
                    else:
                        for _ in range(4):
                            ctl.step(x, u, u, stream=s)
                    outs.append(((lps, place, spc, graph), u))
        assert ctl.sync(stream=s) == 0
    s.synchronize()
    for tag, u in outs[1:]:
        assert torch.equal(u, outs[0][1]), tag
    assert float(outs[0][1].abs().max()) > 0.0


def test_layout_arguments_are_checked(native):
    from paper_2511_21264_gb300.native import MPPIError
    sc, gm, om, ctl = _controller(native, 2, K=64, H=4)
    for bad in ((12, 0), (16, 2), (64, 0)):
        with pytest.raises(MPPIError):
            ctl.set_layout(*bad)
    with pytest.raises(MPPIError):
        ctl.set_layout(8, 0)    # a 7-link arm does not fit 4 lanes per arm
    ctl.set_layout(16, 1)
    assert ctl.get_layout()[:2] == (16, 1)


def _boxes_under_links(sc, links, half=0.04, pen=0.01):
    """The scene with its first boxes moved under the given (arm, link)
    segments of the home pose: a cube below the link's midpoint, lowered
    until the oracle's capsule-box distance is -pen.  The tilted link meets
    the cube's top edge, so every contact point is unique (a segment
    parallel to a face would make the deepest point a flat minimum, where
    the two sides may pick different points of the minimising interval)."""
    import dataclasses
    f = oracle.Model(sc.to_blob()).fk(sc.x0[:sc.nq])
    bc, bh = np.array(sc.boxes_c), np.array(sc.boxes_h)
    for j, (a, i) in enumerate(links):
        a0, a1 = f["a0"][a, i], f["a1"][a, i]
        mid = 0.5 * (a0 + a1)
        rc = sc.links[a][i].radius
        lo, hi = 0.0, 1.0
        for _ in range(80):   # bisection on the drop of the cube's centre
            dz = 0.5 * (lo + hi)
            if oracle.capsule_box(a0, a1, rc, mid - np.array([0.0, 0.0, dz]), np.full(3, half))[0] < -pen:
                lo = dz
            else:
                hi = dz
        bc[j] = mid - np.array([0.0, 0.0, 0.5 * (lo + hi)])
        bh[j] = half
    return dataclasses.replace(sc, boxes_c=bc, boxes_h=bh)


def test_link_box_contacts_single_step_every_layout(native):
    # capsule-box contacts found through the cull (bounding spheres, overlap,
    # the segment against the box inflated by the capsule radius) and the
    # exact minimum: single steps against the oracle, same bits in every
    # layout, with many link-box contacts among the oracle's contacts
    sc = _boxes_under_links(scenes.config(3), [(0, 2), (0, 4), (1, 3), (1, 5)])
    blob = sc.to_blob()
    gm, om = native.Model(blob), oracle.Model(blob)
    n = 101
    X = _states(sc, om, n, seed=91, q_spread=0.15, v_spread=0.2)
    U1 = _f32(np.random.default_rng(92).normal(scale=0.3, size=(n, sc.nu)))
    ctl = native.Controller(gm, n, 1, sc.lam, sc.sigma_vec(), 9)
    outs = []
    for lps, place in _layouts(3):
        ctl.set_layout(lps, place)
        xs = _t(X)
        ctl.sim_step(xs, _t(U1))
        assert ctl.sync() == 0
        outs.append(xs.cpu().numpy())
    for g in outs[1:]:
        np.testing.assert_array_equal(g, outs[0])
    link_box = 0
    for i in range(n):
        xo, info, lam, cons = om.step(X[i], U1[i], want_contacts=True)
        link_box += sum(1 for c in cons if c["box"] >= 0 and c["bodyA"] < 2 * sc.n_a)
        assert np.abs(outs[0][i] - xo).max() <= 1e-4 * max(1.0, np.abs(xo).max()), i
    assert link_box >= 30, link_box
