"""GPU (C ABI) against the FP64 oracle, element by element.

Tolerances (stated for this path):
  single simulator step        max |dx| <= 1e-4 * max(1, |x|_inf) per state
  sample cost over H <= 8      |dc| <= 1e-3 |c|
  weighted control update      max |du| <= 1e-3
  Philox words                 bit-exact
  Gaussian noise               |d eps| <= 2e-6 (FP32 log/sin vs FP64)
Inputs are rounded to float32 first and the oracle takes exactly those
values.  Parity scenes keep every contact distance at least 1e-5 away from
zero along the compared steps, because an FP32/FP64 difference can flip a
contact's activation there (a reading stated with the design)."""
import os

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


def _t(a, dtype=np.float32):
    return torch.tensor(np.ascontiguousarray(np.asarray(a, dtype)), device=DEV)


def _f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def _parity_states(sc, om, n, seed, min_gap=1e-4, **kw):
    out, s = [], seed
    while len(out) < n:
        for x in _f32(scenes.random_states(sc, 2 * n, s, **kw)):
            if om.min_abs_dist(x) > min_gap:
                out.append(x)
                if len(out) == n:
                    break
        s += 1000
    return np.array(out)


def _setup(cfg, K, H, seed=None, sigma=None, lam=None):
    from paper_2511_21264_gb300 import native as nat
    sc = scenes.config(cfg)
    blob = sc.to_blob()
    gm = nat.Model(blob)
    om = oracle.Model(blob)
    sig = sc.sigma_vec() if sigma is None else sigma
    key = scenes.controller_key(cfg, 1) if seed is None else seed
    ctl = nat.Controller(gm, K, H, sc.lam if lam is None else lam, sig, key)
    return sc, gm, om, ctl, key


# ------------------------------------------------------------------ random
def test_philox_words_bit_exact(native):
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(1000, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    key = 0x299F31D0A4093822
    out = torch.empty((1000, 4), dtype=torch.int32, device=DEV)
    native.debug_philox(_t(ctr.view(np.int32), np.int32), key, out)
    got = out.cpu().numpy().view(np.uint32)
    for i in range(0, 1000, 7):
        assert list(got[i]) == oracle.philox4x32_10(ctr[i], [key & 0xFFFFFFFF, key >> 32])
    # published answer for counter 0 / key 0
    z = torch.zeros((1, 4), dtype=torch.int32, device=DEV)
    o = torch.empty_like(z)
    native.debug_philox(z, 0, o)
    assert [int(v) for v in o.cpu().numpy().view(np.uint32)[0]] == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]


@pytest.mark.parametrize("cfg", [1, 2])
def test_noise_matches_oracle(native, cfg):
    sc, gm, om, ctl, key = _setup(cfg, K=37, H=5)
    eps = torch.empty((37, 5, sc.nu), device=DEV)
    ctl.debug_noise(3, eps)
    ref = oracle.noise(key, 3, 37, 5, sc.nu, _f32(sc.sigma_vec()))
    np.testing.assert_allclose(eps.cpu().numpy(), ref, atol=2e-6, rtol=0)


# ------------------------------------------------------------- simulator
@pytest.mark.parametrize("cfg", [1, 2, 3])
def test_single_step_parity(native, cfg):
    n = 101  # several CTAs and a ragged tail
    sc, gm, om, ctl, _ = _setup(cfg, K=n, H=1)
    X = _parity_states(sc, om, n, seed=cfg)
    rng = np.random.default_rng(cfg)
    U1 = _f32(rng.normal(scale=0.5, size=(n, sc.nu)))
    xs = _t(X)
    ctl.sim_step(xs, _t(U1))
    assert ctl.sync() == 0
    G = xs.cpu().numpy().astype(np.float64)
    ncon = []
    for i in range(n):
        xo, info = om.step(X[i], U1[i])
        ncon.append(info.ncon)
        err = np.abs(G[i] - xo).max() / max(1.0, np.abs(xo).max())
        assert err <= 1e-4, (i, err, info.ncon)
    assert max(ncon) >= 2          # contacts were exercised
    assert np.mean(np.array(ncon) > 0) > 0.5


def test_fast_ball_spin_rotation_step(native):
    # the ball's rotation step is a Taylor series below |w| dt / 2 = 1/2 and
    # the sine/cosine form above it: spins from 10 to 300 rad/s about random
    # axes, ball lifted clear of every contact, against the oracle's step
    n = 64
    sc, gm, om, ctl, _ = _setup(2, K=n, H=1)
    X = scenes.random_states(sc, n, seed=7, ball_lift=3.0)
    rng = np.random.default_rng(7)
    axis = rng.normal(size=(n, 3))
    axis /= np.linalg.norm(axis, axis=1, keepdims=True)
    speed = np.geomspace(10.0, 300.0, n)
    w0 = sc.nq + 2 * sc.n_a + 3
    X[:, w0:w0 + 3] = axis * speed[:, None]
    X = _f32(X)
    half = speed * sc.dt / 2
    assert (half < 0.5).any() and (half >= 0.5).any()
    U1 = np.zeros((n, sc.nu))
    xs = _t(X)
    ctl.sim_step(xs, _t(U1))
    assert ctl.sync() == 0
    G = xs.cpu().numpy().astype(np.float64)
    q0 = 2 * sc.n_a + 3
    for i in range(n):
        xo, info = om.step(X[i], U1[i])
        assert info.ncon == 0
        assert np.abs(G[i, q0:q0 + 4] - xo[q0:q0 + 4]).max() <= 1e-5, (i, speed[i])
        assert np.abs(G[i] - xo).max() <= 1e-4 * max(1.0, np.abs(xo).max()), (i, speed[i])


def _traj_ok(om, x, U, gap=1e-5):
    c, T = om.rollout(x, U, traj=True)
    return all(om.min_abs_dist(T[h]) > gap for h in range(T.shape[0] - 1)), c, T


@pytest.mark.parametrize("cfg", [1, 2, 3])
def test_rollout_cost_parity_h8(native, cfg):
    n, H = 67, 8
    sc, gm, om, ctl, _ = _setup(cfg, K=n, H=H)
    X = _parity_states(sc, om, n, seed=10 + cfg, q_spread=0.2, v_spread=0.2)
    rng = np.random.default_rng(20 + cfg)
    U = _f32(rng.normal(scale=sc.sigma, size=(n, H, sc.nu)))
    costs = torch.empty(n, device=DEV)
    xo = torch.empty((n, sc.nq + sc.nv), device=DEV)
    ctl.rollout_batch(_t(X), _t(U), costs, xo)
    assert ctl.sync() == 0
    gc = costs.cpu().numpy()
    gx = xo.cpu().numpy()
    kept = 0
    for i in range(n):
        ok, c, T = _traj_ok(om, X[i], U[i])
        if not ok:
            continue
        kept += 1
        assert abs(gc[i] - c) <= 1e-3 * abs(c), (i, gc[i], c)
        assert np.abs(gx[i] - T[-1]).max() <= 1e-3 * max(1.0, np.abs(T[-1]).max())
    assert kept >= 0.8 * n


# ----------------------------------------------------------------- update
@pytest.mark.parametrize("cfg", [1, 2])
def test_update_parity(native, cfg):
    K, H = 257, 6
    sc, gm, om, ctl, key = _setup(cfg, K=K, H=H)
    rng = np.random.default_rng(cfg)
    costs = _f32(rng.uniform(10.0, 10.5, K))
    u_nom = _f32(rng.normal(scale=0.2, size=(H, sc.nu)))
    out = torch.empty((H, sc.nu), device=DEV)
    ctl.update(_t(costs), _t(u_nom), out)
    assert ctl.sync() == 0
    eps = oracle.noise(key, 0, K, H, sc.nu, _f32(sc.sigma_vec()))
    ref, w, st = oracle.mppi_update(costs, u_nom[None] + eps, sc.lam, u_nom)
    assert st == 0
    np.testing.assert_allclose(out.cpu().numpy(), ref, atol=1e-3, rtol=0)
    # sharper: the FP32 path agrees to ~1e-6 here
    assert np.abs(out.cpu().numpy() - ref).max() < 2e-5


def test_update_all_nonfinite_keeps_nominal(native):
    sc, gm, om, ctl, key = _setup(1, K=32, H=4)
    u_nom = _t(np.arange(4 * sc.nu).reshape(4, sc.nu) * 0.01)
    out = torch.empty_like(u_nom)
    ctl.update(_t(np.full(32, np.nan)), u_nom, out)
    assert ctl.sync() == 4   # MPPI_ERR_NONFINITE
    assert torch.equal(out, u_nom)
    # non-finite costs get zero weight when others are finite
    c = np.full(32, np.inf)
    c[5] = 1.0
    ctl.update(_t(c), u_nom, out)
    assert ctl.sync() == 0
    eps = torch.empty((32, 4, sc.nu), device=DEV)
    ctl.debug_noise(0, eps)
    np.testing.assert_allclose(out.cpu().numpy(), (u_nom + eps[5]).cpu().numpy(), atol=1e-6)


def test_lq_update_through_gpu_update_path(native):
    """Eq. 8a on x_{h+1} = x_h + dt u_h with host-computed LQ costs: the GPU
    update of the first control matches the tilted-Gaussian mean."""
    H, sigma, lam, K = 4, 0.5, 2.0, 1 << 17
    sc, gm, om, ctl, key = _setup(1, K=K, H=H, sigma=np.full(6, sigma), lam=lam)
    eps = torch.empty((K, H, sc.nu), device=DEV)
    ctl.debug_noise(0, eps)
    e = eps[..., 0].double().cpu().numpy()
    u_nom = np.zeros((H, sc.nu))
    u_nom[:, 0] = (0.2, -0.1, 0.0, 0.3)
    U0 = u_nom[None, :, 0] + e
    dt, q, r = 0.1, 1.0, 0.1
    S = dt * np.tril(np.ones((H, H)))
    Q = q * S.T @ S + r * np.eye(H)
    b = q * S.T @ np.ones(H)
    costs = np.einsum("ki,ij,kj->k", U0, Q, U0) + 2 * U0 @ b + q * H
    out = torch.empty((H, sc.nu), device=DEV)
    ctl.update(_t(costs), _t(u_nom), out)
    assert ctl.sync() == 0
    Si = np.eye(H) / sigma ** 2
    expect = np.linalg.solve(Si + 2 * Q / lam, Si @ u_nom[:, 0] - 2 * b / lam)
    w = np.exp(-(costs - costs.min()) / lam)
    k_eff = w.sum() ** 2 / (w ** 2).sum()
    se = np.sqrt(np.diag(np.linalg.inv(Si + 2 * Q / lam)) / k_eff)
    assert np.all(np.abs(out.cpu().numpy()[:, 0] - expect) < 5 * se)


# ------------------------------------------------------------- full step
def test_mppi_step_parity_planar(native):
    K, H = 64, 8
    sc, gm, om, ctl, key = _setup(1, K=K, H=H)
    x = _f32(sc.x0)
    u0 = np.zeros((H, sc.nu))
    u = _t(u0)
    out = torch.empty_like(u)
    ctl.step(_t(x), u, out)
    assert ctl.sync() == 0
    assert ctl.iteration() == 1
    ref = om.mppi_iteration(x, u0, K, sc.lam, _f32(sc.sigma_vec()), key, 0)
    np.testing.assert_allclose(out.cpu().numpy(), ref["u_nom"], atol=1e-3, rtol=0)


@pytest.mark.parametrize("cfg,lift", [(1, 0.03), (3, 0.0)])
def test_profile_contact_counts_match_oracle_rollouts(native, cfg, lift):
    # mppi_profile's device counts against the oracle's rollouts of the same
    # Philox samples: active contacts per sample-step, and the steps whose
    # only contact is the ball against static geometry (the lone-contact
    # solve).  The start states mix steps with no contact, a lone ball
    # contact and arm contacts.  Contact activation at |distance| ~ 0 may
    # differ between FP32 and FP64, so the means agree to 2% of the steps.
    K, H = 64, 16
    sc, gm, om, ctl, key = _setup(cfg, K=K, H=H)
    x = _f32(scenes.random_states(sc, 1, 1, ball_lift=lift)[0])
    u0 = np.zeros((H, sc.nu))
    ctl.profile(1)
    out = _t(u0)
    ctl.step(_t(x), _t(u0), out)
    assert ctl.sync() == 0
    kt = ctl.profile_read()
    ctl.profile(0)
    U = om.mppi_iteration(x, u0, K, sc.lam, _f32(sc.sigma_vec()), key, 0, want_samples=True)["U"]
    ball = 2 * sc.n_a
    con = lone = 0
    for k in range(K):
        xk = x
        for h in range(H):
            xk, info, lam, cl = om.step(xk, U[k, h], want_contacts=True)
            con += info.ncon
            lone += int(info.ncon == 1 and cl[0]["bodyA"] == ball and cl[0]["bodyB"] == -1)
    assert kt["iterations"] == 1
    assert abs(kt["contacts_per_step"] - con / (K * H)) <= 0.02, (kt, con / (K * H))
    assert abs(kt["lone_ball_per_step"] - lone / (K * H)) <= 0.02, (kt, lone / (K * H))
    assert 0.2 < lone / (K * H) < 0.8  # both kinds of step occur
    assert kt["lone_ball_per_step"] <= kt["contacts_per_step"] + 1e-12


def test_step_aliasing_and_graph_replay_are_deterministic(native):
    K, H = 96, 8
    sc, gm, om, ctl, key = _setup(2, K=K, H=H)
    x = _t(_f32(sc.x0))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        u1 = torch.zeros((H, sc.nu), device=DEV)
        for _ in range(3):
            ctl.step(x, u1, u1, stream=s)        # in place (aliased)
        ctl.set_iteration(0, stream=s)
        u2 = torch.zeros((H, sc.nu), device=DEV)
        ctl.solve(x, u2, 3, stream=s)           # captured graph
        ctl.set_iteration(0, stream=s)
        u3 = torch.zeros((H, sc.nu), device=DEV)
        ctl.solve(x, u3, 3, stream=s)           # graph replay
        assert ctl.iteration(stream=s) == 3
    s.synchronize()
    assert torch.equal(u1, u2) and torch.equal(u2, u3)
    assert float(u1.abs().max()) > 0


def test_step_with_host_buffers_matches_device_step(native):
    # mppi_step_host (host arrays, staged copies) against mppi_step on device
    # buffers: the same iterations, bitwise, also in place
    K, H = 256, 16
    sc, gm, om, ctl, key = _setup(2, K=K, H=H)
    x = np.asarray(sc.x0, np.float32)
    ud = torch.zeros((H, sc.nu), device=DEV)
    for _ in range(3):
        ctl.step(_t(x), ud, ud)
    assert ctl.sync() == 0
    ctl.set_iteration(0)
    uh = np.zeros((H, sc.nu), np.float32)
    uh = ctl.step_host(x, uh)
    ctl.step_host(x, uh, uh)
    ctl.step_host(x, uh, uh)
    assert ctl.sync() == 0
    np.testing.assert_array_equal(uh, ud.cpu().numpy())
    assert ctl.iteration() == 3


def test_launch_shape_does_not_change_results(native):
    # one sample per CTA (the default below 8 x the SM count, plain launches)
    # and 2, 4 or 16 samples per CTA (programmatic dependent launches), one or
    # two samples per warp: the same iterations, bitwise, eager and from the
    # captured graph
    K, H = 1024, 32
    sc, gm, om, ctl, key = _setup(2, K=K, H=H)
    x = _t(_f32(sc.x0))
    s = torch.cuda.Stream()
    outs = []
    with torch.cuda.stream(s):
        for lps, spc in ((32, 0), (32, 1), (32, 2), (32, 4), (32, 16), (16, 2), (16, 8), (16, 16)):
            ctl.set_layout(lps, 0)
            ctl.set_launch(spc)
            for graph in (False, True):
                ctl.set_iteration(0, stream=s)
                u = torch.zeros((H, sc.nu), device=DEV)
                if graph:
                    ctl.solve(x, u, 3, stream=s)
                else:
                    for _ in range(3):
                        ctl.step(x, u, u, stream=s)
                outs.append(u)
        assert ctl.sync(stream=s) == 0
    s.synchronize()
    assert all(torch.equal(outs[0], o) for o in outs[1:])
    assert float(outs[0].abs().max()) > 0.0
    # a shape whose workspaces exceed one CTA's shared memory is refused
    from paper_2511_21264_gb300.native import MPPIError
    ctl.set_layout(16, 0)
    ctl.set_launch(32)
    with pytest.raises(MPPIError):
        ctl.step(x, u, u)


def test_edge_cases(native):
    sc, gm, om, ctl, key = _setup(1, K=1, H=3)
    # K = 1: the update returns the single sample
    u = torch.zeros((3, sc.nu), device=DEV)
    out = torch.empty_like(u)
    ctl.step(_t(_f32(sc.x0)), u, out)
    assert ctl.sync() == 0
    eps = torch.empty((1, 3, sc.nu), device=DEV)
    ctl.debug_noise(0, eps)
    np.testing.assert_allclose(out.cpu().numpy(), eps[0].cpu().numpy(), atol=1e-6)
    # empty rollout is a no-op; n > K is rejected
    from paper_2511_21264_gb300.native import MPPIError
    e = torch.empty((0, sc.nq + sc.nv), device=DEV)
    ctl.rollout_batch(e, torch.empty((0, 3, sc.nu), device=DEV), torch.empty(0, device=DEV))
    with pytest.raises(MPPIError):
        ctl.rollout_batch(torch.zeros((2, sc.nq + sc.nv), device=DEV), torch.zeros((2, 3, sc.nu), device=DEV),
                          torch.zeros(2, device=DEV))
    # a non-finite state is reported
    bad = _f32(sc.x0)
    bad[sc.nq] = np.nan
    c = torch.empty(1, device=DEV)
    ctl.rollout_batch(_t(bad[None]), torch.zeros((1, 3, sc.nu), device=DEV), c)
    assert ctl.sync() == 4


# ------------------------------------------------ full-size (bench) shapes
@pytest.mark.parametrize("cfg", [2, 3])
def test_full_size_sampled_and_properties(native, cfg):
    sc = scenes.config(cfg)
    K, H = sc.K, sc.H
    sc, gm, om, ctl, key = _setup(cfg, K=K, H=H)
    x = _t(_f32(sc.x0))
    u0 = np.zeros((H, sc.nu), np.float32)
    u = _t(u0)
    out = torch.empty_like(u)
    # noise: sampled entries against the oracle
    eps = torch.empty((K, H, sc.nu), device=DEV)
    ctl.debug_noise(0, eps)
    rng = np.random.default_rng(cfg)
    ks = rng.choice(K, 6, replace=False)
    ref = oracle.noise(key, 0, K, H, sc.nu, _f32(sc.sigma_vec()))
    np.testing.assert_allclose(eps.cpu().numpy()[ks], ref[ks], atol=2e-6)
    # one iteration; its costs equal rollout_batch of the same samples, and
    # its update equals mppi_update on those costs (bitwise)
    ctl.step(x, u, out)
    assert ctl.sync() == 0
    U = (u[None] + eps).contiguous()
    costs = torch.empty(K, device=DEV)
    ctl.rollout_batch(x.expand(K, -1).contiguous(), U, costs)
    out2 = torch.empty_like(u)
    ctl.set_iteration(0)
    ctl.update(costs, u, out2)
    assert ctl.sync() == 0
    assert torch.equal(out, out2)
    # the update is a convex combination of the samples
    lo, hi = U.min(0).values, U.max(0).values
    assert bool(((out >= lo) & (out <= hi)).all())
    # sampled per-sample costs over the first 8 steps against the oracle
    ctl8 = __import__("paper_2511_21264_gb300.native", fromlist=["x"]).Controller(gm, K, 8, sc.lam,
                                                                                  sc.sigma_vec(), key)
    c8 = torch.empty(K, device=DEV)
    ctl8.rollout_batch(x.expand(K, -1).contiguous(), U[:, :8].contiguous(), c8)
    assert ctl8.sync() == 0
    Uh = U[:, :8].cpu().numpy().astype(np.float64)
    checked = 0
    for k in ks:
        ok, c, _ = _traj_ok(om, _f32(sc.x0), Uh[k])
        if ok:
            checked += 1
            assert abs(float(c8[k]) - c) <= 1e-3 * abs(c)
    assert checked >= 4


# ------------------------------------------------------- statistical parity
@pytest.mark.parametrize("cfg,K,H,iters,lps", [(1, 64, 20, 10, 0), (2, 128, 32, 5, 0), (3, 64, 16, 5, 16)])
def test_statistical_parity_100_seeds(native, cfg, K, H, iters, lps):
    """Longer contact rollouts are compared statistically: final nominal cost
    after `iters` MPPI iterations from the home state, 100 controller seeds,
    GPU vs oracle (two-sample KS) and the improvement rate over zero controls
    (two proportions).  Config 1 at its own K, H and iteration count; the
    7-DoF lift at K = 128 (the oracle's share of the test stays in seconds)
    and its full horizon H = 32, where the rollouts are long and chaotic; the
    8-box transfer at K = 64, H = 16 on the 16-lane layout its full size
    runs on."""
    from scipy import stats
    sc = scenes.config(cfg)
    blob = sc.to_blob()
    from paper_2511_21264_gb300 import native as nat
    gm = nat.Model(blob)
    om = oracle.Model(blob)
    x = _f32(sc.x0)
    sig = _f32(sc.sigma_vec())
    zero = om.rollout(x, np.zeros((H, sc.nu)))
    g_final, o_final = [], []
    nthreads = max(1, min(16, os.cpu_count() or 1))
    eval_ctl = nat.Controller(gm, 1, H, sc.lam, sig, 0)
    for s in range(100):
        key = scenes.controller_key(1000 * cfg + s, 0)
        ctl = nat.Controller(gm, K, H, sc.lam, sig, key)
        if lps:
            ctl.set_layout(lps, 0)
        u = torch.zeros((H, sc.nu), device=DEV)
        for _ in range(iters):
            ctl.step(_t(x), u, u)
        c = torch.empty(1, device=DEV)
        eval_ctl.rollout_batch(_t(x[None]), u[None].contiguous(), c)
        g_final.append(float(c[0]))
        uo = np.zeros((H, sc.nu))
        for it in range(iters):
            uo = om.mppi_iteration(x, uo, K, sc.lam, sig, key, it, nthreads=nthreads)["u_nom"]
        o_final.append(om.rollout(x, uo))
    g_final, o_final = np.array(g_final), np.array(o_final)
    assert stats.ks_2samp(g_final, o_final).pvalue > 0.01
    pg, po = np.mean(g_final < zero), np.mean(o_final < zero)
    p = 0.5 * (pg + po)
    if 0 < p < 1:
        zstat = (pg - po) / np.sqrt(2 * p * (1 - p) / 100)
        assert abs(zstat) < 2.58


# ------------------------------------------------------- checkpoint / resume
def test_checkpoint_resume_reproduces_iterations_bitwise(native):
    """Snapshot (state, u_nom, Philox key, iteration counter); restoring it
    reproduces the next iterations bitwise (warm start, Sec. III-A)."""
    sc, gm, om, ctl, key = _setup(2, K=128, H=8)
    x = _t(_f32(sc.x0))
    u = torch.zeros((8, sc.nu), device=DEV)
    for _ in range(2):
        ctl.step(x, u, u)
    snap_u, snap_it = u.clone(), ctl.iteration()
    for _ in range(3):
        ctl.step(x, u, u)
    first = u.clone()
    ctl2 = __import__("paper_2511_21264_gb300.native", fromlist=["x"]).Controller(gm, 128, 8, sc.lam,
                                                                                   sc.sigma_vec(), key)
    ctl2.set_iteration(snap_it)
    u2 = snap_u.clone()
    for _ in range(3):
        ctl2.step(x, u2, u2)
    assert ctl.sync() == 0 and ctl2.sync() == 0
    assert torch.equal(first, u2)
