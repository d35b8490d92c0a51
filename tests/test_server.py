"""Replan server with continuous batching (srv_*): each result is the same
alone and in the mix, admission follows the device-memory budget, requests
can be cancelled, the resident state and warm start advance."""
import numpy as np
import pytest

from paper_2511_21264_gb300 import scenes

torch = pytest.importorskip("torch")


def test_server_rejects_bad_config_without_device_work():
    import ctypes as C
    from paper_2511_21264_gb300 import native
    native.build()
    L = native.lib()
    h = C.c_void_p()
    cfg = native.ServerConfig(0, 1, 1, 0)             # no budget
    assert L.srv_create(C.byref(cfg), C.byref(h)) == 1
    cfg = native.ServerConfig(1 << 20, 0, 1, 0)       # no slots
    assert L.srv_create(C.byref(cfg), C.byref(h)) == 1
    cfg = native.ServerConfig(1 << 20, 4, 0, 0)       # no iterations
    assert L.srv_create(C.byref(cfg), C.byref(h)) == 1


def _scene(i, K=256, H=16):
    return scenes.dh_scene(seed=500 + i, n_boxes=i % 5, K=K, H=H, task="transfer")


@pytest.mark.gpu
def test_result_is_the_same_alone_and_in_the_mix():
    from paper_2511_21264_gb300 import native
    native.build()
    M = 4
    target = _scene(3)
    tm = native.Model(target.to_blob())
    key = scenes.controller_key(3, 0)
    # alone
    s1 = native.Server(1 << 24, 64, M)
    sid = s1.add_scene(tm, target.K, target.H, target.lam, target.sigma_vec(), key)
    s1.start()
    st, done, u_alone, lat = s1.poll(s1.submit(sid), sid, wait_ms=60000)
    assert done and st == 0 and lat > 0
    s1.stop()
    # in a mix of 20 scenes of different K and H, submitted at once: three
    # size classes, whose iterations overlap on their own streams
    s2 = native.Server(1 << 24, 64, M)
    models, ids = [], []
    for i in range(20):
        sc = target if i == 3 else _scene(i, K=[64, 128, 256, 512, 2048][i % 5], H=[8, 16, 24][i % 3])
        m = tm if i == 3 else native.Model(sc.to_blob())
        models.append(m)
        ids.append(s2.add_scene(m, sc.K, sc.H, sc.lam, sc.sigma_vec(), key if i == 3 else scenes.controller_key(i, 0)))
    s2.start()
    tickets = [s2.submit(i) for i in ids]
    outs = [s2.poll(t, i, wait_ms=60000) for t, i in zip(tickets, ids)]
    assert all(o[1] and o[0] == 0 for o in outs)
    np.testing.assert_array_equal(outs[3][2], u_alone)
    assert s2.stats()["mean_active"] > 1.0
    s2.stop()
    # the same mix in one batch (a single size class)
    s3 = native.Server(1 << 24, 64, M, size_classes=1)
    ids3 = []
    for i in range(20):
        sc = target if i == 3 else _scene(i, K=[64, 128, 256, 512, 2048][i % 5], H=[8, 16, 24][i % 3])
        ids3.append(s3.add_scene(models[i], sc.K, sc.H, sc.lam, sc.sigma_vec(),
                                 key if i == 3 else scenes.controller_key(i, 0)))
    s3.start()
    outs3 = [s3.poll(t, i, wait_ms=60000) for t, i in zip([s3.submit(i) for i in ids3], ids3)]
    s3.stop()
    for a, b in zip(outs, outs3):
        np.testing.assert_array_equal(a[2], b[2])
    # and both equal M iterations of the handle path
    ctl = native.Controller(tm, target.K, target.H, target.lam, target.sigma_vec(), key)
    x = torch.tensor(tm.home(), device="cuda")
    u = torch.zeros((target.H, target.nu), device="cuda")
    for _ in range(M):
        ctl.step(x, u, u)
    assert ctl.sync() == 0
    np.testing.assert_array_equal(u.cpu().numpy(), u_alone)


@pytest.mark.gpu
def test_admission_follows_the_memory_budget_and_cancel():
    from paper_2511_21264_gb300 import native
    native.build()
    K = 512
    budget = 2 * K * 4                     # room for two requests' workspaces
    srv = native.Server(budget, 64, 3)
    models = []
    for i in range(6):
        sc = _scene(i, K=K, H=8)
        m = native.Model(sc.to_blob())
        models.append(m)
        srv.add_scene(m, K, 8, sc.lam, sc.sigma_vec(), scenes.controller_key(i, 1))
    # a scene whose single request can never fit is refused at registration
    big = _scene(9, K=4096, H=8)
    bm = native.Model(big.to_blob())
    with pytest.raises(native.MPPIError) as ei:
        srv.add_scene(bm, 4096, 8, big.lam, big.sigma_vec(), 1)
    assert ei.value.code == 6   # MPPI_ERR_ADMISSION
    tickets = [srv.submit(i) for i in range(6)]
    extra = srv.submit(0)      # same scene as the first: waits for it, so it can be cancelled
    assert srv.cancel(extra) == 0
    assert srv.cancel(extra) != 0
    srv.start()
    for t, i in zip(tickets, range(6)):
        st, done, u, lat = srv.poll(t, i, wait_ms=60000)
        assert done and st == 0
    s = srv.stats()
    assert s["completed"] == 6 and s["mean_active"] <= 2.0 and s["admission_waits"] > 0
    srv.stop()


@pytest.mark.gpu
def test_resident_state_and_warm_start_advance():
    from paper_2511_21264_gb300 import native
    native.build()
    sc = _scene(1, K=256, H=8)
    m = native.Model(sc.to_blob())
    srv = native.Server(1 << 22, 8, 2)
    sid = srv.add_scene(m, sc.K, sc.H, sc.lam, sc.sigma_vec(), 7)
    x0 = srv.state(sid)
    srv.start()
    st, done, u1, _ = srv.poll(srv.submit(sid), sid, wait_ms=60000)
    assert done and st == 0
    x1 = srv.state(sid)
    assert np.abs(x1 - x0).max() > 0          # one simulator step under u1[0]
    st, done, u2, _ = srv.poll(srv.submit(sid), sid, wait_ms=60000)
    assert done and st == 0 and not np.array_equal(u1, u2)
    srv.stop()


@pytest.mark.gpu
def test_poisson_load_completes_and_reports_latency():
    from paper_2511_21264_gb300 import native
    native.build()
    srv = native.Server(1 << 24, 32, 2)
    models = []
    for i in range(16):
        sc = _scene(i, K=[128, 256][i % 2], H=[8, 16][i % 2])
        m = native.Model(sc.to_blob())
        models.append(m)
        srv.add_scene(m, sc.K, sc.H, sc.lam, sc.sigma_vec(), scenes.controller_key(i, 2))
    srv.start()
    srv.run_load(200.0, 0.5, seed=1, drain_ms=60000)
    s = srv.stats()
    assert s["completed"] > 20 and s["waiting"] == 0 and s["active"] == 0
    assert s["p99_ms"] >= s["p50_ms"] > 0 and s["sample_steps_per_s"] > 0
    srv.stop()


@pytest.mark.gpu
@pytest.mark.parametrize("qp", [0, 8])
def test_server_full_eq8_and_projection(qp):
    # scenes with the full Eq. 8 (elite set, eta, covariance blocks that carry
    # over between requests) and, with qp, the projection of every request's
    # samples: each result equals the same scene's controller run M
    # iterations per request, bitwise, alone and in a mix of classes
    from paper_2511_21264_gb300 import native
    native.build()
    M = 3
    cfgs = [(256, 16, 32, 0.7, True), (512, 16, 0, 1.0, False), (128, 8, 16, 0.5, True), (2048, 16, 64, 0.8, True)]
    mix = []
    for i, (K, H, ne, eta, cov) in enumerate(cfgs):
        sc = _scene(20 + i, K=K, H=H)
        mix.append((sc, native.Model(sc.to_blob()), K, H, ne, eta, cov, scenes.controller_key(20 + i, 0)))
    srv = native.Server(1 << 26, 16, M, qp_iters=qp)
    ids = []
    for sc, m, K, H, ne, eta, cov, key in mix:
        sid = srv.add_scene(m, K, H, sc.lam, sc.sigma_vec(), key)
        srv.set_scene_update(sid, ne, eta, cov, 1e-6)
        if qp:
            srv.set_scene_projection(sid, scenes.projection_bounds(sc))
        ids.append(sid)
    srv.start()
    plans = []
    for rnd in range(2):   # two requests per scene: the warm start (u_nom, Sigma) carries over
        tickets = [srv.submit(i) for i in ids]
        outs = [srv.poll(t, i, wait_ms=60000) for t, i in zip(tickets, ids)]
        assert all(o[1] and o[0] == 0 for o in outs)
        plans.append([o[2] for o in outs])
    srv.stop()
    for j, (sc, m, K, H, ne, eta, cov, key) in enumerate(mix):
        ctl = native.Controller(m, K, H, sc.lam, sc.sigma_vec(), key)
        ctl.set_update(ne or K, eta, cov, 1e-6)
        if qp:
            ctl.set_projection(scenes.projection_bounds(sc), iters=qp)
        x = torch.tensor(m.home(), device="cuda")
        u = torch.zeros((H, sc.nu), device="cuda")
        for rnd in range(2):
            for _ in range(M):
                ctl.step(x, u, u)
            assert ctl.sync() == 0
            np.testing.assert_array_equal(u.cpu().numpy(), plans[rnd][j], err_msg=f"scene {j} request {rnd}")
            # the server executes u_nom[0] and shifts the warm start
            x1 = x[None].clone()
            ctl.sim_step(x1, u[:1].contiguous())
            x = x1[0].clone()
            u = torch.cat([u[1:], u[-1:]], 0).contiguous()
