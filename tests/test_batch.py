"""Batched controllers (mppi_batch_*): each instance's update is bitwise the
one mppi_step computes for it alone, under every launch shape, eagerly and
from the captured graph; the autotuner's table persists."""
import os

import numpy as np
import pytest

from paper_2511_21264_gb300 import scenes


def test_tune_table_store_and_lookup(tmp_path, monkeypatch):
    import ctypes as C
    from paper_2511_21264_gb300 import native
    native.build()
    L = native.lib()
    path = tmp_path / "sub" / "tune.txt"
    monkeypatch.setenv("MPPI_TUNE_FILE", str(path))
    s, o, lp, pl = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    look = lambda k: L.mppi_tune_lookup(k, C.byref(s), C.byref(o), C.byref(lp), C.byref(pl))
    assert look(b"nv20_nb8_n4_K100_H16") != 0
    assert L.mppi_tune_store(b"nv20_nb8_n4_K100_H16", 4, 1, 32, 0, C.c_float(1.5)) == 0
    assert L.mppi_tune_store(b"other", 2, 0, 16, 1, C.c_float(0.5)) == 0
    assert L.mppi_tune_store(b"nv20_nb8_n4_K100_H16", 8, 0, 16, 1, C.c_float(1.2)) == 0  # later entry wins
    assert look(b"nv20_nb8_n4_K100_H16") == 0
    assert (s.value, o.value, lp.value, pl.value) == (8, 0, 16, 1)
    assert L.mppi_tune_store(b"bad key", 4, 1, 32, 0, C.c_float(1.0)) == 1
    assert L.mppi_tune_store(b"k", 0, 1, 32, 0, C.c_float(1.0)) == 1
    assert L.mppi_tune_store(b"k", 4, 1, 12, 0, C.c_float(1.0)) == 1
    assert L.mppi_tune_store(b"k", 4, 1, 16, 2, C.c_float(1.0)) == 1
    assert len(path.read_text().splitlines()) == 3


def _instances(native, seeds=(0, 1, 2, 3, 4, 5)):
    """Uneven K, H and box counts, 7-DoF arms."""
    Ks = [64, 200, 257, 96, 33, 130]
    Hs = [8, 16, 12, 8, 20, 16]
    boxes = [0, 4, 8, 2, 16, 1]
    out = []
    for i, s in enumerate(seeds):
        sc = scenes.dh_scene(seed=100 + s, n_boxes=boxes[i], K=Ks[i], H=Hs[i], task="transfer")
        m = native.Model(sc.to_blob())
        out.append((sc, m, Ks[i], Hs[i], sc.lam, sc.sigma_vec(), scenes.controller_key(100 + s, i)))
    return out


@pytest.mark.gpu
def test_batch_matches_single_controllers_bitwise_under_every_shape(tmp_path, monkeypatch):
    import torch
    from paper_2511_21264_gb300 import native
    monkeypatch.setenv("MPPI_TUNE_FILE", str(tmp_path / "tune.txt"))
    native.build()
    inst = _instances(native)
    # reference: each controller alone, two iterations
    ref = []
    for sc, m, K, H, lam, sig, key in inst:
        ctl = native.Controller(m, K, H, lam, sig, key)
        x = torch.tensor(m.home(), device="cuda")
        u = torch.zeros((H, sc.nu), device="cuda")
        ctl.step(x, u, u)
        ctl.step(x, u, u)
        assert ctl.sync() == 0
        ref.append(u.clone())
    b = native.Batch([(m, K, H, lam, sig, key) for sc, m, K, H, lam, sig, key in inst])
    xs = [torch.tensor(m.home(), device="cuda") for sc, m, *_ in inst]
    for lps, place in ((32, 0), (32, 1), (16, 0), (16, 1)):
        b.set_layout(lps, place)
        for spc in (1, 2, 4, 8):
            for order in (0, 1):
                b.set_launch(spc, order)
                b.set_iteration(-1, 0)
                us = [torch.zeros((H, sc.nu), device="cuda") for sc, m, K, H, *_ in inst]
                b.step(xs, us)
                b.step(xs, us)
                rc, errs = b.sync()
                assert rc == 0, errs
                for i in range(len(inst)):
                    assert torch.equal(us[i], ref[i]), (lps, place, spc, order, i)
                    assert b.iteration(i) == 2


@pytest.mark.gpu
def test_batch_graph_replay_and_autotune(tmp_path, monkeypatch):
    import torch
    from paper_2511_21264_gb300 import native
    monkeypatch.setenv("MPPI_TUNE_FILE", str(tmp_path / "tune.txt"))
    native.build()
    inst = _instances(native)
    b = native.Batch([(m, K, H, lam, sig, key) for sc, m, K, H, lam, sig, key in inst])
    xs = [torch.tensor(m.home(), device="cuda") for sc, m, *_ in inst]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ue = [torch.zeros((H, sc.nu), device="cuda") for sc, m, K, H, *_ in inst]
        for _ in range(3):
            b.step(xs, ue, stream=s)
        b.set_iteration(-1, 0, stream=s)
        ug = [torch.zeros((H, sc.nu), device="cuda") for sc, m, K, H, *_ in inst]
        for _ in range(3):
            b.step(xs, ug, stream=s, graph=True)
        rc, _ = b.sync(stream=s)
        assert rc == 0
        for a, c in zip(ue, ug):
            assert torch.equal(a, c)
        # autotune on scratch copies; counters are restored
        scratch = [u.clone() for u in ug]
        ms = b.autotune(xs, scratch, reps=2, stream=s)
        assert ms > 0
        assert all(b.iteration(i, stream=s) == 3 for i in range(len(inst)))
    text = (tmp_path / "tune.txt").read_text().split()
    assert text[0].startswith("nv20_") and int(text[1]) in (1, 2, 4, 8, 16) and int(text[2]) in (0, 1)
    assert int(text[3]) in (16, 32) and int(text[4]) in (0, 1)
    # a new batch with the same key picks the stored shape up
    b2 = native.Batch([(m, K, H, lam, sig, key) for sc, m, K, H, lam, sig, key in inst])
    assert b2.get_launch() == (int(text[1]), int(text[2]))
    assert b2.get_layout() == (int(text[3]), int(text[4]))


@pytest.mark.gpu
@pytest.mark.parametrize("proj", [False, True])
def test_batch_full_eq8_and_projection_match_single_controllers(tmp_path, monkeypatch, proj):
    # instances with the elite set, a learning rate and covariance blocks
    # (and, with proj, the QP projection of every sample) give bitwise the
    # iterations a single controller with the same settings gives
    import torch
    from paper_2511_21264_gb300 import native
    monkeypatch.setenv("MPPI_TUNE_FILE", str(tmp_path / "tune.txt"))
    native.build()
    inst = _instances(native)
    settings = [(16, 0.7, True), (0, 1.0, False), (40, 0.5, True), (8, 1.0, False), (10, 0.8, True), (0, 0.6, False)]
    bounds = [scenes.projection_bounds(sc) for sc, *_ in inst]
    ref = []
    for (sc, m, K, H, lam, sig, key), (ne, eta, cov) in zip(inst, settings):
        ctl = native.Controller(m, K, H, lam, sig, key)
        ctl.set_update(ne or K, eta, cov, 1e-6)
        if proj:
            ctl.set_projection(scenes.projection_bounds(sc), iters=10)
        x = torch.tensor(m.home(), device="cuda")
        u = torch.zeros((H, sc.nu), device="cuda")
        for _ in range(3):
            ctl.step(x, u, u)
        assert ctl.sync() == 0
        ref.append(u.clone())
    xs = [torch.tensor(m.home(), device="cuda") for sc, m, *_ in inst]
    s = torch.cuda.Stream()
    for lps, graph in ((32, False), (16, True)):
        # a fresh batch per pass: the covariance blocks start from diag(sigma^2)
        b = native.Batch([(m, K, H, lam, sig, key) for sc, m, K, H, lam, sig, key in inst])
        for i, (ne, eta, cov) in enumerate(settings):
            b.set_update(i, ne, eta, cov, 1e-6)
        if proj:
            b.set_projection(np.stack(bounds), iters=10)
        b.set_layout(lps, 0)
        us = [torch.zeros((H, sc.nu), device="cuda") for sc, m, K, H, *_ in inst]
        with torch.cuda.stream(s):
            for _ in range(3):
                b.step(xs, us, stream=s, graph=graph)
        rc, errs = b.sync(stream=s)
        assert rc == 0, errs
        for i in range(len(inst)):
            assert torch.equal(us[i], ref[i]), (lps, graph, i)
        b.close()
