"""The bounds-check build: the library compiled with -DMPPI_BOUNDS_CHECK,
in which every index the rollout, update, elite-set and QP kernels use into
shared memory, the staged model and device buffers is compared with its
extent (a failed check sets a bit in a device word and diverts the access;
no trap).  It stands in for a memory checker: small cases (K = 4, H = 2) of
every path on configs 1-3 run through it, match the FP64 oracle, and leave
the word at 0.

The build loads in a child process, because a process holds one libmppi."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
import oracle
from paper_2511_21264_gb300 import native, scenes
native.LIB_PATH = native.BOUNDS_LIB_PATH
import ctypes as C
import torch
L = native.lib()
word, checked = C.c_uint(), C.c_int()

def take():
    assert L.mppi_debug_bounds(C.byref(word), C.byref(checked)) == 0
    return int(word.value)

out = {"checked": None, "words": {}, "cost_err": {}}
take()
out["checked"] = int(checked.value)
f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
T = lambda a: torch.tensor(np.ascontiguousarray(np.asarray(a, np.float32)), device="cuda")
for cfg in (1, 2, 3):
    sc = scenes.config(cfg)
    blob = sc.to_blob()
    gm, om = native.Model(blob), oracle.Model(blob)
    K, H = 4, 2
    ctl = native.Controller(gm, K, H, sc.lam, sc.sigma_vec(), scenes.controller_key(cfg, 2))
    x = T(sc.x0)
    lays = [(32, 0), (16, 1)] + ([(8, 0)] if cfg == 1 else [])
    for lps, pl in lays:
        ctl.set_layout(lps, pl)
        u = torch.zeros((H, sc.nu), device="cuda")
        ctl.step(x, u, u)
        ctl.solve(x, u, 2)
        assert ctl.sync() == 0
    out["words"][f"cfg{cfg}_step"] = take()
    # explicit controls against the oracle (states kept clear of contact switches)
    X, s = [], 7
    while len(X) < K:
        for xs in f32(scenes.random_states(sc, 8, s, q_spread=0.2, v_spread=0.2)):
            if om.min_abs_dist(xs) > 1e-4 and len(X) < K:
                X.append(xs)
        s += 100
    X = np.array(X)
    U = f32(np.random.default_rng(cfg).normal(scale=sc.sigma, size=(K, H, sc.nu)))
    costs = torch.empty(K, device="cuda")
    ctl.set_layout(16, 0)
    ctl.rollout_batch(T(X), T(U), costs)
    xs = T(X)
    ctl.sim_step(xs, T(U[:, 0]))
    assert ctl.sync() == 0
    ref = np.array([om.rollout(X[i], U[i]) for i in range(K)])
    out["cost_err"][f"cfg{cfg}"] = float(np.max(np.abs(costs.cpu().numpy() - ref) / np.abs(ref)))
    out["words"][f"cfg{cfg}_rollout"] = take()
    # the full Eq. 8 update with covariance, then the QP projection
    ctl.set_update(2, 0.7, True, 1e-6)
    u = torch.zeros((H, sc.nu), device="cuda")
    ctl.step(x, u, u)
    ctl.set_projection(scenes.projection_bounds(sc), iters=5)
    ctl.step(x, u, u)
    assert ctl.sync() == 0
    out["words"][f"cfg{cfg}_elite_qp"] = take()
    # the projection's thread kernel (H > 32) and the standalone form
    c2 = native.Controller(gm, K, 40, sc.lam, sc.sigma_vec(), 5)
    c2.set_projection(scenes.projection_bounds(sc), iters=3)
    u2 = torch.zeros((40, sc.nu), device="cuda")
    c2.step(x, u2, u2)
    assert c2.sync() == 0
    out["words"][f"cfg{cfg}_qp_thread"] = take()
# a batch of two controllers
sc = scenes.config(3)
m = native.Model(sc.to_blob())
b = native.Batch([(m, 4, 2, sc.lam, sc.sigma_vec(), 1), (m, 6, 3, sc.lam, sc.sigma_vec(), 2)])
xs = [T(sc.x0), T(sc.x0)]
us = [torch.zeros((2, sc.nu), device="cuda"), torch.zeros((3, sc.nu), device="cuda")]
b.set_layout(16, 1)
b.step(xs, us)
rc, errs = b.sync()
assert rc == 0, errs
out["words"]["batch"] = take()
print(json.dumps(out))
'''


def test_bounds_check_build_runs_clean_on_small_cases():
    from paper_2511_21264_gb300 import native
    native.build(bounds=True)
    p = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT), 1)], capture_output=True,
                       text=True, timeout=900, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-3000:]
    res = json.loads(p.stdout.strip().splitlines()[-1])
    assert res["checked"] == 1                 # the checks are compiled in
    assert all(w == 0 for w in res["words"].values()), res["words"]
    assert all(e <= 1e-3 for e in res["cost_err"].values()), res["cost_err"]
