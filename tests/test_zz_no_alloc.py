"""mppi_step_noalloc: one MPPI iteration for callers that cannot allocate
device memory (a control loop that must not call cudaMalloc once it runs, or
code inside a framework that owns the GPU's memory budget).  Its scratch is a
static device array in the library.

Checked against the handle-based entry point (mppi_step) on two calls in a
row: same scene, seed and iteration counter, so the same samples; the
updated nominal controls must agree within the tolerance the parity tests
use for the control update (1e-3; the kernels are the same, so the match is
in fact exact).  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from paper_2511_21264_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_noalloc_step_matches_handle_step_on_two_calls():
    from paper_2511_21264_gb300 import native
    native.build()
    L = native.lib()
    sc = scenes.config(2)
    K, H = 512, 16
    blob = sc.to_blob()
    sigma = sc.sigma_vec().astype(np.float32)
    seed = scenes.controller_key(7, 3)
    model = native.Model(blob)
    ctl = native.Controller(model, K, H, sc.lam, sigma, seed)
    x = torch.tensor(model.home(), device="cuda")
    u_ref = torch.zeros((H, sc.nu), device="cuda")
    u_na = torch.zeros((H, sc.nu), device="cuda")
    out_ref = torch.empty_like(u_ref)
    out_na = torch.empty_like(u_na)
    buf = C.create_string_buffer(blob, len(blob))
    sig = np.ascontiguousarray(sigma)
    stream = torch.cuda.current_stream().cuda_stream or None
    for it in range(2):
        ctl.step(x, u_ref, out_ref)                      # handle path, counter = it
        status = C.c_int(-1)
        rc = L.mppi_step_noalloc(buf, len(blob), K, H, C.c_float(sc.lam), sig.ctypes.data, C.c_uint64(seed),
                                 C.c_uint64(it), x.data_ptr(), u_na.data_ptr(), out_na.data_ptr(),
                                 C.byref(status), stream)
        assert rc == 0 and status.value == 0
        assert ctl.sync() == 0
        np.testing.assert_allclose(out_na.cpu().numpy(), out_ref.cpu().numpy(), atol=1e-3, rtol=0)
        assert float(out_na.abs().max()) > 0
        u_ref.copy_(out_ref)
        u_na.copy_(out_na)


def test_noalloc_rejects_sizes_beyond_the_maximum():
    from paper_2511_21264_gb300 import native
    native.build()
    L = native.lib()
    sc = scenes.config(1)
    blob = sc.to_blob()
    buf = C.create_string_buffer(blob, len(blob))
    sig = np.ascontiguousarray(sc.sigma_vec().astype(np.float32))
    x = torch.zeros(sc.nq + sc.nv, device="cuda")
    u = torch.zeros((4, sc.nu), device="cuda")
    too_many = 8192 + 1
    rc = L.mppi_step_noalloc(buf, len(blob), too_many, 4, C.c_float(0.1), sig.ctypes.data, C.c_uint64(1),
                             C.c_uint64(0), x.data_ptr(), u.data_ptr(), u.data_ptr(), None, None)
    assert rc == 1   # MPPI_ERR_INVALID_ARG
