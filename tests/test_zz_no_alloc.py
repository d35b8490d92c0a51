"""mppi_step_noalloc: one MPPI iteration for callers that cannot allocate
device memory (a control loop that must not call cudaMalloc once it runs, or
code inside a framework that owns the GPU's memory budget).  Its scratch is a
static device array in the library.

Checked against the handle-based entry point (mppi_step) on two calls in a
row: same scene, seed and iteration counter, so the same samples; the
updated nominal controls must agree within the tolerance the parity tests
use for the control update (1e-3; the kernels are the same, so the match is
in fact exact).  A warm call must leave the device's free memory unchanged,
and u_nom_out may alias u_nom.  This file is collected last on purpose."""
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


def test_noalloc_warm_call_allocates_nothing_and_may_alias():
    # After a warm call, a second call leaves the device's free memory
    # unchanged, and u_nom_out may be u_nom itself.
    from paper_2511_21264_gb300 import native
    native.build()
    L = native.lib()
    sc = scenes.config(1)
    K, H = 256, 12
    blob = sc.to_blob()
    buf = C.create_string_buffer(blob, len(blob))
    sig = np.ascontiguousarray(sc.sigma_vec().astype(np.float32))
    seed = scenes.controller_key(3, 1)
    model = native.Model(blob)
    x = torch.tensor(model.home(), device="cuda")
    rng = np.random.default_rng(5)
    u0 = torch.tensor(rng.normal(scale=0.1, size=(H, sc.nu)).astype(np.float32), device="cuda")
    u_in = u0.clone()
    u_out = torch.empty_like(u0)
    stream = torch.cuda.current_stream().cuda_stream or None

    def call(src, dst, it):
        st = C.c_int(-1)
        rc = L.mppi_step_noalloc(buf, len(blob), K, H, C.c_float(sc.lam), sig.ctypes.data, C.c_uint64(seed),
                                 C.c_uint64(it), x.data_ptr(), src.data_ptr(), dst.data_ptr(), C.byref(st), stream)
        assert rc == 0 and st.value == 0

    call(u_in, u_out, 0)                       # warm: address lookup, module load
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    call(u_in, u_out, 1)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    # aliased: the update written over its own input
    u_alias = u0.clone()
    u_in.copy_(u0)
    call(u_in, u_out, 2)
    call(u_alias, u_alias, 2)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(u_alias.cpu().numpy(), u_out.cpu().numpy())
    assert float((u_out - u0).abs().max()) > 0


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
