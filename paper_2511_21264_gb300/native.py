"""ctypes binding of libmppi (include/mppi.h).

Argument marshalling only: every step of the optimiser and the simulator runs
in the library's CUDA kernels.  PyTorch supplies device memory and streams;
tensors are passed as raw device pointers.  There is no CPU fallback: if the
library is missing or cannot load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import glob
import os
import subprocess
from typing import Optional

_HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(_HERE, "csrc")
BUILD = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(BUILD, "libmppi.so")
# the bounds-check build (-DMPPI_BOUNDS_CHECK): every kernel index compared
# with its extent, failures counted in device words (mppi_debug_bounds)
BOUNDS_BUILD = os.path.join(_HERE, "_build_bounds")
BOUNDS_LIB_PATH = os.path.join(BOUNDS_BUILD, "libmppi.so")
INCLUDE = os.path.join(os.path.dirname(_HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# FP32 division and square root by the hardware's approximate forms (errors of
# a few ulp) rather than the correctly rounded sequences; denormals are kept.
# The divisions and square roots sit on the rollout's dependent chains (contact
# normals, capsule parameters, PGS row inverses), and the parity bounds against
# the FP64 oracle are orders of magnitude above that.
FP_FLAGS = ["-prec-div=false", "-prec-sqrt=false"]

ERRORS = {0: "MPPI_OK", 1: "MPPI_ERR_INVALID_ARG", 2: "MPPI_ERR_OOM", 3: "MPPI_ERR_CUDA",
          4: "MPPI_ERR_NONFINITE", 5: "MPPI_ERR_TIMEOUT", 6: "MPPI_ERR_ADMISSION",
          7: "MPPI_ERR_CHOLESKY", 8: "MPPI_ERR_UNSUPPORTED"}


class MPPIError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {ERRORS.get(code, code)}")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _stale(lib_path: str = LIB_PATH) -> bool:
    if not os.path.exists(lib_path):
        return True
    t = os.path.getmtime(lib_path)
    deps = _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) \
        + glob.glob(os.path.join(INCLUDE, "*.h"))
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False, bounds: bool = False) -> str:
    """Compile every translation unit under csrc/ for sm_103a (in parallel)
    and link libmppi.so in-tree; bounds=True makes the bounds-check build in
    its own folder."""
    build_dir, lib_path = (BOUNDS_BUILD, BOUNDS_LIB_PATH) if bounds else (BUILD, LIB_PATH)
    if not force and not _stale(lib_path):
        return lib_path
    os.makedirs(build_dir, exist_ok=True)
    objs, procs = [], []
    for src in _sources():
        obj = os.path.join(build_dir, os.path.basename(src) + ".o")
        cmd = ["nvcc", "-O3", *FP_FLAGS, "-std=c++17", "-Xcompiler", "-fPIC", *ARCH, "-lineinfo",
               "-I", INCLUDE, "-c", src, "-o", obj]
        if bounds:
            cmd.insert(1, "-DMPPI_BOUNDS_CHECK")
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT), src))
        objs.append(obj)
    failed = []
    for p, src in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            print(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(src)
    if failed:
        raise RuntimeError(f"nvcc failed for {failed}")
    tmp = lib_path + f".tmp{os.getpid()}"
    subprocess.run(["nvcc", "-shared", *ARCH, "-o", tmp, *objs, "-lcudart", "-lpthread"], check=True)
    os.replace(tmp, lib_path)
    return lib_path


_lib = None
EXPORTS = []


def _decl(L, name, restype, argtypes):
    f = getattr(L, name)
    f.restype = restype
    f.argtypes = argtypes
    EXPORTS.append(name)
    return f


def lib():
    """Load libmppi.so (built in-tree).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libmppi.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    i, vp, fp, sz = C.c_int, C.c_void_p, C.c_void_p, C.c_size_t
    u64 = C.c_uint64
    _decl(L, "mppi_strerror", C.c_char_p, [i])
    _decl(L, "mppi_model_load", i, [vp, sz, C.POINTER(vp)])
    _decl(L, "mppi_model_free", None, [vp])
    _decl(L, "mppi_model_dims", i, [vp, C.POINTER(i), C.POINTER(i), C.POINTER(i), C.POINTER(i)])
    _decl(L, "mppi_model_home", i, [vp, fp])
    _decl(L, "mppi_create", i, [vp, i, i, C.c_float, fp, u64, C.POINTER(vp)])
    _decl(L, "mppi_destroy", i, [vp])
    _decl(L, "mppi_step", i, [vp, fp, fp, fp, vp])
    _decl(L, "mppi_step_host", i, [vp, vp, vp, vp, vp])
    _decl(L, "mppi_solve", i, [vp, fp, fp, i, fp, vp])
    _decl(L, "mppi_update", i, [vp, fp, fp, fp, vp])
    _decl(L, "rollout_batch", i, [vp, i, fp, fp, fp, fp, vp])
    _decl(L, "sim_step", i, [vp, i, fp, fp, vp])
    _decl(L, "mppi_debug_noise", i, [vp, u64, fp, vp])
    _decl(L, "mppi_debug_philox", i, [i, fp, u64, fp, vp])
    _decl(L, "mppi_get_iteration", i, [vp, C.POINTER(u64), vp])
    _decl(L, "mppi_set_iteration", i, [vp, u64, vp])
    _decl(L, "mppi_sync", i, [vp, vp])
    _decl(L, "mppi_set_launch", i, [vp, i])
    _decl(L, "mppi_debug_bounds", i, [C.POINTER(C.c_uint), C.POINTER(i)])
    _decl(L, "mppi_set_layout", i, [vp, i, i])
    _decl(L, "mppi_get_layout", i, [vp, C.POINTER(i), C.POINTER(i), C.POINTER(i)])
    _decl(L, "mppi_set_update", i, [vp, i, C.c_float, i, C.c_float])
    _decl(L, "mppi_get_covariance", i, [vp, fp, vp])
    _decl(L, "mppi_set_covariance", i, [vp, fp, vp])
    _decl(L, "mppi_best_controls", i, [vp, fp, vp])
    _decl(L, "mppi_step_noalloc", i, [vp, sz, i, i, C.c_float, fp, u64, u64, fp, fp, fp, C.POINTER(i), vp])
    _decl(L, "mppi_batch_create", i, [vp, i, C.POINTER(vp)])
    _decl(L, "mppi_batch_destroy", i, [vp])
    _decl(L, "mppi_batch_step", i, [vp, vp, vp, vp])
    _decl(L, "mppi_batch_step_graph", i, [vp, vp, vp, vp])
    _decl(L, "mppi_batch_sync", i, [vp, C.POINTER(i), vp])
    _decl(L, "mppi_batch_iteration", i, [vp, i, C.POINTER(u64), vp])
    _decl(L, "mppi_batch_set_iteration", i, [vp, i, u64, vp])
    _decl(L, "mppi_batch_costs", C.c_void_p, [vp, i])
    _decl(L, "mppi_batch_set_launch", i, [vp, i, i])
    _decl(L, "mppi_batch_get_launch", i, [vp, C.POINTER(i), C.POINTER(i)])
    _decl(L, "mppi_batch_set_layout", i, [vp, i, i])
    _decl(L, "mppi_batch_set_update", i, [vp, i, i, C.c_float, i, C.c_float])
    _decl(L, "mppi_batch_set_projection", i, [vp, fp, i, C.c_float, fp])
    _decl(L, "mppi_batch_get_layout", i, [vp, C.POINTER(i), C.POINTER(i)])
    _decl(L, "mppi_batch_autotune", i, [vp, vp, vp, i, vp, C.POINTER(C.c_float)])
    _decl(L, "mppi_tune_store", i, [C.c_char_p, i, i, i, i, C.c_float])
    _decl(L, "mppi_tune_lookup", i, [C.c_char_p, C.POINTER(i), C.POINTER(i), C.POINTER(i), C.POINTER(i)])
    _decl(L, "srv_create", i, [C.POINTER(ServerConfig), C.POINTER(vp)])
    _decl(L, "srv_destroy", i, [vp])
    _decl(L, "srv_add_scene", i, [vp, vp, i, i, C.c_float, fp, u64, fp, C.POINTER(i)])
    _decl(L, "srv_start", i, [vp])
    _decl(L, "srv_stop", i, [vp])
    _decl(L, "srv_set_scene_update", i, [vp, i, i, C.c_float, i, C.c_float])
    _decl(L, "srv_set_scene_projection", i, [vp, i, fp, C.c_float, fp])
    _decl(L, "srv_submit", i, [vp, i, C.POINTER(u64)])
    _decl(L, "srv_cancel", i, [vp, u64])
    _decl(L, "srv_poll", i, [vp, u64, fp, i, C.POINTER(C.c_double), C.POINTER(i), i])
    _decl(L, "srv_get_state", i, [vp, i, fp])
    _decl(L, "srv_stats", i, [vp, C.POINTER(SrvStats)])
    _decl(L, "srv_run_load", i, [vp, C.c_double, C.c_double, u64, i])
    _decl(L, "mppi_profile", i, [vp, i])
    _decl(L, "mppi_profile_read", i, [vp, C.POINTER(i), C.POINTER(C.c_float), C.POINTER(C.c_float),
                                       C.POINTER(C.c_double), C.POINTER(C.c_double)])
    _decl(L, "mppi_profile_projection", i, [vp, C.POINTER(C.c_float)])
    _decl(L, "mppi_profile_lone_contacts", i, [vp, C.POINTER(C.c_double)])
    _decl(L, "mppi_qp_project", i, [i, i, C.c_float, fp, i, C.c_float, fp, fp, fp, fp, fp, vp])
    _decl(L, "mppi_set_projection", i, [vp, fp, i, C.c_float, fp])
    _decl(L, "mppi_get_samples", i, [vp, fp, vp])
    _decl(L, "mppi_set_task_cost", i, [vp, fp, i])
    _decl(L, "mppi_run_episode", i, [vp, fp, fp, C.POINTER(EpisodeConfig), fp, fp, fp, C.POINTER(EpisodeResult), vp])
    _lib = L
    return L


def _check(rc: int, what: str):
    if rc != 0:
        raise MPPIError(rc, what)


def _ptr(t) -> Optional[int]:
    """Device pointer of a CUDA float32 contiguous tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError("expected a contiguous float32 CUDA tensor")
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def debug_philox(ctr, key: int, out, stream=None):
    """Raw Philox words for the counters in ctr (CUDA int32/uint32 n x 4)."""
    import torch
    for t in (ctr, out):
        if not t.is_cuda or t.dtype not in (torch.int32, torch.uint32) or not t.is_contiguous():
            raise ValueError("expected contiguous 32-bit integer CUDA tensors")
    _check(lib().mppi_debug_philox(ctr.shape[0], ctr.data_ptr(), C.c_uint64(key), out.data_ptr(),
                                   _stream(stream)), "mppi_debug_philox")
    return out


def step_noalloc(blob: bytes, K: int, H: int, lam: float, sigma, seed: int, iteration: int, state, u_nom,
                 u_out, stream=None, want_status: bool = False):
    """One MPPI iteration through mppi_step_noalloc (no device allocation;
    scratch in the library's static device array).  Returns the device
    status when want_status (synchronises the stream), else None."""
    import numpy as np
    sig = np.ascontiguousarray(np.asarray(sigma, dtype=np.float32))
    buf = C.create_string_buffer(blob, len(blob))
    st = C.c_int(0)
    _check(lib().mppi_step_noalloc(buf, len(blob), int(K), int(H), float(lam), sig.ctypes.data, C.c_uint64(seed),
                                   C.c_uint64(iteration), _ptr(state), _ptr(u_nom), _ptr(u_out),
                                   C.byref(st) if want_status else None, _stream(stream)), "mppi_step_noalloc")
    return st.value if want_status else None


QP_SCALES = (0.1, 1.0, 2.0, 4.0)  # the library's MPPI_QP_SCALE_* defaults


def _host_f32(a, n=None):
    import numpy as np
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def qp_project(v_in, bounds, q0, qd0, dt: float, iters: int = 30, rho: float = 1.0, scales=None, v_out=None,
               stream=None):
    """QP smoothing projection (Eq. 5) of n sequences (CUDA n x H) sharing
    one set of bounds (8 host values: lo, hi for position, velocity,
    acceleration, jerk); q0, qd0: CUDA n present positions and velocities."""
    n, H = v_in.shape
    v_out = v_in if v_out is None else v_out
    b = _host_f32(bounds, 8)
    sc = None if scales is None else _host_f32(scales, 4)
    _check(lib().mppi_qp_project(int(n), int(H), float(dt), b.ctypes.data, int(iters), float(rho),
                                 None if sc is None else sc.ctypes.data, _ptr(q0), _ptr(qd0), _ptr(v_in),
                                 _ptr(v_out), _stream(stream)), "mppi_qp_project")
    return v_out


class EpisodeConfig(C.Structure):
    _fields_ = [("iters", C.c_int), ("n_avg", C.c_int), ("max_steps", C.c_int), ("goal_tol", C.c_float),
                ("lift_dz", C.c_float), ("drop_dz", C.c_float), ("pick_tol", C.c_float)]


class EpisodeResult(C.Structure):
    _fields_ = [("outcome", C.c_int), ("plans", C.c_int), ("steps", C.c_int), ("switch_step", C.c_int),
                ("task_time_s", C.c_double), ("comp_mean_ms", C.c_double), ("comp_std_ms", C.c_double)]


EPISODE_OUTCOMES = {0: "success", 1: "timeout", 2: "collision", 3: "dropped"}


class ServerConfig(C.Structure):
    _fields_ = [("mem_budget_bytes", C.c_size_t), ("max_active", C.c_int), ("iters_per_request", C.c_int),
                ("samples_per_cta", C.c_int), ("lanes_per_sample", C.c_int), ("size_classes", C.c_int),
                ("qp_iters", C.c_int)]


class SrvStats(C.Structure):
    _fields_ = [(n, C.c_longlong) for n in ("completed", "iterations", "waiting", "active", "admission_waits")] + \
               [(n, C.c_double) for n in ("p50_ms", "p99_ms", "mean_ms", "mean_active", "sample_steps_per_s")]


class Server:
    """Replan server with continuous batching (srv_*)."""

    def __init__(self, mem_budget_bytes: int, max_active: int, iters_per_request: int, samples_per_cta: int = 0,
                 lanes_per_sample: int = 0, size_classes: int = 0, qp_iters: int = 0):
        cfg = ServerConfig(int(mem_budget_bytes), int(max_active), int(iters_per_request), int(samples_per_cta),
                           int(lanes_per_sample), int(size_classes), int(qp_iters))
        h = C.c_void_p()
        _check(lib().srv_create(C.byref(cfg), C.byref(h)), "srv_create")
        self._h = h
        self._keep = []
        self.dims = {}

    def add_scene(self, model, K, H, lam, sigma, seed, x0=None) -> int:
        import numpy as np
        sig = np.ascontiguousarray(np.asarray(sigma, dtype=np.float32))
        x = None if x0 is None else np.ascontiguousarray(np.asarray(x0, dtype=np.float32))
        self._keep.append((model, sig, x))
        sid = C.c_int()
        _check(lib().srv_add_scene(self._h, model._h, int(K), int(H), float(lam), sig.ctypes.data, C.c_uint64(seed),
                                   None if x is None else x.ctypes.data, C.byref(sid)), "srv_add_scene")
        self.dims[sid.value] = (int(H), model.nu, model.nx)
        return sid.value

    def start(self):
        _check(lib().srv_start(self._h), "srv_start")

    def stop(self) -> int:
        return lib().srv_stop(self._h)

    def set_scene_update(self, scene: int, n_elite: int, eta: float = 1.0, update_cov: bool = False,
                         cov_floor: float = 0.0):
        _check(lib().srv_set_scene_update(self._h, int(scene), int(n_elite), float(eta), int(bool(update_cov)),
                                          float(cov_floor)), "srv_set_scene_update")

    def set_scene_projection(self, scene: int, bounds, rho: float = 1.0, scales=None):
        b = _host_f32(bounds)
        sc = None if scales is None else _host_f32(scales, 4)
        _check(lib().srv_set_scene_projection(self._h, int(scene), b.ctypes.data, float(rho),
                                              None if sc is None else sc.ctypes.data), "srv_set_scene_projection")

    def submit(self, scene: int) -> int:
        t = C.c_uint64()
        _check(lib().srv_submit(self._h, int(scene), C.byref(t)), "srv_submit")
        return t.value

    def cancel(self, ticket: int) -> int:
        return lib().srv_cancel(self._h, C.c_uint64(ticket))

    def poll(self, ticket: int, scene: int, wait_ms: int = 0):
        """(status, done, plan H x nu, latency_ms)."""
        import numpy as np
        H, nu, _ = self.dims[scene]
        u = np.zeros((H, nu), dtype=np.float32)
        lat, done = C.c_double(), C.c_int()
        st = lib().srv_poll(self._h, C.c_uint64(ticket), u.ctypes.data, H * nu, C.byref(lat), C.byref(done),
                            int(wait_ms))
        return st, bool(done.value), u, lat.value

    def state(self, scene: int):
        import numpy as np
        x = np.zeros(self.dims[scene][2], dtype=np.float32)
        _check(lib().srv_get_state(self._h, int(scene), x.ctypes.data), "srv_get_state")
        return x

    def stats(self) -> dict:
        st = SrvStats()
        _check(lib().srv_stats(self._h, C.byref(st)), "srv_stats")
        return {n: getattr(st, n) for n, _ in SrvStats._fields_}

    def run_load(self, rate_hz: float, duration_s: float, seed: int = 0, drain_ms: int = 120000):
        _check(lib().srv_run_load(self._h, float(rate_hz), float(duration_s), C.c_uint64(seed), int(drain_ms)),
               "srv_run_load")

    def close(self):
        if getattr(self, "_h", None):
            lib().srv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchDesc(C.Structure):
    _fields_ = [("model", C.c_void_p), ("K", C.c_int), ("H", C.c_int), ("lam", C.c_float),
                ("sigma", C.c_void_p), ("seed", C.c_uint64)]


class Batch:
    """Many controllers advanced together (mppi_batch_*).  `instances` is a
    list of (Model, K, H, lam, sigma, seed)."""

    def __init__(self, instances):
        import numpy as np
        self._keep = []
        descs = (BatchDesc * len(instances))()
        for i, (model, K, H, lam, sigma, seed) in enumerate(instances):
            sig = np.ascontiguousarray(np.asarray(sigma, dtype=np.float32).reshape(model.nu))
            self._keep.append((model, sig))
            descs[i] = BatchDesc(model._h.value, int(K), int(H), float(lam), sig.ctypes.data, int(seed))
        h = C.c_void_p()
        _check(lib().mppi_batch_create(descs, len(instances), C.byref(h)), "mppi_batch_create")
        self._h = h
        self.n = len(instances)

    @staticmethod
    def _ptrs(ts):
        arr = (C.c_void_p * len(ts))(*[_ptr(t) for t in ts])
        return arr

    def step(self, states, us, stream=None, graph=False):
        fn = lib().mppi_batch_step_graph if graph else lib().mppi_batch_step
        _check(fn(self._h, self._ptrs(states), self._ptrs(us), _stream(stream)), "mppi_batch_step")

    def sync(self, stream=None):
        errs = (C.c_int * self.n)()
        rc = lib().mppi_batch_sync(self._h, errs, _stream(stream))
        return rc, list(errs)

    def iteration(self, i, stream=None) -> int:
        v = C.c_uint64()
        _check(lib().mppi_batch_iteration(self._h, i, C.byref(v), _stream(stream)), "mppi_batch_iteration")
        return v.value

    def set_iteration(self, i, it, stream=None):
        _check(lib().mppi_batch_set_iteration(self._h, i, C.c_uint64(it), _stream(stream)),
               "mppi_batch_set_iteration")

    def costs_ptr(self, i) -> int:
        return lib().mppi_batch_costs(self._h, i)

    def set_launch(self, samples_per_cta, order):
        _check(lib().mppi_batch_set_launch(self._h, samples_per_cta, order), "mppi_batch_set_launch")

    def get_launch(self):
        s, o = C.c_int(), C.c_int()
        _check(lib().mppi_batch_get_launch(self._h, C.byref(s), C.byref(o)), "mppi_batch_get_launch")
        return s.value, o.value

    def set_layout(self, lanes_per_sample=32, placement=0):
        _check(lib().mppi_batch_set_layout(self._h, int(lanes_per_sample), int(placement)), "mppi_batch_set_layout")

    def set_update(self, i: int, n_elite: int, eta: float = 1.0, update_cov: bool = False, cov_floor: float = 0.0):
        """The full Eq. 8 for instance i (-1: all); n_elite 0 = every sample."""
        _check(lib().mppi_batch_set_update(self._h, int(i), int(n_elite), float(eta), int(bool(update_cov)),
                                           float(cov_floor)), "mppi_batch_set_update")

    def set_projection(self, bounds, iters: int = 30, rho: float = 1.0, scales=None):
        """QP projection (Eq. 5) of every instance: bounds n x nu x 8 (host);
        iters = 0 turns it off."""
        if int(iters) == 0:
            _check(lib().mppi_batch_set_projection(self._h, None, 0, 1.0, None), "mppi_batch_set_projection")
            return
        b = _host_f32(bounds)
        sc = None if scales is None else _host_f32(scales, 4)
        _check(lib().mppi_batch_set_projection(self._h, b.ctypes.data, int(iters), float(rho),
                                               None if sc is None else sc.ctypes.data), "mppi_batch_set_projection")

    def get_layout(self):
        l, p = C.c_int(), C.c_int()
        _check(lib().mppi_batch_get_layout(self._h, C.byref(l), C.byref(p)), "mppi_batch_get_layout")
        return l.value, p.value

    def autotune(self, states, us, reps=3, stream=None):
        ms = C.c_float()
        _check(lib().mppi_batch_autotune(self._h, self._ptrs(states), self._ptrs(us), reps, _stream(stream),
                                         C.byref(ms)), "mppi_batch_autotune")
        return ms.value

    def close(self):
        if getattr(self, "_h", None):
            lib().mppi_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Model:
    """A scene uploaded to the device (mppi_model_load)."""

    def __init__(self, blob: bytes):
        L = lib()
        h = C.c_void_p()
        buf = C.create_string_buffer(blob, len(blob))
        _check(L.mppi_model_load(buf, len(blob), C.byref(h)), "mppi_model_load")
        self._h = h
        nq, nv, nu, nb = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        _check(L.mppi_model_dims(h, C.byref(nq), C.byref(nv), C.byref(nu), C.byref(nb)), "mppi_model_dims")
        self.nq, self.nv, self.nu, self.n_boxes = nq.value, nv.value, nu.value, nb.value
        self.nx = self.nq + self.nv

    def home(self):
        import numpy as np
        x = np.zeros(self.nx, dtype=np.float32)
        _check(lib().mppi_model_home(self._h, x.ctypes.data), "mppi_model_home")
        return x

    def close(self):
        if getattr(self, "_h", None):
            lib().mppi_model_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Controller:
    """One MPPI controller (mppi_create).  All tensor arguments are CUDA
    float32 tensors; `stream` defaults to torch's current stream."""

    def __init__(self, model: Model, K: int, H: int, lam: float, sigma, seed: int):
        import numpy as np
        self.model = model
        self.K, self.H = int(K), int(H)
        sig = np.ascontiguousarray(np.asarray(sigma, dtype=np.float32).reshape(model.nu))
        h = C.c_void_p()
        _check(lib().mppi_create(model._h, self.K, self.H, float(lam), sig.ctypes.data, C.c_uint64(seed),
                                 C.byref(h)), "mppi_create")
        self._h = h

    def step(self, state, u_nom, u_out=None, stream=None):
        u_out = u_nom if u_out is None else u_out
        _check(lib().mppi_step(self._h, _ptr(state), _ptr(u_nom), _ptr(u_out), _stream(stream)), "mppi_step")
        return u_out

    def step_host(self, state, u_nom, u_out=None, stream=None):
        """One iteration with host arrays (numpy float32: state nx, u_nom
        H x nu); returns u_out (a new array unless given).  The library
        stages the copies and synchronises the stream."""
        import numpy as np
        x = _host_f32(state, self.model.nx)
        u = _host_f32(u_nom, self.H * self.model.nu)
        out = np.empty((self.H, self.model.nu), np.float32) if u_out is None else u_out
        if not (isinstance(out, np.ndarray) and out.dtype == np.float32 and out.flags.c_contiguous
                and out.size == self.H * self.model.nu):
            raise ValueError("u_out: C-contiguous float32 array of H x nu values")
        _check(lib().mppi_step_host(self._h, x.ctypes.data, u.ctypes.data, out.ctypes.data, _stream(stream)),
               "mppi_step_host")
        return out

    def solve(self, state, u_nom_inout, iters: int, best=None, stream=None):
        _check(lib().mppi_solve(self._h, _ptr(state), _ptr(u_nom_inout), int(iters), _ptr(best), _stream(stream)),
               "mppi_solve")
        return u_nom_inout

    def update(self, costs, u_nom, u_out, stream=None):
        _check(lib().mppi_update(self._h, _ptr(costs), _ptr(u_nom), _ptr(u_out), _stream(stream)), "mppi_update")
        return u_out

    def rollout_batch(self, states, U, costs, states_out=None, stream=None):
        n = states.shape[0]
        _check(lib().rollout_batch(self._h, n, _ptr(states), _ptr(U), _ptr(costs), _ptr(states_out),
                                   _stream(stream)), "rollout_batch")
        return costs

    def sim_step(self, states, U1, stream=None):
        _check(lib().sim_step(self._h, states.shape[0], _ptr(states), _ptr(U1), _stream(stream)), "sim_step")
        return states

    def debug_noise(self, iteration: int, eps, stream=None):
        _check(lib().mppi_debug_noise(self._h, C.c_uint64(iteration), _ptr(eps), _stream(stream)),
               "mppi_debug_noise")
        return eps

    def iteration(self, stream=None) -> int:
        v = C.c_uint64()
        _check(lib().mppi_get_iteration(self._h, C.byref(v), _stream(stream)), "mppi_get_iteration")
        return v.value

    def set_iteration(self, it: int, stream=None):
        _check(lib().mppi_set_iteration(self._h, C.c_uint64(it), _stream(stream)), "mppi_set_iteration")

    def sync(self, stream=None) -> int:
        """Synchronise and return the device error code (0 = ok)."""
        return lib().mppi_sync(self._h, _stream(stream))

    def profile(self, n: int):
        """Record kernel times and contact counts for the next n iterations."""
        _check(lib().mppi_profile(self._h, int(n)), "mppi_profile")

    def profile_read(self):
        n, tr, tu = C.c_int(), C.c_float(), C.c_float()
        cps, bps, lps = C.c_double(), C.c_double(), C.c_double()
        _check(lib().mppi_profile_read(self._h, C.byref(n), C.byref(tr), C.byref(tu), C.byref(cps),
                                       C.byref(bps)), "mppi_profile_read")
        _check(lib().mppi_profile_lone_contacts(self._h, C.byref(lps)), "mppi_profile_lone_contacts")
        return {"iterations": n.value, "rollout_ms": tr.value, "update_ms": tu.value,
                "contacts_per_step": cps.value, "box_tests_per_step": bps.value,
                "lone_ball_per_step": lps.value}

    def set_update(self, n_elite: int, eta: float = 1.0, update_cov: bool = False, cov_floor: float = 0.0):
        """The paper's full Eq. 8: elite set size, learning rate, covariance update."""
        _check(lib().mppi_set_update(self._h, int(n_elite), float(eta), int(bool(update_cov)), float(cov_floor)),
               "mppi_set_update")

    def covariance(self, out, stream=None):
        _check(lib().mppi_get_covariance(self._h, _ptr(out), _stream(stream)), "mppi_get_covariance")
        return out

    def set_covariance(self, Sigma, stream=None):
        _check(lib().mppi_set_covariance(self._h, _ptr(Sigma), _stream(stream)), "mppi_set_covariance")

    def best_controls(self, out, stream=None):
        _check(lib().mppi_best_controls(self._h, _ptr(out), _stream(stream)), "mppi_best_controls")
        return out

    def set_launch(self, samples_per_cta: int):
        _check(lib().mppi_set_launch(self._h, int(samples_per_cta)), "mppi_set_launch")

    def set_layout(self, lanes_per_sample: int = 32, placement: int = 0):
        """Rollout layout: lanes per sample (32, 16, or 8 for 3-link arms) and
        the placement of a lone ball contact's solve (0 fused, 1 after)."""
        _check(lib().mppi_set_layout(self._h, int(lanes_per_sample), int(placement)), "mppi_set_layout")

    def get_layout(self):
        l, p, s = C.c_int(), C.c_int(), C.c_int()
        _check(lib().mppi_get_layout(self._h, C.byref(l), C.byref(p), C.byref(s)), "mppi_get_layout")
        return l.value, p.value, s.value

    def set_projection(self, bounds, iters: int = 30, rho: float = 1.0, scales=None):
        """QP smoothing projection (Eq. 5) of every sample: bounds is nu x 8
        (per joint: lo, hi for position, velocity, acceleration, jerk); iters=0
        turns it off."""
        if int(iters) == 0:
            _check(lib().mppi_set_projection(self._h, None, 0, 1.0, None), "mppi_set_projection")
            return
        b = _host_f32(bounds, 8 * self.model.nu)
        sc = None if scales is None else _host_f32(scales, 4)
        _check(lib().mppi_set_projection(self._h, b.ctypes.data, int(iters), float(rho),
                                         None if sc is None else sc.ctypes.data), "mppi_set_projection")

    def set_task_cost(self, params=None):
        """The paper's ball-task cost suite (Sec. IV-B) in place of the
        scene's stage cost: params is the MPPI_TASK_N + nu array that
        scenes.ball_task builds; None turns it off."""
        if params is None:
            _check(lib().mppi_set_task_cost(self._h, None, 0), "mppi_set_task_cost")
            return
        p = _host_f32(params)
        _check(lib().mppi_set_task_cost(self._h, p.ctypes.data, int(p.size)), "mppi_set_task_cost")

    def run_episode(self, x0, u_nom, iters=10, n_avg=4, max_steps=500, goal_tol=0.03, lift_dz=0.05, drop_dz=0.05,
                    pick_tol=0.0, record=True, stream=None):
        """One closed-loop receding-horizon run (mppi_run_episode) from the
        host state x0 with the CUDA warm start u_nom (H x nu, updated).
        Returns a dict with the outcome and metrics, and with record the
        world trajectory, executed controls and per-plan compute times."""
        import numpy as np
        x = np.ascontiguousarray(np.asarray(x0, dtype=np.float32))
        cfg = EpisodeConfig(int(iters), int(n_avg), int(max_steps), float(goal_tol), float(lift_dz), float(drop_dz),
                            float(pick_tol))
        nx, nu = self.model.nx, self.model.nu
        traj = np.zeros((max_steps + 1, nx), np.float32) if record else None
        uex = np.zeros((max_steps, nu), np.float32) if record else None
        comp = np.zeros(max_steps, np.float32) if record else None
        res = EpisodeResult()
        _check(lib().mppi_run_episode(self._h, x.ctypes.data, _ptr(u_nom), C.byref(cfg),
                                      None if traj is None else traj.ctypes.data,
                                      None if uex is None else uex.ctypes.data,
                                      None if comp is None else comp.ctypes.data, C.byref(res), _stream(stream)),
               "mppi_run_episode")
        out = {n: getattr(res, n) for n, _ in EpisodeResult._fields_}
        out["outcome_name"] = EPISODE_OUTCOMES.get(res.outcome, str(res.outcome))
        if record:
            out["traj"] = traj[:res.steps + 1]
            out["u_exec"] = uex[:res.steps]
            out["comp_ms"] = comp[:res.plans]
        return out

    def samples(self, out, stream=None):
        """The last iteration's samples as rolled out (H x K x nu)."""
        _check(lib().mppi_get_samples(self._h, _ptr(out), _stream(stream)), "mppi_get_samples")
        return out

    def profile_projection(self) -> float:
        ms = C.c_float()
        _check(lib().mppi_profile_projection(self._h, C.byref(ms)), "mppi_profile_projection")
        return ms.value

    def close(self):
        if getattr(self, "_h", None):
            lib().mppi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
