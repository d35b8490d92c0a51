"""FP64 CPU oracle for the MPPI + contact-rollout path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It wraps ``mppi_oracle.c`` (plain C, FP64),
which shares no code with the CUDA path.  ``build()`` compiles it with gcc.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mppi_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

MAXL, MAXB, MAXC, MAXNV, MAXNQ = 7, 16, 16, 20, 21


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, -O2)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class StepInfo(C.Structure):
    _fields_ = [("ncon", C.c_int), ("nactive", C.c_int), ("pen_all", C.c_double),
                ("pen_box", C.c_double), ("chol_fail", C.c_int)]


class Contact(C.Structure):
    _fields_ = [("dist", C.c_double), ("p", C.c_double * 3), ("n", C.c_double * 3),
                ("bodyA", C.c_int), ("bodyB", C.c_int), ("box", C.c_int)]


class FK(C.Structure):
    _fields_ = [(name, C.c_double * (2 * MAXL * k)) for name, k in
                (("R", 9), ("p", 3), ("z", 3), ("o", 3), ("c", 3), ("a0", 3), ("a1", 3), ("Iw", 9))]


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        d, i, u32p, dp = C.c_double, C.c_int, C.POINTER(C.c_uint32), C.POINTER(C.c_double)
        vp = C.c_void_p
        L.or_model_size.restype = i
        L.or_model_parse.argtypes = [vp, C.c_size_t, vp]
        L.or_model_parse.restype = i
        L.or_forward_kinematics.argtypes = [vp, dp, C.POINTER(FK)]
        L.or_mass_matrix.argtypes = [vp, dp, dp]
        L.or_bias.argtypes = [vp, dp, dp, dp]
        L.or_rnea.argtypes = [vp, dp, dp, dp, dp]
        L.or_sphere_capsule.argtypes = [dp, d, dp, dp, d, dp, dp, dp]
        L.or_box_sdf.argtypes = [dp, dp, dp, dp, dp, dp]
        L.or_sphere_box.argtypes = [dp, d, dp, dp, dp, dp, dp]
        L.or_capsule_box.argtypes = [dp, dp, d, dp, dp, dp, dp, dp, dp]
        L.or_step_ex.argtypes = [vp, dp, dp, dp, C.POINTER(StepInfo), dp, C.POINTER(Contact)]
        L.or_step_ex.restype = i
        L.or_stage_cost.argtypes = [vp, dp, dp, C.POINTER(StepInfo)]
        L.or_stage_cost.restype = d
        L.or_rollout.argtypes = [vp, dp, dp, i, dp]
        L.or_rollout.restype = d
        L.or_rollout_many.argtypes = [vp, dp, i, dp, i, i, dp, i]
        L.or_min_abs_dist.argtypes = [vp, dp]
        L.or_min_abs_dist.restype = d
        L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.or_normals4.argtypes = [u32p, dp]
        L.or_noise.argtypes = [C.c_uint64, C.c_uint64, i, i, i, dp, dp]
        L.or_mppi_update.argtypes = [i, i, i, dp, dp, d, dp, dp, dp]
        L.or_mppi_update.restype = i
        L.or_mppi_iteration.argtypes = [vp, dp, dp, i, i, d, dp, C.c_uint64, C.c_uint64, dp, dp, dp, i]
        L.or_mppi_iteration.restype = i
        ip = C.POINTER(C.c_int)
        L.or_elite_update.argtypes = [i, i, i, dp, dp, i, d, d, i, d, dp, dp, dp, dp, ip]
        L.or_elite_update.restype = i
        L.or_sample_cov.argtypes = [vp, C.c_uint64, C.c_uint64, i, i, dp, dp, dp]
        L.or_sample_cov.restype = i
        L.or_qp_project.argtypes = [i, d, d, dp, i, dp, d, d, dp, dp, dp]
        L.or_qp_project.restype = d
        L.or_capsule_capsule.argtypes = [dp, dp, d, dp, dp, d, dp]
        L.or_rot_to_quat.argtypes = [dp, dp]
        L.or_ee_state.argtypes = [vp, dp, dp]
        L.or_pair_distances.argtypes = [vp, dp, i, dp]
        L.or_pair_distances.restype = i
        L.or_task_cost_features.argtypes = [dp, i, i, i, dp, dp, dp, dp]
        L.or_task_cost_features.restype = d
        L.or_task_cost.argtypes = [vp, dp, dp, i, dp]
        L.or_task_cost.restype = d
        L.or_rollout_task.argtypes = [vp, dp, dp, dp, i, dp, dp]
        L.or_rollout_task.restype = d
        L.or_rollout_task_many.argtypes = [vp, dp, dp, dp, i, i, dp, i]
        L.or_mppi_iteration_task.argtypes = [vp, dp, dp, dp, i, i, d, dp, C.c_uint64, C.c_uint64, dp, dp, dp, i]
        L.or_mppi_iteration_task.restype = i
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Model:
    """A parsed scene in the oracle's own representation."""

    def __init__(self, blob: bytes):
        L = lib()
        self._buf = C.create_string_buffer(L.or_model_size())
        self._blob = C.create_string_buffer(blob, len(blob))
        rc = L.or_model_parse(self._blob, len(blob), self._buf)
        if rc != 0:
            raise ValueError(f"oracle: malformed scene blob ({rc})")
        hdr = np.frombuffer(blob[16:16 + 8 * 3], dtype="<f8")
        self.na = int(hdr[0])
        self.nq, self.nv, self.nu = 2 * self.na + 7, 2 * self.na + 6, 2 * self.na

    @property
    def ptr(self):
        return C.cast(self._buf, C.c_void_p)

    # -- kinematics and dynamics ------------------------------------------
    def fk(self, q):
        f = FK()
        q = _f64(q)
        lib().or_forward_kinematics(self.ptr, _dp(q), C.byref(f))
        na = self.na

        def arr(name, k):
            return np.array(getattr(f, name)).reshape(2, MAXL, k)[:, :na]
        return {n: arr(n, k) for n, k in (("R", 9), ("p", 3), ("z", 3), ("o", 3), ("c", 3),
                                           ("a0", 3), ("a1", 3), ("Iw", 9))}

    def mass_matrix(self, q):
        M = np.zeros((self.nv, self.nv))
        lib().or_mass_matrix(self.ptr, _dp(_f64(q)), _dp(M))
        return M

    def bias(self, q, qd):
        c = np.zeros(self.nv)
        lib().or_bias(self.ptr, _dp(_f64(q)), _dp(_f64(qd)), _dp(c))
        return c

    def rnea(self, q, qd, qdd):
        t = np.zeros(self.nv)
        lib().or_rnea(self.ptr, _dp(_f64(q)), _dp(_f64(qd)), _dp(_f64(qdd)), _dp(t))
        return t

    # -- stepping ----------------------------------------------------------
    def step(self, x, u, want_contacts=False):
        x = _f64(x)
        u = _f64(u)
        xo = np.zeros(self.nq + self.nv)
        info = StepInfo()
        lam = np.zeros(3 * MAXC)
        cons = (Contact * MAXC)()
        rc = lib().or_step_ex(self.ptr, _dp(x), _dp(u), _dp(xo), C.byref(info), _dp(lam), cons)
        if rc != 0:
            raise FloatingPointError("oracle: mass matrix not positive definite")
        if not want_contacts:
            return xo, info
        clist = [dict(dist=c.dist, p=np.array(c.p), n=np.array(c.n), bodyA=c.bodyA, bodyB=c.bodyB,
                      box=c.box) for c in cons[:info.ncon]]
        return xo, info, lam[:3 * info.ncon].copy(), clist

    def min_abs_dist(self, x):
        """Smallest |signed distance| over all candidate pairs at x."""
        return lib().or_min_abs_dist(self.ptr, _dp(_f64(x)))

    def stage_cost(self, x_next, u, info):
        return lib().or_stage_cost(self.ptr, _dp(_f64(x_next)), _dp(_f64(u)), C.byref(info))

    def rollout(self, x, U, traj=False):
        U = _f64(U)
        H = U.shape[0]
        T = np.zeros((H + 1, self.nq + self.nv)) if traj else None
        c = lib().or_rollout(self.ptr, _dp(_f64(x)), _dp(U), H, _dp(T) if traj else None)
        return (c, T) if traj else c

    def rollout_many(self, x, U, per_sample_state=False, nthreads=1):
        U = _f64(U)
        K, H = U.shape[0], U.shape[1]
        costs = np.zeros(K)
        lib().or_rollout_many(self.ptr, _dp(_f64(x)), int(per_sample_state), _dp(U), K, H,
                              _dp(costs), nthreads)
        return costs

    # -- ball-task cost suite (Sec. IV-B) ---------------------------------
    def ee_state(self, x):
        """End effectors at state x: dict p (2x3), v (2x3), quat (2x4)."""
        ee = np.zeros(20)
        lib().or_ee_state(self.ptr, _dp(_f64(x)), _dp(ee))
        return {"p": ee[0:6].reshape(2, 3), "v": ee[6:12].reshape(2, 3), "quat": ee[12:20].reshape(2, 4)}

    def pair_distances(self, x, phase: int):
        d = np.zeros(MAX_PAIRS)
        n = lib().or_pair_distances(self.ptr, _dp(_f64(x)), int(phase), _dp(d))
        return d[:n].copy()

    def task_cost(self, task, traj):
        """(total, terms[8]) of a trajectory of H+1 states."""
        traj = _f64(traj)
        terms = np.zeros(8)
        c = lib().or_task_cost(self.ptr, _dp(_f64(task)), _dp(traj), traj.shape[0] - 1, _dp(terms))
        return c, terms

    def rollout_task(self, x, U, task):
        """(total, terms[8], trajectory) of the rollout of U (H x nu)."""
        U = _f64(U)
        H = U.shape[0]
        traj = np.zeros((H + 1, self.nq + self.nv))
        terms = np.zeros(8)
        c = lib().or_rollout_task(self.ptr, _dp(_f64(task)), _dp(_f64(x)), _dp(U), H, _dp(traj), _dp(terms))
        return c, terms, traj

    def sample_cov(self, seed, iteration, K, nu_in, Sigma):
        """Samples U (K x H x nu) from per-step covariance blocks."""
        nu_in = _f64(nu_in)
        H = nu_in.shape[0]
        U = np.zeros((K, H, self.nu))
        rc = lib().or_sample_cov(self.ptr, C.c_uint64(seed), C.c_uint64(iteration), K, H, _dp(nu_in),
                                 _dp(_f64(Sigma)), _dp(U))
        if rc != 0:
            raise FloatingPointError("oracle: covariance block not positive definite")
        return U

    def rollout_task_many(self, x, U, task, nthreads=1):
        """Ball-task-suite costs of K sequences U (K x H x nu) from x."""
        U = _f64(U)
        K, H = U.shape[0], U.shape[1]
        costs = np.zeros(K)
        lib().or_rollout_task_many(self.ptr, _dp(_f64(task)), _dp(_f64(x)), _dp(U), K, H, _dp(costs), nthreads)
        return costs

    def mppi_iteration(self, x, u_nom, K, lam, sigma, seed, iteration, nthreads=1,
                       want_samples=False, task=None):
        """One iteration; task (the suite's parameter array) replaces the
        scene's stage cost by the ball-task suite."""
        u_nom = _f64(u_nom)
        H = u_nom.shape[0]
        u_out = np.zeros_like(u_nom)
        costs = np.zeros(K)
        U = np.zeros((K, H, self.nu)) if want_samples else None
        tail = (float(lam), _dp(_f64(sigma)), C.c_uint64(seed), C.c_uint64(iteration),
                _dp(u_out), _dp(costs), _dp(U) if want_samples else None, nthreads)
        if task is None:
            st = lib().or_mppi_iteration(self.ptr, _dp(_f64(x)), _dp(u_nom), K, H, *tail)
        else:
            st = lib().or_mppi_iteration_task(self.ptr, _dp(_f64(task)), _dp(_f64(x)), _dp(u_nom), K, H, *tail)
        out = dict(u_nom=u_out, costs=costs, status=st)
        if want_samples:
            out["U"] = U
        return out


# -- closed-loop receding horizon (Sec. III-A; metrics of Sec. IV-A) --------
EPISODE_OUTCOMES = ("success", "timeout", "collision", "dropped")


def probe(model: Model, x):
    """(smallest link-box distance, smallest left-right link distance, ball
    centre, end-effector midpoint) at state x, from the collision pairs'
    signed distances and the end effectors' positions."""
    d = model.pair_distances(x, 1)
    na = model.na
    nlb = len(d) - na * na                 # every link against every box, then left x right links
    link_box = d[:nlb].min() if nlb else np.inf
    arm_arm = d[nlb:].min()
    ball = _f64(x)[2 * na:2 * na + 3]
    mid = model.ee_state(x)["p"].mean(axis=0)
    return link_box, arm_arm, ball, mid


def run_episode(model: Model, x0, K, H, lam, sigma, seed, iters, n_avg, max_steps, goal_tol, lift_dz,
                drop_dz, pick_tol=0.0, task=None, goal=None, nthreads=1):
    """Receding-horizon control with the simulator as the world (Sec. III-A,
    Alg. 1 and the paragraph after Eq. 8).

    Each planning step runs `iters` MPPI iterations from the world state on
    the warm-started nominal sequence (iteration counter running on across
    planning steps, so iteration i draws the i-th noise block of `seed`),
    takes the lowest-cost sample of the last iteration, averages its first
    n_avg controls, applies the average for n_avg world steps and shifts the
    nominal sequence by n_avg steps (the last step repeated).  After every
    world step: collision (a link inside a box, or the two arms' links
    touching when they were apart at the start), success (the ball centre
    within goal_tol of the goal: the task's target with the ball-task suite,
    else `goal`), drop (the ball more than drop_dz below the highest point
    it reached after rising lift_dz above its start), in that order; a
    timeout after max_steps world steps.  With the suite in its pick phase
    and pick_tol > 0 the task switches to the move phase once the end
    effectors' midpoint is within pick_tol of the pick point (eps below the
    ball's start).  Returns outcome, steps, plans, switch_step, the world
    trajectory and the executed controls."""
    x = _f64(x0).copy()
    nu = model.nu
    task = None if task is None else _f64(task).copy()
    goal = _f64(task[15:18] if task is not None else goal)
    switching = task is not None and task[0] == 0.0 and pick_tol > 0.0
    pick_point = task[12:15] - np.array([0.0, 0.0, task[11]]) if task is not None else None
    u = np.zeros((H, nu))
    it = 0
    lb0, aa0, ball0, _ = probe(model, x)
    z0 = ball0[2]
    zmax, lifted = z0, False
    out = dict(outcome="timeout", steps=0, plans=0, switch_step=-1)
    traj, uex = [x.copy()], []
    done = False
    while not done and out["steps"] < max_steps:
        for _ in range(iters):
            r = model.mppi_iteration(x, u, K, lam, sigma, seed, it, nthreads=nthreads, want_samples=True,
                                     task=task)
            it += 1
            u = r["u_nom"]
        costs = np.where(np.isfinite(r["costs"]), r["costs"], np.inf)
        best = int(np.argmin(costs))           # lowest index among equal costs
        u1 = r["U"][best, :n_avg].mean(axis=0)
        for _ in range(n_avg):
            if out["steps"] >= max_steps:
                break
            x, _info = model.step(x, u1)
            out["steps"] += 1
            traj.append(x.copy())
            uex.append(u1.copy())
            lb, aa, ball, mid = probe(model, x)
            if not lifted and ball[2] > z0 + lift_dz:
                lifted = True
            zmax = max(zmax, ball[2])
            if lb < 0.0 or (aa0 >= 0.0 and aa < 0.0):
                out["outcome"], done = "collision", True
            elif np.linalg.norm(ball - goal) < goal_tol:
                out["outcome"], done = "success", True
            elif lifted and ball[2] < zmax - drop_dz:
                out["outcome"], done = "dropped", True
            if done:
                break
            if switching and np.linalg.norm(mid - pick_point) < pick_tol:
                task[0] = 1.0
                switching = False
                out["switch_step"] = out["steps"]
        out["plans"] += 1
        if done:
            break
        u = np.concatenate([u[n_avg:], np.repeat(u[-1:], min(n_avg, H), axis=0)])[:H]
    out["traj"] = np.array(traj)
    out["u_exec"] = np.array(uex).reshape(-1, nu)
    return out


# -- narrow phase (module level, for brute-force tests) --------------------
def sphere_capsule(c, r, a, b, rc):
    dist, p, n = C.c_double(), np.zeros(3), np.zeros(3)
    lib().or_sphere_capsule(_dp(_f64(c)), r, _dp(_f64(a)), _dp(_f64(b)), rc, C.byref(dist), _dp(p), _dp(n))
    return dist.value, p, n


def box_sdf(x, bc, bh):
    s, n, surf = C.c_double(), np.zeros(3), np.zeros(3)
    lib().or_box_sdf(_dp(_f64(x)), _dp(_f64(bc)), _dp(_f64(bh)), C.byref(s), _dp(n), _dp(surf))
    return s.value, n, surf


def sphere_box(c, r, bc, bh):
    dist, p, n = C.c_double(), np.zeros(3), np.zeros(3)
    lib().or_sphere_box(_dp(_f64(c)), r, _dp(_f64(bc)), _dp(_f64(bh)), C.byref(dist), _dp(p), _dp(n))
    return dist.value, p, n


def capsule_box(a, b, rc, bc, bh):
    dist, p, n, t = C.c_double(), np.zeros(3), np.zeros(3), C.c_double()
    lib().or_capsule_box(_dp(_f64(a)), _dp(_f64(b)), rc, _dp(_f64(bc)), _dp(_f64(bh)), C.byref(dist),
                         _dp(p), _dp(n), C.byref(t))
    return dist.value, p, n, t.value


# -- random numbers ---------------------------------------------------------
def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def normals4(words):
    w = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in words])
    z = np.zeros(4)
    lib().or_normals4(w, _dp(z))
    return z


def noise(seed, iteration, K, H, nu, sigma):
    eps = np.zeros((K, H, nu))
    lib().or_noise(C.c_uint64(seed), C.c_uint64(iteration), K, H, nu, _dp(_f64(sigma)), _dp(eps))
    return eps


def elite_update(costs, U, n_elite, beta, eta, nu_in, Sigma_in, update_cov=True, cov_floor=0.0):
    """Eq. 8 in full: elite set, learning rate, per-step covariance blocks.
    Returns (nu', Sigma', elite indices in cost order, status)."""
    costs = _f64(costs)
    U = _f64(U)
    K, H, nu = U.shape
    nu_out = np.zeros((H, nu))
    S_out = np.zeros((H, nu, nu))
    elite = np.zeros(max(1, min(n_elite, K)), dtype=np.int32)
    st = lib().or_elite_update(K, H, nu, _dp(costs), _dp(U), int(n_elite), float(beta), float(eta), int(update_cov),
                               float(cov_floor), _dp(_f64(nu_in)), _dp(_f64(Sigma_in)), _dp(nu_out), _dp(S_out),
                               elite.ctypes.data_as(C.POINTER(C.c_int)))
    return nu_out, S_out, elite, st


TASK_N = 26        # task parameters before theta_home
MAX_PAIRS = 2 * 7 * 16 + 2 * 7 + 7 * 7
TASK_TERMS = ("C_c", "C_theta", "C_yz", "C_v", "C_r", "C_l", "C_eef_obj", "C_obj_targ")


def capsule_capsule(a0, a1, ra, b0, b1, rb) -> float:
    d = np.zeros(1)
    lib().or_capsule_capsule(_dp(_f64(a0)), _dp(_f64(a1)), float(ra), _dp(_f64(b0)), _dp(_f64(b1)), float(rb),
                             _dp(d))
    return float(d[0])


def rot_to_quat(R):
    q = np.zeros(4)
    lib().or_rot_to_quat(_dp(_f64(R).reshape(9).copy()), _dp(q))
    return q


def task_cost_features(task, D, TH, EE):
    """Task cost from features of x_0..x_H: D (H+1, B), TH (H+1, nu),
    EE (H+1, 20).  Returns (total, terms[8])."""
    D, TH, EE = _f64(D), _f64(TH), _f64(EE)
    terms = np.zeros(8)
    c = lib().or_task_cost_features(_dp(_f64(task)), TH.shape[1], D.shape[1], D.shape[0] - 1, _dp(D), _dp(TH),
                                    _dp(EE), _dp(terms))
    return c, terms


QP_SCALES = (0.1, 1.0, 2.0, 4.0)


def qp_project(vt, bounds, q, qd, dt, rho=1.0, iters=100, scales=QP_SCALES):
    """QP smoothing projection of one joint's velocity sequence (Eq. 5):
    `iters` ADMM iterations on the row groups (position, velocity,
    acceleration, jerk) scaled by `scales`.  bounds: (lo, hi) for position,
    velocity, acceleration, jerk (8 values; +-inf leaves a group free).
    Returns (v, scaled duals in row order P, V, A, J, largest violation)."""
    vt = _f64(vt)
    H = vt.shape[0]
    v = np.zeros(H)
    y = np.zeros(4 * H - 1)
    r = lib().or_qp_project(H, float(dt), float(rho), _dp(_f64(scales)), int(iters), _dp(_f64(bounds)), float(q),
                            float(qd), _dp(vt), _dp(v), _dp(y))
    return v, y, r


def mppi_update(costs, U, lam, u_nom):
    costs = _f64(costs)
    U = _f64(U)
    K, H, nu = U.shape
    u_out = np.zeros((H, nu))
    w = np.zeros(K)
    st = lib().or_mppi_update(K, H, nu, _dp(costs), _dp(U), float(lam), _dp(_f64(u_nom)), _dp(u_out), _dp(w))
    return u_out, w, st
