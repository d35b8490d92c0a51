"""Seeded synthetic scenes and the model-blob format.

This module is the input generator shared by the CUDA path, the tests and the
benchmark.  It builds scene descriptions (kinematic parameters, inertias,
geometry, contact constants, cost weights, home state) and serialises them to
the versioned blob that ``mppi_model_load`` and the FP64 oracle both parse with
their own code.  It performs none of the simulator's or the optimiser's
arithmetic: no kinematics, dynamics, collision detection or sampling.  The
only geometry here is scene validation (axis-aligned overlap tests and a voxel
reachability search used to reject obstacle layouts).

The scenes stand in for the paper's ball lifting / transport task (Sec. IV-B)
with two arms; the paper's UR5e models and PerAct2 scenes are not available,
so link lengths, masses and obstacle layouts are drawn from a seed.

Blob layout (all little-endian)::

    u32 magic 0x4950504D ("MPPI"), u32 version (1), u32 n (float64 count), u32 0
    f64[n] payload:
      [0] n_a   joints per arm (1..7)        [1] n_boxes (0..16)
      [2] max_contacts (1..16; the GPU path takes up to 8)  [3] dt
      [4] PGS sweeps                          [5] friction mu
      [6] impedance d in (0,1]                [7] ERP
      [8..10] gravity                         [11] floor height
      [12] ball radius  [13] ball mass  [14] ball inertia (isotropic)
      [15..17] goal     [18] w_goal  [19] w_u  [20] w_pen  [21] w_obst
      [22] w_grasp
      then per arm a=0,1 (left, right): base rotation (9, row-major), base
      position (3); then per link i: F rotation (9), F translation (3), mass,
      COM (3, link frame), inertia about COM (9, link frame), capsule end
      points s0 (3), s1 (3) (link frame), capsule radius, damping, kv,
      drive gain, tau_max, u_lo, u_hi, gravcomp flag  (39 values per link)
      then per box: centre (3), half-extents (3)
      then the home state x0 = (q, qdot), nq + nv values.

Joint model: the frame of link i is ``T_{i-1} * Rz(q_i) * F_i`` with
``T_{-1}`` the base transform; joint i turns about the z axis of ``T_{i-1}``.
For a standard Denavit-Hartenberg link ``F = Rz(theta0) Tz(d) Tx(a) Rx(alpha)``.
A planar arm is the special case alpha = 0 with the base z axis along the
world y axis.  State layout: q = (left arm, right arm, ball position, ball
quaternion w-first), qdot = (left arm, right arm, ball linear velocity,
ball angular velocity, both in world coordinates).
"""
from __future__ import annotations

import math
import struct
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

MAGIC = 0x4950504D
VERSION = 1
HEADER_VALUES = 23
LINK_VALUES = 39
BOX_VALUES = 6
MAX_LINKS = 7
MAX_BOXES = 16
MAX_CONTACTS = 8
BIG = 1.0e30


def dims(n_a: int):
    """(nq, nv, nu) for two arms of n_a joints and one free ball."""
    return 2 * n_a + 7, 2 * n_a + 6, 2 * n_a


@dataclass
class Link:
    F_R: np.ndarray
    F_p: np.ndarray
    mass: float
    com: np.ndarray
    inertia: np.ndarray
    s0: np.ndarray
    s1: np.ndarray
    radius: float
    damping: float = 0.1
    kv: float = 10.0
    gear: float = 10.0
    tau_max: float = 10.0
    u_lo: float = -BIG
    u_hi: float = BIG
    gravcomp: float = 1.0


@dataclass
class Scene:
    """One scene: the model, the home state and the MPPI run settings."""
    name: str
    n_a: int
    base_R: List[np.ndarray]
    base_p: List[np.ndarray]
    links: List[List[Link]]
    boxes_c: np.ndarray
    boxes_h: np.ndarray
    x0: np.ndarray
    dt: float = 0.01
    sweeps: int = 4
    mu: float = 0.8
    impedance: float = 0.9
    erp: float = 0.2
    gravity: Sequence[float] = (0.0, 0.0, -9.81)
    floor_z: float = 0.0
    ball_r: float = 0.1
    ball_m: float = 0.5
    ball_I: float = 0.0
    goal: Sequence[float] = (0.0, 0.0, 0.4)
    w_goal: float = 10.0
    w_u: float = 0.01
    w_pen: float = 100.0
    w_obst: float = 0.0
    w_grasp: float = 0.0
    max_contacts: int = MAX_CONTACTS
    # MPPI run settings (not part of the blob)
    K: int = 64
    H: int = 20
    lam: float = 0.1
    sigma: float = 0.3
    iters: int = 10
    seed: int = 0

    @property
    def nq(self):
        return dims(self.n_a)[0]

    @property
    def nv(self):
        return dims(self.n_a)[1]

    @property
    def nu(self):
        return dims(self.n_a)[2]

    @property
    def n_boxes(self):
        return int(self.boxes_c.shape[0])

    def sigma_vec(self) -> np.ndarray:
        return np.full(self.nu, self.sigma, dtype=np.float64)

    def to_blob(self) -> bytes:
        vals: List[float] = [
            self.n_a, self.n_boxes, self.max_contacts, self.dt, self.sweeps,
            self.mu, self.impedance, self.erp, *self.gravity, self.floor_z,
            self.ball_r, self.ball_m, self.ball_I, *self.goal, self.w_goal,
            self.w_u, self.w_pen, self.w_obst, self.w_grasp,
        ]
        assert len(vals) == HEADER_VALUES
        for a in range(2):
            vals += list(np.asarray(self.base_R[a], float).reshape(9))
            vals += list(np.asarray(self.base_p[a], float).reshape(3))
            for ln in self.links[a]:
                row = (list(np.asarray(ln.F_R, float).reshape(9))
                       + list(np.asarray(ln.F_p, float).reshape(3))
                       + [ln.mass] + list(np.asarray(ln.com, float).reshape(3))
                       + list(np.asarray(ln.inertia, float).reshape(9))
                       + list(np.asarray(ln.s0, float).reshape(3))
                       + list(np.asarray(ln.s1, float).reshape(3))
                       + [ln.radius, ln.damping, ln.kv, ln.gear, ln.tau_max,
                          ln.u_lo, ln.u_hi, ln.gravcomp])
                assert len(row) == LINK_VALUES
                vals += row
        for b in range(self.n_boxes):
            vals += list(self.boxes_c[b]) + list(self.boxes_h[b])
        assert self.x0.shape == (self.nq + self.nv,)
        vals += list(self.x0)
        head = struct.pack("<IIII", MAGIC, VERSION, len(vals), 0)
        return head + np.asarray(vals, dtype="<f8").tobytes()


# ----------------------------------------------------------------------------
# model construction helpers (closed-form mass properties of the link solids)
# ----------------------------------------------------------------------------

def capsule_inertia(mass: float, length: float, radius: float):
    """Principal moments (axial, transverse) about the centre of a uniform
    solid capsule: a cylinder of the given length and radius capped by two
    hemispheres.  The transverse term uses the hemisphere's inertia about its
    flat face, 2/5 m r^2, moved to the capsule centre (centroid 3r/8 from the
    face)."""
    v_cyl = math.pi * radius * radius * length
    v_sph = 4.0 / 3.0 * math.pi * radius ** 3
    m_cyl = mass * v_cyl / (v_cyl + v_sph)
    m_sph = mass - m_cyl
    axial = 0.5 * m_cyl * radius ** 2 + 0.4 * m_sph * radius ** 2
    trans = (m_cyl * (length ** 2 / 12.0 + radius ** 2 / 4.0)
             + m_sph * (0.4 * radius ** 2 + length ** 2 / 4.0 + 3.0 * length * radius / 8.0))
    return axial, trans


def _rot_x(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]], dtype=float)


def _rot_z(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]], dtype=float)


def dh_link(a: float, alpha: float, d: float, theta0: float, mass: float,
            radius: float, **kw) -> Link:
    """Link with the fixed part Rz(theta0) Tz(d) Tx(a) Rx(alpha) of a standard
    DH transform.  Its capsule runs from the previous frame's origin (seen
    from this link's frame) to this link's origin; COM at the midpoint."""
    Rf = _rot_z(theta0) @ _rot_x(alpha)
    pf = _rot_z(theta0) @ np.array([a, 0.0, d])
    s0 = -Rf.T @ pf
    s1 = np.zeros(3)
    length = float(np.linalg.norm(s1 - s0))
    ax_m, tr_m = capsule_inertia(mass, length, radius)
    axis = (s1 - s0) / length
    inertia = tr_m * np.eye(3) + (ax_m - tr_m) * np.outer(axis, axis)
    return Link(F_R=Rf, F_p=pf, mass=mass, com=0.5 * (s0 + s1), inertia=inertia,
                s0=s0, s1=s1, radius=radius, **kw)


def resting_depth(dt, impedance, erp, g=9.81):
    """Steady depth of a body resting on one soft contact, as the scenes use to
    place the ball: g dt^2 (1-d) / (d ERP)."""
    return g * dt * dt * (1.0 - impedance) / (impedance * erp)


# base frames.  Planar arms: joint axis along the world y axis, link x axis
# pointing at the other arm, positive joint angle turns the arm downwards.
PLANAR_BASE_R = [
    np.array([[1, 0, 0], [0, 0, 1], [0, -1, 0]], dtype=float),
    np.array([[-1, 0, 0], [0, 0, -1], [0, -1, 0]], dtype=float),
]
# DH arms: link x axis straight up at q = 0; negative q_1 leans the arm
# towards the other arm (mirror-symmetric).
DH_BASE_R = [
    np.array([[0, -1, 0], [0, 0, -1], [1, 0, 0]], dtype=float),
    np.array([[0, 1, 0], [0, 0, 1], [1, 0, 0]], dtype=float),
]

# Planar home pose: absolute link angles (-80, 40.98, 95.48) degrees, which
# put the distal capsule end 0.05 m outside the 0.1 m ball at ball-centre
# height for bases 0.3 m high and 0.8 m apart (checked in the tests).
PLANAR_HOME = (math.radians(-80.0), math.radians(120.98), math.radians(54.50))
DH_HOME_TILT = math.radians(35.0)


def _ball_state(n_a, pos):
    nq, nv, _ = dims(n_a)
    x = np.zeros(nq + nv)
    x[2 * n_a:2 * n_a + 3] = pos
    x[2 * n_a + 3] = 1.0
    return x


def planar_scene(K=64, H=20, iters=10, seed=0, sigma=0.3, lam=0.1) -> Scene:
    """Two planar 3-link arms facing each other 0.8 m apart, a 0.1 m / 0.5 kg
    ball on the floor, no obstacles; goal 0.3 m above the ball's start."""
    n_a = 3
    links = [[dh_link(0.30, 0.0, 0.0, 0.0, 1.0, 0.04) for _ in range(n_a)] for _ in range(2)]
    ball_r, ball_m = 0.10, 0.5
    dt, imp, erp = 0.01, 0.9, 0.2
    start = np.array([0.0, 0.0, ball_r - resting_depth(dt, imp, erp)])
    x0 = _ball_state(n_a, start)
    x0[0:3] = PLANAR_HOME
    x0[3:6] = PLANAR_HOME
    return Scene(name="planar3_ball", n_a=n_a, base_R=PLANAR_BASE_R,
                 base_p=[np.array([-0.4, 0.0, 0.3]), np.array([0.4, 0.0, 0.3])],
                 links=links, boxes_c=np.zeros((0, 3)), boxes_h=np.zeros((0, 3)),
                 x0=x0, dt=dt, sweeps=3, mu=0.8, impedance=imp, erp=erp,
                 ball_r=ball_r, ball_m=ball_m, ball_I=0.4 * ball_m * ball_r ** 2,
                 goal=tuple(start + np.array([0.0, 0.0, 0.3])), w_goal=10.0,
                 w_u=0.01, w_pen=100.0, K=K, H=H, lam=lam, sigma=sigma,
                 iters=iters, seed=seed)


def _dh_arms(rng: np.random.Generator, n_a=7, radius=0.05):
    lengths = rng.uniform(0.10, 0.35, size=(2, n_a))
    links = []
    for a in range(2):
        arm = []
        for i in range(n_a):
            alpha = math.pi / 2 if i % 2 == 0 else -math.pi / 2
            arm.append(dh_link(float(lengths[a, i]), alpha, 0.0, 0.0, 1.0, radius))
        links.append(arm)
    return links, lengths


def _stick_points(base, tilt_sign_x, length, tilt, n=200):
    """Points along a straight arm leaning by `tilt` from vertical."""
    d = np.array([tilt_sign_x * math.sin(tilt), 0.0, math.cos(tilt)])
    s = np.linspace(0.0, length, n)
    return base[None, :] + s[:, None] * d[None, :]


def _box_clear(c, h, ball_r, start, goal, sticks, cap_r, margin=0.02):
    """A box must not overlap the start or goal ball nor the home arms
    (axis-aligned overlap of the inflated box with sample points)."""
    for p in (start, goal):
        if np.all(np.abs(p - c) <= h + ball_r + margin):
            return False
    for pts in sticks:
        if np.any(np.all(np.abs(pts - c[None, :]) <= h[None, :] + cap_r + margin, axis=1)):
            return False
    return True


def _path_exists(bc, bh, ball_r, start, goal, voxel=0.02,
                 lo=(-0.5, -0.4, 0.0), hi=(0.5, 0.4, 0.6)):
    """Reachability of the goal from the start for the ball centre on a
    voxel grid (boxes inflated by the ball radius, 6-connected free cells)."""
    from scipy import ndimage
    lo = np.asarray(lo)
    hi = np.asarray(hi)
    shape = np.maximum(1, np.round((hi - lo) / voxel).astype(int))
    axes = [lo[i] + (np.arange(shape[i]) + 0.5) * voxel for i in range(3)]
    X, Y, Z = np.meshgrid(*axes, indexing="ij")
    free = Z >= ball_r
    for c, h in zip(bc, bh):
        free &= ~((np.abs(X - c[0]) <= h[0] + ball_r) & (np.abs(Y - c[1]) <= h[1] + ball_r)
                  & (np.abs(Z - c[2]) <= h[2] + ball_r))

    def cell(p):
        idx = np.floor((np.asarray(p) - lo) / voxel).astype(int)
        return tuple(np.clip(idx, 0, shape - 1))

    s, g = cell(start), cell(goal)
    # the start ball rests on the floor: begin from the first cell above it
    s = (s[0], s[1], max(s[2], int(math.ceil((ball_r - lo[2]) / voxel - 0.5))))
    if not free[s] or not free[g]:
        return False
    labels, _ = ndimage.label(free)
    return bool(labels[s] == labels[g])


def _sample_boxes(rng, n_boxes, ball_r, start, goal, sticks, cap_r, max_tries=200):
    """Rejection sampling of an obstacle layout: boxes are drawn one at a
    time (centres uniform in the 1.0 x 0.8 x 0.6 m workspace, half-extents
    uniform in [0.03, 0.15] m) until each clears the start, goal and arms;
    the whole layout is redrawn until a path for the ball exists."""
    for _ in range(max_tries):
        bc, bh = [], []
        while len(bc) < n_boxes:
            c = rng.uniform([-0.5, -0.4, 0.0], [0.5, 0.4, 0.6])
            h = rng.uniform(0.03, 0.15, size=3)
            if _box_clear(c, h, ball_r, start, goal, sticks, cap_r):
                bc.append(c)
                bh.append(h)
        bc, bh = np.array(bc).reshape(-1, 3), np.array(bh).reshape(-1, 3)
        if _path_exists(bc, bh, ball_r, start, goal):
            return bc, bh
    raise RuntimeError("no valid obstacle layout")


def dh_scene(seed=0, n_boxes=0, K=1024, H=32, iters=50, sigma=0.2, lam=0.05,
             task="lift", ball_r: Optional[float] = None, n_a=7) -> Scene:
    """Two 7-DoF DH arms 0.6 m apart with seeded link lengths in [0.10, 0.35]
    m and 0.05 m capsules, a ball and `n_boxes` static boxes.

    task="lift": 0.12 m ball lifted from the floor to a centre height of
    0.4 m (floor only).  task="transfer": ball carried from (0,-0.3) on the
    floor to (0,0.3,0.4) past the boxes, with the obstacle and
    grasp-maintenance terms in the cost."""
    rng = np.random.default_rng(seed)
    links, lengths = _dh_arms(rng, n_a=n_a)
    dt, imp, erp = 0.01, 0.9, 0.2
    if ball_r is None:
        ball_r = 0.12 if task == "lift" else 0.10
    ball_m = 0.5
    rest = resting_depth(dt, imp, erp)
    bases = [np.array([-0.3, 0.0, 0.05]), np.array([0.3, 0.0, 0.05])]
    if task == "lift":
        start = np.array([0.0, 0.0, ball_r - rest])
        goal = np.array([0.0, 0.0, 0.4])
    else:
        start = np.array([0.0, -0.3, ball_r - rest])
        goal = np.array([0.0, 0.3, 0.4])
    sticks = [_stick_points(bases[0], +1.0, lengths[0].sum(), DH_HOME_TILT),
              _stick_points(bases[1], -1.0, lengths[1].sum(), DH_HOME_TILT)]
    bc = np.zeros((0, 3))
    bh = np.zeros((0, 3))
    if n_boxes > 0:
        bc, bh = _sample_boxes(rng, n_boxes, ball_r, start, goal, sticks, 0.05)
    x0 = _ball_state(n_a, start)
    x0[0] = -DH_HOME_TILT
    x0[n_a] = -DH_HOME_TILT
    w_obst = 50.0 if (task != "lift") else 0.0
    w_grasp = 1.0 if (task != "lift") else 0.0
    return Scene(name=f"dh7_{task}_b{n_boxes}_s{seed}", n_a=n_a, base_R=DH_BASE_R,
                 base_p=bases, links=links, boxes_c=bc, boxes_h=bh, x0=x0,
                 dt=dt, sweeps=4, mu=0.8, impedance=imp, erp=erp, ball_r=ball_r,
                 ball_m=ball_m, ball_I=0.4 * ball_m * ball_r ** 2, goal=tuple(goal),
                 w_goal=10.0, w_u=0.01, w_pen=100.0, w_obst=w_obst, w_grasp=w_grasp,
                 K=K, H=H, lam=lam, sigma=sigma, iters=iters, seed=seed)


def config(n: int, seed: int = 0) -> Scene:
    """The five workload configurations (1-based), single-instance form.

    1: planar 3-link arms, K=64, H=20, 10 iterations.
    2: 7-DoF DH arms, ball lift, K=1024, H=32, 50 iterations.
    3: 7-DoF DH arms, 8 boxes, ball transfer, K=4096, H=64, 100 iterations.
    4/5: one representative instance of the batched / served pools
         (see `batched_pool` and `served_pool`)."""
    if n == 1:
        return planar_scene(seed=seed)
    if n == 2:
        return dh_scene(seed=seed, n_boxes=0, K=1024, H=32, iters=50, task="lift")
    if n == 3:
        return dh_scene(seed=seed, n_boxes=8, K=4096, H=64, iters=100, sigma=0.2,
                        lam=0.05, task="transfer")
    if n in (4, 5):
        return batched_pool(1, seed=seed)[0]
    raise ValueError(n)


K_CHOICES = (256, 512, 1024, 2048, 4096)
H_CHOICES = (16, 32, 48, 64)


def batched_pool(n_instances=64, seed=0, k_choices=K_CHOICES, h_choices=H_CHOICES,
                 max_boxes=16) -> List[Scene]:
    """Independent MPPI instances with K, H and box counts drawn uniformly
    from the given sets (seeded); 7-DoF arms, ball transfer task."""
    rng = np.random.default_rng(10_000 + seed)
    out = []
    for i in range(n_instances):
        K = int(rng.choice(k_choices))
        H = int(rng.choice(h_choices))
        nb = int(rng.integers(0, max_boxes + 1))
        sc = dh_scene(seed=1000 * (seed + 1) + i, n_boxes=nb, K=K, H=H, iters=10,
                      sigma=0.2, lam=0.05, task="transfer")
        out.append(sc)
    return out


def served_pool(n_scenes=256, seed=0, k_choices=(512, 1024, 2048, 4096),
                h_choices=H_CHOICES) -> List[Scene]:
    """The scene pool the replan server draws requests from."""
    return batched_pool(n_scenes, seed=seed + 77, k_choices=k_choices, h_choices=h_choices)


def lift_goal(scene: Scene, seed: int) -> tuple:
    """A randomised lift goal for closed-loop runs (seeded): the ball's start
    moved by U(-0.1, 0.1) m sideways and U(0.15, 0.3) m up."""
    rng = np.random.default_rng(5000 + seed)
    start = np.array(scene.x0[scene.nu:scene.nu + 3])
    return tuple(start + np.array([rng.uniform(-0.1, 0.1), 0.0, rng.uniform(0.15, 0.3)]))


def controller_key(scene_seed: int, instance: int) -> int:
    """64-bit Philox key for one controller instance (splitmix64 of the pair)."""
    z = (scene_seed * 0x9E3779B97F4A7C15 + instance * 0xBF58476D1CE4E5B9 + 0x94D049BB133111EB)
    z &= (1 << 64) - 1
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & ((1 << 64) - 1)
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & ((1 << 64) - 1)
    return z ^ (z >> 31)


def random_states(scene: Scene, n: int, seed: int, q_spread=0.3, v_spread=0.3,
                  ball_lift=0.0) -> np.ndarray:
    """n perturbed copies of the home state (seeded), for parity tests."""
    rng = np.random.default_rng(seed)
    nq, nv = scene.nq, scene.nv
    X = np.repeat(scene.x0[None, :], n, axis=0).copy()
    na2 = 2 * scene.n_a
    X[:, :na2] += rng.uniform(-q_spread, q_spread, size=(n, na2))
    X[:, nq:nq + na2] = rng.uniform(-v_spread, v_spread, size=(n, na2))
    X[:, nq + na2:nq + nv] = rng.uniform(-v_spread, v_spread, size=(n, 6))
    X[:, na2 + 2] += ball_lift
    quat = rng.normal(size=(n, 4))
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    X[:, na2 + 3:na2 + 7] = quat
    return X


def projection_bounds(scene: Scene, pos_margin: float = 1.0, vel: float = math.pi, acc: float = 10.0,
                      jerk: float = 300.0) -> np.ndarray:
    """Bounds of the QP smoothing projection (Eq. 5), nu x 8 per joint:
    position within pos_margin of the home pose, velocity within +-vel and
    the control bounds, acceleration +-acc, jerk +-jerk.  The paper gives no
    values; these are UR5e-like rates (3.1 rad/s, 10 rad/s^2) and a jerk
    bound that makes the projection active on white-noise samples."""
    b = np.zeros((scene.nu, 8))
    q_home = scene.x0[: scene.nu]
    for j in range(scene.nu):
        ln = scene.links[j // scene.n_a][j % scene.n_a]
        b[j] = [q_home[j] - pos_margin, q_home[j] + pos_margin, max(ln.u_lo, -vel), min(ln.u_hi, vel),
                -acc, acc, -jerk, jerk]
    return b


TASK_N = 26  # task parameters before theta_home


def ball_task(scene: Scene, phase: int = 0, w_c: float = 1.0, gamma: float = 0.2, w_theta: float = 0.1,
              w_yz: float = 1.0, w_v: float = 1.0, w_r: float = 0.2, w_l: float = 5.0, w_eef_obj: float = 5.0,
              w_obj_targ: float = 5.0, eps: float = 0.02, l_ball: Optional[float] = None) -> np.ndarray:
    """Parameters of the ball-task cost suite (Sec. IV-B) as the flat array
    the library and the oracle read: phase (0 pick, 1 move), weights, the
    barrier rate gamma, the EE distance l_ball, the vertical offset eps, the
    ball position before the pick (the scene's start), the target (the
    scene's goal), the target EE orientations and theta_home (the scene's
    home pose).  l_ball defaults to the end effectors 5 mm inside the ball's
    surface on opposite sides.  The paper tunes its weights by hand and prints none; these
    defaults weight each term to the same order of magnitude on the scenes
    here.  Target orientations: the last link frames turned +-90 degrees
    about the world y axis (fixed constants, w first)."""
    # end effectors pressing 5 mm into the ball on opposite sides: the EE
    # points sit a ball radius plus a capsule radius from the centre at contact
    rc = scene.links[0][scene.n_a - 1].radius
    lb = 2.0 * (scene.ball_r + rc) - 0.01 if l_ball is None else l_ball
    c = math.cos(math.pi / 4)
    v = [float(phase), w_c, gamma, w_theta, w_yz, w_v, w_r, w_l, lb, w_eef_obj, w_obj_targ, eps]
    v += list(scene.x0[scene.nu:scene.nu + 3])        # ball position before the pick
    v += list(scene.goal)                              # target
    v += [c, 0.0, c, 0.0, c, 0.0, -c, 0.0]             # q1*, q2*
    v += list(scene.x0[:scene.nu])                     # theta_home
    assert len(v) == TASK_N + scene.nu
    return np.array(v, dtype=np.float64)
