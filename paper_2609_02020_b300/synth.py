"""Seeded synthetic inputs for the torque-sampling MPPI workloads.

This module draws random numbers and lays them out; it holds none of the
method's arithmetic (no kinematics, dynamics, cost or update).  It is the one
module that both the CUDA path's users (tests, benchmark) and the CPU oracle's
callers take their inputs from.

The paper's experiments use a real 7-DoF Franka arm, whose parameters are not
given (Sec. IV-A).  The stand-in is a seeded serial arm:
  * joint i (0-based) rotates about the local z axis for even i and the local
    y axis for odd i; joint 0 sits 0.1 m above the base, joint i>0 at
    (0, 0, l_{i-1}) in link i-1's frame, no fixed rotations;
  * link lengths l_i ~ U(0.1, 0.4) m, masses m_i ~ U(0.5, 4) kg, modelled as
    solid rods of radius 0.04 m along z: CoM (0, 0, l_i/2), principal
    inertia Ixx = Iyy = m (l^2/12 + r^2/4), Izz = m r^2 / 2 (diagonal);
  * end-effector point (0, 0, l_6) in the last link frame;
  * joint damping 0.1 N m s/rad, armature a_i (Eq. 8) 0.1 kg m^2 by default;
  * limits q in [-2.5, 2.5] rad, |qd| <= 2.5 rad/s, |tau| <= 60 N m;
    gravity (0, 0, -9.81) m/s^2.
States: q ~ U(-2.5, 2.5) per joint, qd ~ N(0, 0.2).  Goals: a position drawn
uniformly in a ball of radius 0.6 * reach around the first joint, and a
uniformly random unit quaternion (w, x, y, z).
"""
from __future__ import annotations

import numpy as np

N_JOINTS = 7
ROD_RADIUS = 0.04
BASE_HEIGHT = 0.1

# purpose tags so that robot, state, goal and plan streams never overlap
_ROBOT, _STATE, _GOAL, _PLAN, _BATCH, _GENERAL = 1, 2, 3, 4, 5, 6


def _rng(seed: int, purpose: int) -> np.random.Generator:
    return np.random.default_rng([int(seed) & 0xFFFFFFFF, purpose])


def arm(seed: int = 0, armature: float = 0.1, damping: float = 0.1) -> dict:
    """Seeded 7-revolute-joint serial arm (see module docstring)."""
    g = _rng(seed, _ROBOT)
    n = N_JOINTS
    length = g.uniform(0.1, 0.4, n)
    mass = g.uniform(0.5, 4.0, n)
    r = ROD_RADIUS
    joint_xyz = np.zeros((n, 3))
    joint_xyz[0, 2] = BASE_HEIGHT
    joint_xyz[1:, 2] = length[:-1]
    axis = np.zeros((n, 3))
    for i in range(n):
        axis[i, 2 if i % 2 == 0 else 1] = 1.0
    com = np.zeros((n, 3))
    com[:, 2] = length / 2
    inertia = np.zeros((n, 6))
    inertia[:, 0] = mass * (length ** 2 / 12 + r ** 2 / 4)
    inertia[:, 1] = inertia[:, 0]
    inertia[:, 2] = mass * r ** 2 / 2
    return dict(
        n=n,
        joint_xyz=joint_xyz,
        joint_rpy=np.zeros((n, 3)),
        axis=axis,
        com=com,
        mass=mass,
        inertia=inertia,
        armature=np.full(n, float(armature)),
        damping=np.full(n, float(damping)),
        ee_xyz=np.array([0.0, 0.0, length[-1]]),
        q_min=np.full(n, -2.5),
        q_max=np.full(n, 2.5),
        qd_max=np.full(n, 2.5),
        tau_max=np.full(n, 60.0),
        gravity=np.array([0.0, 0.0, -9.81]),
        length=length,
    )


def arm_general(seed: int = 0, armature: float = 0.1, damping: float = 0.1) -> dict:
    """The seeded arm with general geometry: each joint's fixed rotation is a
    random roll-pitch-yaw, its axis a random unit vector in its own frame,
    the joint offsets, centres of mass and end-effector point leave the
    link axis, and the link inertias carry products of inertia (the rod's
    principal inertia turned by a random rotation)."""
    a = arm(seed, armature, damping)
    g = _rng(seed, _GENERAL)
    n = N_JOINTS
    a["joint_rpy"] = g.uniform(-np.pi, np.pi, (n, 3))
    ax = g.normal(0.0, 1.0, (n, 3))
    a["axis"] = ax / np.linalg.norm(ax, axis=1, keepdims=True)
    a["joint_xyz"] = a["joint_xyz"] + np.concatenate(
        [np.zeros((1, 3)), g.uniform(-0.05, 0.05, (n - 1, 3))])
    a["com"] = a["com"] + g.uniform(-0.03, 0.03, (n, 3))
    a["ee_xyz"] = a["ee_xyz"] + g.uniform(-0.03, 0.03, 3)
    inertia = np.zeros((n, 6))
    for i in range(n):
        d = a["inertia"][i]
        Q, _ = np.linalg.qr(g.normal(0.0, 1.0, (3, 3)))
        I = Q @ np.diag(d[:3]) @ Q.T
        inertia[i] = [I[0, 0], I[1, 1], I[2, 2], I[0, 1], I[0, 2], I[1, 2]]
    a["inertia"] = inertia
    return a


def state(seed: int, robot: dict) -> tuple[np.ndarray, np.ndarray]:
    """q ~ U(q_min, q_max), qd ~ N(0, 0.2) (both float64, length n)."""
    g = _rng(seed, _STATE)
    n = int(robot["n"])
    q = g.uniform(np.asarray(robot["q_min"]), np.asarray(robot["q_max"]), n)
    qd = g.normal(0.0, 0.2, n)
    return q, qd


def goal(seed: int, robot: dict) -> np.ndarray:
    """(p_des xyz, unit quaternion wxyz) as 7 float64."""
    g = _rng(seed, _GOAL)
    reach = float(np.sum(robot["length"]))
    d = g.normal(size=3)
    d /= np.linalg.norm(d)
    rad = 0.6 * reach * g.uniform() ** (1.0 / 3.0)
    p = np.array([0.0, 0.0, BASE_HEIGHT]) + rad * d
    qt = g.normal(size=4)
    qt /= np.linalg.norm(qt)
    if qt[0] < 0:
        qt = -qt
    return np.concatenate([p, qt])


def plan(seed: int, T: int, n: int = N_JOINTS, scale: float = 0.0) -> np.ndarray:
    """Initial nominal torque plan [T, n]; zero unless a scale is given."""
    if scale == 0.0:
        return np.zeros((T, n))
    return _rng(seed, _PLAN).normal(0.0, scale, (T, n))


def cost_free_space() -> dict:
    """Weights of the one-update parity workload (free space, no contact):
    cost spread of a few lambda so that the weights are not one-hot."""
    return dict(
        w_pos=np.array([10.0, 10.0, 10.0]),
        w_ori=np.array([1.0, 1.0, 1.0]),
        w_force=0.0, f_des=0.0, w_reg=0.0,
        w_qlim=10.0, w_qdlim=10.0, w_tau=10.0, w_posture=0.01,
        q_posture=np.zeros(N_JOINTS),
        w_terminal=0.0,
        contact=0, k_contact=0.0, d_contact=0.0,
    )


def cost_contact() -> dict:
    """Pose tracking + plane contact force to a 10 N target + limit hinges
    (k = 2000 N/m, d = 50 N s/m)."""
    c = cost_free_space()
    c.update(w_force=1.0, f_des=10.0, w_reg=0.0, contact=1, k_contact=2000.0, d_contact=50.0)
    return c


def cost_force_estimate(w_fz: float = 1e-3, base: dict | None = None) -> dict:
    """C_force on the wrench estimate of Eq. 13 added to a free-space cost:
    push 10 N along -z at the end-effector (W_force on the z force only)
    with a light regulariser on all six axes."""
    c = dict(cost_free_space() if base is None else base)
    c.update(force_estimate=1,
             w_force6=np.array([0.0, 0.0, w_fz, 0.0, 0.0, 0.0]),
             f_des6=np.array([0.0, 0.0, -10.0, 0.0, 0.0, 0.0]),
             w_reg6=np.full(6, 1e-2 * w_fz))
    return c


def cost_collision(mode: int = 1, w: float = 10.0, base: dict | None = None,
                   th_self: float = 0.05, th_obs: float = 0.2, obstacles=None) -> dict:
    """C_collision of Eq. 15 added to a free-space cost: link capsules of the
    rod radius, link-link threshold th_self, link-object threshold th_obs
    (0.2 m as in the paper's obstacle experiment); mode 1 indicator, 2
    squared hinge."""
    c = dict(cost_free_space() if base is None else base)
    c.update(collision=mode, w_collision=w, d_th_self=th_self, d_th_obs=th_obs,
             link_radius=np.full(N_JOINTS, ROD_RADIUS),
             obstacles=np.zeros((0, 7)) if obstacles is None else np.asarray(obstacles, float))
    return c


def obstacles_near(points: np.ndarray, seed: int, count: int = 3, dist=(0.12, 0.3),
                   radius: float = 0.05) -> np.ndarray:
    """`count` capsule obstacles (a xyz, b xyz, radius) beside seeded
    choices of the given link points, at a distance drawn from `dist`, each
    0.05-0.2 m long in a random direction."""
    g = _rng(seed, _BATCH + 1)
    out = np.zeros((count, 7))
    for o in range(count):
        p = points[g.integers(1, len(points))]
        u = g.normal(size=3)
        u /= np.linalg.norm(u)
        c = p + g.uniform(*dist) * u
        a = g.normal(size=3)
        a *= g.uniform(0.05, 0.2) / (2 * np.linalg.norm(a))
        out[o, :3], out[o, 3:6], out[o, 6] = c - a, c + a, radius
    return out


def plane_through(point_z: float, penetration: float = 0.02) -> np.ndarray:
    """Horizontal plane n = (0, 0, 1) with offset d placed `penetration` above
    a given height (so a point at that height starts inside the contact)."""
    return np.array([0.0, 0.0, 1.0, float(point_z) + penetration])


NO_PLANE = np.array([0.0, 0.0, 1.0, -1.0e9])


def serving_mix(seed: int, count: int, k_range=(512, 8192), t_range=(10, 50)):
    """Uneven (K, T) pairs of the batched-serving workload."""
    g = _rng(seed, _BATCH)
    K = g.integers(k_range[0], k_range[1] + 1, count)
    T = g.integers(t_range[0], t_range[1] + 1, count)
    return K, T
