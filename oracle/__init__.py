"""FP64 CPU oracle of the torque-sampling MPPI update (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library and its Python binding
never import it, and it never imports them: the two share no code.  The
arithmetic lives in ``mppi_oracle.c`` (plain C, double precision); this module
only compiles it with gcc and marshals numpy arrays through ctypes.

What each wrapped function follows in the paper:
  normals / philox ........ Eq. 2 (noise), generator documented in the C file
  fk / jacobian ........... Fig. 1 (per-rollout kinematics, end-effector pose)
  rnea / crba / aba ....... Eq. 5-6 (rigid-body dynamics, forward dynamics)
  mass_eq8 ................ Eq. 8 (inertia by Jacobian accumulation)
  forward_dynamics ........ Eq. 6
  contact ................. Eq. 5 (tau_ext = J^T F_ext), contact-law reading
  so3_log / motion_cost ... Eq. 11
  stage_cost .............. Eq. 9-12, 14
  rollout ................. Eq. 1-3, 5-7
  mppi_update ............. Eq. 4a-4b and the warm-start shift
  mppi_partial / merge .... Eq. 4 over K split into shards (log-sum-exp merge)
  mppi_update_mix ......... Eq. 4 with two proposal plans (learned proposal and
                            the plain warm start as its fallback)
  mlp_forward / loss_grad . the learned proposal network (no paper equation:
                            an MLP and its backpropagation, from the definitions)
  mppi_step ............... the full update
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mppi_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")

NMAX = 7

METHOD_CRBA = 0
METHOD_ABA = 1
METHOD_EQ8 = 2


class Robot(C.Structure):
    _fields_ = [
        ("n", C.c_int),
        ("joint_xyz", C.c_double * 3 * NMAX),
        ("joint_rpy", C.c_double * 3 * NMAX),
        ("axis", C.c_double * 3 * NMAX),
        ("com", C.c_double * 3 * NMAX),
        ("mass", C.c_double * NMAX),
        ("inertia", C.c_double * 6 * NMAX),
        ("armature", C.c_double * NMAX),
        ("damping", C.c_double * NMAX),
        ("ee_xyz", C.c_double * 3),
        ("q_min", C.c_double * NMAX),
        ("q_max", C.c_double * NMAX),
        ("qd_max", C.c_double * NMAX),
        ("tau_max", C.c_double * NMAX),
        ("gravity", C.c_double * 3),
    ]


class Cost(C.Structure):
    _fields_ = [
        ("w_pos", C.c_double * 3),
        ("w_ori", C.c_double * 3),
        ("w_force", C.c_double),
        ("f_des", C.c_double),
        ("w_reg", C.c_double),
        ("w_qlim", C.c_double),
        ("w_qdlim", C.c_double),
        ("w_tau", C.c_double),
        ("w_posture", C.c_double),
        ("q_posture", C.c_double * NMAX),
        ("w_terminal", C.c_double),
        ("contact", C.c_int),
        ("k_contact", C.c_double),
        ("d_contact", C.c_double),
        ("force_estimate", C.c_int),
        ("w_force6", C.c_double * 6),
        ("f_des6", C.c_double * 6),
        ("w_reg6", C.c_double * 6),
        ("collision", C.c_int),
        ("w_collision", C.c_double),
        ("d_th_self", C.c_double),
        ("d_th_obs", C.c_double),
        ("link_radius", C.c_double * NMAX),
        ("n_obs", C.c_int),
        ("obs", C.c_double * 7 * 8),
        ("ext_wrench", C.c_int),
        ("f_ext", C.c_double * 6),
    ]


def build(force: bool = False) -> str:
    """Compile mppi_oracle.c into liborc.so (gcc, -O2, OpenMP)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC", "-std=c11",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


_dp = C.POINTER(C.c_double)


def _declare(L):
    RP, CP = C.POINTER(Robot), C.POINTER(Cost)
    u32p = C.POINTER(C.c_uint32)
    L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
    L.orc_normals.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, _dp]
    L.orc_rpy_matrix.argtypes = [_dp, _dp]
    L.orc_axis_angle.argtypes = [_dp, C.c_double, _dp]
    L.orc_quat_matrix.argtypes = [_dp, _dp]
    L.orc_fk.argtypes = [RP, _dp, _dp, _dp, _dp, _dp]
    L.orc_com_positions.argtypes = [RP, _dp, _dp]
    L.orc_jacobian.argtypes = [RP, _dp, _dp]
    L.orc_rnea.argtypes = [RP, _dp, _dp, _dp, _dp]
    L.orc_crba.argtypes = [RP, _dp, _dp]
    L.orc_aba.argtypes = [RP, _dp, _dp, _dp, _dp]
    L.orc_mass_eq8.argtypes = [RP, _dp, _dp]
    L.orc_cholesky_solve.argtypes = [C.c_int, _dp, _dp, _dp]
    L.orc_cholesky_solve.restype = C.c_int
    L.orc_forward_dynamics.argtypes = [RP, _dp, _dp, _dp, C.c_int, _dp]
    L.orc_forward_dynamics.restype = C.c_int
    L.orc_force_estimate.argtypes = [RP, _dp, _dp, _dp]
    L.orc_force_estimate.restype = C.c_int
    L.orc_force_estimate_cost.argtypes = [RP, CP, _dp, _dp]
    L.orc_force_estimate_cost.restype = C.c_double
    L.orc_segment_distance.argtypes = [_dp, _dp, _dp, _dp]
    L.orc_segment_distance.restype = C.c_double
    L.orc_link_points.argtypes = [RP, _dp, _dp]
    L.orc_collision_distances.argtypes = [RP, CP, _dp, _dp]
    L.orc_collision_distances.restype = C.c_int
    L.orc_collision_cost.argtypes = [RP, CP, _dp]
    L.orc_collision_cost.restype = C.c_double
    L.orc_contact.argtypes = [RP, CP, _dp, _dp, _dp, _dp]
    L.orc_contact.restype = C.c_double
    L.orc_so3_log.argtypes = [_dp, _dp]
    L.orc_motion_cost.argtypes = [CP, _dp, _dp, _dp]
    L.orc_motion_cost.restype = C.c_double
    L.orc_joint_cost.argtypes = [RP, CP, _dp, _dp, _dp]
    L.orc_joint_cost.restype = C.c_double
    L.orc_stage_cost.argtypes = [RP, CP, _dp, _dp, _dp, _dp, _dp]
    L.orc_stage_cost.restype = C.c_double
    L.orc_rollout.argtypes = [RP, CP, C.c_double, C.c_int, _dp, C.c_uint64, C.c_uint64,
                              C.c_uint32, _dp, _dp, _dp, _dp, _dp, C.c_int, _dp]
    L.orc_rollout.restype = C.c_double
    L.orc_mppi_update.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp, _dp, C.c_double,
                                  _dp, _dp, _dp]
    L.orc_mppi_update.restype = C.c_int
    L.orc_mppi_step.argtypes = [RP, CP, C.c_double, C.c_int, C.c_int, C.c_double, _dp,
                                C.c_uint64, C.c_uint64, _dp, _dp, _dp, _dp, _dp, C.c_int,
                                C.c_int, _dp, _dp, _dp, _dp, _dp]
    L.orc_mppi_step.restype = C.c_int
    L.orc_max_threads.restype = C.c_int
    L.orc_mppi_partial.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp, C.c_double, _dp]
    L.orc_mppi_merge.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp, C.c_double, _dp, _dp]
    L.orc_mppi_merge.restype = C.c_int
    L.orc_mppi_update_mix.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp, _dp, _dp, C.c_int,
                                      C.c_double, _dp, _dp]
    L.orc_mppi_update_mix.restype = C.c_int
    ip = C.POINTER(C.c_int)
    L.orc_mlp_forward.argtypes = [C.c_int, ip, _dp, C.c_int, _dp, C.c_int, _dp, _dp]
    L.orc_mlp_loss_grad.argtypes = [C.c_int, ip, _dp, C.c_int, _dp, _dp, C.c_int, _dp]
    L.orc_mlp_loss_grad.restype = C.c_double


def _arr(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None:
        assert a.size == n, (a.size, n)
    return a


def _p(a):
    return a.ctypes.data_as(_dp) if a is not None else None


# ---------------------------------------------------------------------------
# parameter records

def make_robot(d: dict) -> Robot:
    """Fill a Robot record from a dict of arrays (the seeded arm description)."""
    r = Robot()
    n = int(d["n"])
    r.n = n

    def put(field, val, shape):
        v = np.asarray(val, dtype=np.float64).reshape(shape)
        dst = getattr(r, field)
        if len(shape) == 1:
            for i in range(shape[0]):
                dst[i] = v[i]
        else:
            for i in range(shape[0]):
                for j in range(shape[1]):
                    dst[i][j] = v[i, j]

    put("joint_xyz", d["joint_xyz"], (n, 3))
    put("joint_rpy", d["joint_rpy"], (n, 3))
    put("axis", d["axis"], (n, 3))
    put("com", d["com"], (n, 3))
    put("mass", d["mass"], (n,))
    put("inertia", d["inertia"], (n, 6))
    put("armature", d["armature"], (n,))
    put("damping", d["damping"], (n,))
    put("ee_xyz", d["ee_xyz"], (3,))
    put("q_min", d["q_min"], (n,))
    put("q_max", d["q_max"], (n,))
    put("qd_max", d["qd_max"], (n,))
    put("tau_max", d["tau_max"], (n,))
    put("gravity", d["gravity"], (3,))
    return r


def make_cost(d: dict) -> Cost:
    c = Cost()
    for a in range(3):
        c.w_pos[a] = float(np.asarray(d["w_pos"])[a])
        c.w_ori[a] = float(np.asarray(d["w_ori"])[a])
    c.w_force = float(d.get("w_force", 0.0))
    c.f_des = float(d.get("f_des", 0.0))
    c.w_reg = float(d.get("w_reg", 0.0))
    c.w_qlim = float(d.get("w_qlim", 0.0))
    c.w_qdlim = float(d.get("w_qdlim", 0.0))
    c.w_tau = float(d.get("w_tau", 0.0))
    c.w_posture = float(d.get("w_posture", 0.0))
    qp = np.asarray(d.get("q_posture", np.zeros(NMAX)), dtype=np.float64)
    for j in range(min(NMAX, qp.size)):
        c.q_posture[j] = qp[j]
    c.w_terminal = float(d.get("w_terminal", 0.0))
    c.contact = int(d.get("contact", 0))
    c.k_contact = float(d.get("k_contact", 0.0))
    c.d_contact = float(d.get("d_contact", 0.0))
    c.force_estimate = int(d.get("force_estimate", 0))
    for name in ("w_force6", "f_des6", "w_reg6"):
        v = np.asarray(d.get(name, np.zeros(6)), dtype=np.float64).reshape(6)
        dst = getattr(c, name)
        for a in range(6):
            dst[a] = v[a]
    c.collision = int(d.get("collision", 0))
    for name in ("w_collision", "d_th_self", "d_th_obs"):
        setattr(c, name, float(d.get(name, 0.0)))
    lr = np.asarray(d.get("link_radius", np.zeros(NMAX)), dtype=np.float64)
    for j in range(min(NMAX, lr.size)):
        c.link_radius[j] = lr[j]
    obs = np.asarray(d.get("obstacles", np.zeros((0, 7))), dtype=np.float64).reshape(-1, 7)
    if obs.shape[0] > 8:
        raise ValueError("at most 8 obstacles")
    c.n_obs = obs.shape[0]
    for o in range(obs.shape[0]):
        for a in range(7):
            c.obs[o][a] = obs[o, a]
    c.ext_wrench = int(d.get("ext_wrench", 0))
    fe = np.asarray(d.get("f_ext", np.zeros(6)), dtype=np.float64)
    for a in range(6):
        c.f_ext[a] = fe[a]
    return c


# ---------------------------------------------------------------------------
# wrapped functions

def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    o = np.zeros(4, dtype=np.uint32)
    u32p = C.POINTER(C.c_uint32)
    lib().orc_philox4x32_10(c.ctypes.data_as(u32p), k.ctypes.data_as(u32p),
                            o.ctypes.data_as(u32p))
    return o


def normals(seed, it, k, t):
    z = np.zeros(8)
    lib().orc_normals(seed, it, k, t, _p(z))
    return z


def rpy_matrix(rpy):
    R = np.zeros((3, 3))
    lib().orc_rpy_matrix(_p(_arr(rpy, 3)), _p(R))
    return R


def axis_angle(a, q):
    R = np.zeros((3, 3))
    lib().orc_axis_angle(_p(_arr(a, 3)), float(q), _p(R))
    return R


def quat_matrix(qt):
    R = np.zeros((3, 3))
    lib().orc_quat_matrix(_p(_arr(qt, 4)), _p(R))
    return R


def fk(robot: Robot, q):
    """-> (R links [n,3,3], p links [n,3], R_ee [3,3], p_ee [3])"""
    n = robot.n
    R = np.zeros((NMAX, 3, 3))
    p = np.zeros((NMAX, 3))
    Re = np.zeros((3, 3))
    pe = np.zeros(3)
    lib().orc_fk(C.byref(robot), _p(_arr(q, n)), _p(R), _p(p), _p(Re), _p(pe))
    return R[:n], p[:n], Re, pe


def com_positions(robot: Robot, q):
    c = np.zeros((NMAX, 3))
    lib().orc_com_positions(C.byref(robot), _p(_arr(q, robot.n)), _p(c))
    return c[: robot.n]


def jacobian(robot: Robot, q):
    n = robot.n
    J = np.zeros((6, n))
    lib().orc_jacobian(C.byref(robot), _p(_arr(q, n)), _p(J))
    return J


def ext_torque(robot: Robot, cost: Cost, q0):
    """tau_ext = J(q0)^T F_ext of the cost's constant external wrench (zeros
    when it is off)."""
    t = np.zeros(robot.n)
    lib().orc_ext_torque(C.byref(robot), C.byref(cost), _p(_arr(q0, robot.n)), _p(t))
    return t


def rnea(robot: Robot, q, qd, qdd):
    n = robot.n
    tau = np.zeros(n)
    lib().orc_rnea(C.byref(robot), _p(_arr(q, n)), _p(_arr(qd, n)), _p(_arr(qdd, n)), _p(tau))
    return tau


def crba(robot: Robot, q):
    n = robot.n
    M = np.zeros((n, n))
    lib().orc_crba(C.byref(robot), _p(_arr(q, n)), _p(M))
    return M


def aba(robot: Robot, q, qd, tau):
    n = robot.n
    qdd = np.zeros(n)
    lib().orc_aba(C.byref(robot), _p(_arr(q, n)), _p(_arr(qd, n)), _p(_arr(tau, n)), _p(qdd))
    return qdd


def mass_eq8(robot: Robot, q):
    n = robot.n
    M = np.zeros((n, n))
    lib().orc_mass_eq8(C.byref(robot), _p(_arr(q, n)), _p(M))
    return M


def cholesky_solve(A, b):
    A = _arr(A)
    n = A.shape[0]
    x = np.zeros(n)
    rc = lib().orc_cholesky_solve(n, _p(A), _p(_arr(b, n)), _p(x))
    if rc != 0:
        raise np.linalg.LinAlgError("not positive definite")
    return x


def forward_dynamics(robot: Robot, q, qd, tau, method=METHOD_CRBA):
    n = robot.n
    qdd = np.zeros(n)
    rc = lib().orc_forward_dynamics(C.byref(robot), _p(_arr(q, n)), _p(_arr(qd, n)),
                                    _p(_arr(tau, n)), int(method), _p(qdd))
    if rc != 0:
        raise np.linalg.LinAlgError("mass matrix not positive definite")
    return qdd


def contact(robot: Robot, cost: Cost, plane, q, qd):
    """-> (normal force f, tau_ext [n])"""
    n = robot.n
    tex = np.zeros(n)
    f = lib().orc_contact(C.byref(robot), C.byref(cost), _p(_arr(plane, 4)), _p(_arr(q, n)),
                          _p(_arr(qd, n)), _p(tex))
    return f, tex


def so3_log(R):
    r = np.zeros(3)
    lib().orc_so3_log(_p(_arr(R, 9)), _p(r))
    return r


def motion_cost(cost: Cost, goal, p_ee, R_ee):
    return lib().orc_motion_cost(C.byref(cost), _p(_arr(goal, 7)), _p(_arr(p_ee, 3)),
                                 _p(_arr(R_ee, 9)))


def joint_cost(robot: Robot, cost: Cost, q, qd, v):
    n = robot.n
    return lib().orc_joint_cost(C.byref(robot), C.byref(cost), _p(_arr(q, n)), _p(_arr(qd, n)),
                                _p(_arr(v, n)))


def force_estimate(robot: Robot, q, v):
    """Wrench estimate F_ee = Jbar^T (v - g(q)) (Eq. 13) -> (rc, F[6])."""
    n = robot.n
    F = np.zeros(6)
    rc = lib().orc_force_estimate(C.byref(robot), _p(_arr(q, n)), _p(_arr(v, n)), _p(F))
    return rc, F


def force_estimate_cost(robot: Robot, cost: Cost, q, v):
    n = robot.n
    return lib().orc_force_estimate_cost(C.byref(robot), C.byref(cost), _p(_arr(q, n)),
                                         _p(_arr(v, n)))


def segment_distance(p1, q1, p2, q2):
    return lib().orc_segment_distance(_p(_arr(p1, 3)), _p(_arr(q1, 3)), _p(_arr(p2, 3)),
                                      _p(_arr(q2, 3)))


def link_points(robot: Robot, q):
    P = np.zeros((NMAX + 1, 3))
    lib().orc_link_points(C.byref(robot), _p(_arr(q, robot.n)), _p(P))
    return P[: robot.n + 1]


def collision_distances(robot: Robot, cost: Cost, q):
    d = np.zeros(NMAX * NMAX + NMAX * 8)
    m = lib().orc_collision_distances(C.byref(robot), C.byref(cost), _p(_arr(q, robot.n)), _p(d))
    return d[:m]


def collision_cost(robot: Robot, cost: Cost, q):
    return lib().orc_collision_cost(C.byref(robot), C.byref(cost), _p(_arr(q, robot.n)))


def stage_cost(robot: Robot, cost: Cost, goal, plane, q, qd, v):
    n = robot.n
    return lib().orc_stage_cost(C.byref(robot), C.byref(cost), _p(_arr(goal, 7)),
                                _p(_arr(plane, 4)), _p(_arr(q, n)), _p(_arr(qd, n)),
                                _p(_arr(v, n)))


def rollout(robot: Robot, cost: Cost, dt, T, sigma, seed, it, k, q0, qd0, goal, plane, plan,
            method=METHOD_CRBA, want_noise=False):
    """-> S_k, or (S_k, noise [T, n]) when want_noise."""
    n = robot.n
    noise = np.zeros((T, n)) if want_noise else None
    S = lib().orc_rollout(C.byref(robot), C.byref(cost), float(dt), int(T), _p(_arr(sigma, n)),
                          int(seed), int(it), int(k), _p(_arr(q0, n)), _p(_arr(qd0, n)),
                          _p(_arr(goal, 7)), _p(_arr(plane, 4)), _p(_arr(plan, T * n)),
                          int(method), _p(noise))
    return (S, noise) if want_noise else S


def mppi_update(S, noise, plan, lam):
    """S [K], noise [K, T, n], plan [T, n] -> (rc, ustar, plan_next, stats)"""
    S = _arr(S)
    noise = _arr(noise)
    K, T, n = noise.shape
    plan = _arr(plan, T * n)
    ustar = np.zeros((T, n))
    nxt = np.zeros((T, n))
    stats = np.zeros(4)
    rc = lib().orc_mppi_update(K, T, n, _p(S), _p(noise), _p(plan), float(lam), _p(ustar),
                               _p(nxt), _p(stats))
    return rc, ustar, nxt, stats


def mppi_step(robot: Robot, cost: Cost, dt, T, K, lam, sigma, seed, it, q0, qd0, goal, plane,
              plan, method=METHOD_CRBA, nthreads=1, want_noise=False):
    """Full update -> dict(rc, S, ustar, plan_next, tau0, stats[, noise])."""
    n = robot.n
    S = np.zeros(K)
    noise = np.zeros((K, T, n)) if want_noise else None
    ustar = np.zeros((T, n))
    nxt = np.zeros((T, n))
    stats = np.zeros(4)
    rc = lib().orc_mppi_step(C.byref(robot), C.byref(cost), float(dt), int(T), int(K),
                             float(lam), _p(_arr(sigma, n)), int(seed), int(it),
                             _p(_arr(q0, n)), _p(_arr(qd0, n)), _p(_arr(goal, 7)),
                             _p(_arr(plane, 4)), _p(_arr(plan, T * n)), int(method),
                             int(nthreads), _p(S), _p(noise), _p(ustar), _p(nxt), _p(stats))
    out = dict(rc=rc, S=S, ustar=ustar, plan_next=nxt, tau0=ustar[0].copy(), stats=stats)
    if want_noise:
        out["noise"] = noise
    return out


def mppi_update_mix(S, noise, plan, prop, k_split, lam):
    """Two-proposal update: samples k >= k_split were drawn around `prop`.
    -> (rc, ustar, plan_next)"""
    S = _arr(S)
    noise = _arr(noise)
    K, T, n = noise.shape
    ustar = np.zeros((T, n))
    nxt = np.zeros((T, n))
    rc = lib().orc_mppi_update_mix(K, T, n, _p(S), _p(noise), _p(_arr(plan, T * n)),
                                   _p(_arr(prop, T * n)), int(k_split), float(lam), _p(ustar),
                                   _p(nxt))
    return rc, ustar, nxt


def mixed_step(robot, cost, dt, T, K, lam, sigma, seed, it, q0, qd0, goal, plane, plan, prop,
               k_split, nthreads=8):
    """Full two-proposal update: rollouts around plan (k < k_split) or prop,
    then mppi_update_mix. -> dict(rc, S, ustar, plan_next)"""
    n = robot.n
    S = np.zeros(K)
    noise = np.zeros((K, T, n))
    for k in range(K):
        base = plan if k < k_split else prop
        S[k], noise[k] = rollout(robot, cost, dt, T, sigma, seed, it, k, q0, qd0, goal, plane,
                                 base, want_noise=True)
    rc, us, nxt = mppi_update_mix(S, noise, plan, prop, k_split, lam)
    return dict(rc=rc, S=S, ustar=us, plan_next=nxt)


def mppi_partial(S, noise, lam):
    """One shard's (m, Z, N[T*n]) of the sharded Eq. 4 (noise [K, T, n])."""
    S = _arr(S)
    noise = _arr(noise)
    K, T, n = noise.shape
    part = np.zeros(2 + T * n)
    lib().orc_mppi_partial(K, T, n, _p(S), _p(noise), float(lam), _p(part))
    return part


def mppi_merge(parts, plan, lam):
    """Merge of G shard partials [G, 2 + T*n] -> (rc, ustar, plan_next)."""
    parts = _arr(parts)
    plan = _arr(plan)
    T, n = plan.shape
    G = parts.shape[0]
    ustar = np.zeros((T, n))
    nxt = np.zeros((T, n))
    rc = lib().orc_mppi_merge(G, T, n, _p(parts), _p(plan), float(lam), _p(ustar), _p(nxt))
    return rc, ustar, nxt


def _dims(dims):
    d = np.ascontiguousarray(np.asarray(dims, dtype=np.int32))
    return d, d.ctypes.data_as(C.POINTER(C.c_int))


def mlp_num_params(dims) -> int:
    return int(sum(dims[l - 1] * dims[l] + dims[l] for l in range(1, len(dims))))


def mlp_forward(dims, params, X, bf16=False, want_acts=False):
    """MLP forward (hidden GELU layers, linear output) -> Y [n, out] (and the
    pre-activations of every layer when want_acts)."""
    d, dp = _dims(dims)
    X = _arr(X)
    n = X.shape[0]
    Y = np.zeros((n, dims[-1]))
    acts = np.zeros(n * sum(dims[1:])) if want_acts else None
    lib().orc_mlp_forward(len(dims) - 1, dp, _p(_arr(params)), n, _p(X), int(bf16), _p(Y), _p(acts))
    return (Y, acts) if want_acts else Y


def mlp_loss_grad(dims, params, X, Yt, bf16=False):
    """Mean squared error and its gradient w.r.t. the flat parameters."""
    d, dp = _dims(dims)
    X, Yt = _arr(X), _arr(Yt)
    g = np.zeros(mlp_num_params(dims))
    loss = lib().orc_mlp_loss_grad(len(dims) - 1, dp, _p(_arr(params)), X.shape[0], _p(X), _p(Yt),
                                   int(bf16), _p(g))
    return loss, g


def max_threads() -> int:
    return int(lib().orc_max_threads())
