"""Thin Python binding of the C ABI in include/mppi.h (argument marshalling only).

Every step of an update runs in the CUDA library ``libmppi.so``; this module
only converts numpy arrays / torch tensors to pointers.  There is no CPU
fallback: if the library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmppi.so")

NJ = 7
OBS_MAX = 8  # MPPI_OBS_MAX
IN_FLOATS = 25

OK = 0
ERR_INVALID_ARG = -1
ERR_OOM = -2
ERR_CUDA = -3
ERR_TIMEOUT = -4
ERR_NONFINITE = -5

_ERRNAMES = {ERR_INVALID_ARG: "INVALID_ARG", ERR_OOM: "OOM", ERR_CUDA: "CUDA",
             ERR_TIMEOUT: "TIMEOUT", ERR_NONFINITE: "NONFINITE"}


class MPPIError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class Robot(C.Structure):
    _fields_ = [
        ("n", C.c_int),
        ("joint_xyz", C.c_double * 3 * NJ),
        ("joint_rpy", C.c_double * 3 * NJ),
        ("axis", C.c_double * 3 * NJ),
        ("com", C.c_double * 3 * NJ),
        ("mass", C.c_double * NJ),
        ("inertia", C.c_double * 6 * NJ),
        ("armature", C.c_double * NJ),
        ("damping", C.c_double * NJ),
        ("ee_xyz", C.c_double * 3),
        ("q_min", C.c_double * NJ),
        ("q_max", C.c_double * NJ),
        ("qd_max", C.c_double * NJ),
        ("tau_max", C.c_double * NJ),
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
        ("q_posture", C.c_double * NJ),
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
        ("link_radius", C.c_double * NJ),
        ("n_obstacles", C.c_int),
        ("obstacles", C.c_double * 7 * OBS_MAX),
        ("ext_wrench", C.c_int),
        ("f_ext", C.c_double * 6),
    ]


class Config(C.Structure):
    _fields_ = [
        ("dt", C.c_double),
        ("T", C.c_int),
        ("K", C.c_int),
        ("lambda_", C.c_double),
        ("sigma", C.c_double * NJ),
        ("seed", C.c_uint64),
        ("reduce_fp64", C.c_int),
        ("use_graph", C.c_int),
        ("variant", C.c_int),
    ]


class ServerConfig(C.Structure):
    _fields_ = [
        ("pool_bytes", C.c_size_t),
        ("max_problems", C.c_int),
        ("max_batch", C.c_int),
        ("lanes", C.c_int),
        ("variant", C.c_int),
        ("rollout_block", C.c_int),
    ]


class MLPConfig(C.Structure):
    _fields_ = [
        ("n_in", C.c_int),
        ("n_hidden", C.c_int),
        ("n_layers", C.c_int),
        ("n_out", C.c_int),
        ("max_batch", C.c_int),
        ("seed", C.c_uint64),
        ("beta1", C.c_float),
        ("beta2", C.c_float),
        ("eps", C.c_float),
    ]


# every symbol include/*.h declares
EXPORTS = [
    "mppi_create", "mppi_destroy", "mppi_step", "mppi_step_device", "mppi_sync",
    "mppi_get_costs", "mppi_get_noise", "mppi_get_updated_plan", "mppi_get_stats",
    "mppi_set_plan", "mppi_get_plan", "mppi_set_iter", "mppi_get_iter",
    "mppi_rollout_device", "mppi_update_device", "mppi_ee_pose", "mppi_time_kernels",
    "mppi_noise_words", "mppi_step_static", "mppi_last_error", "mppi_version",
    "mppi_simulate_device", "mppi_set_plan_device", "mppi_get_plan_device",
    "mppi_get_updated_plan_device", "mppi_set_proposal_device", "mppi_gravity_torque",
    "mppi_force_estimate_device", "mppi_set_obstacles", "mppi_set_obstacles_device",
    "mppi_set_external_wrench", "mppi_set_external_wrench_device",
    "mppi_get_variant", "mppi_measure_fp32_peak", "mppi_get_correction_device",
    # include/mppi_serve.h
    "mppi_pool_create", "mppi_pool_destroy", "mppi_pool_alloc", "mppi_pool_free",
    "mppi_pool_stats", "mppi_server_create", "mppi_server_destroy", "mppi_server_add_problem",
    "mppi_server_set_plan", "mppi_server_get_plan", "mppi_server_get_iter", "mppi_server_submit",
    "mppi_server_poll", "mppi_server_wait", "mppi_server_start", "mppi_server_stop",
    "mppi_server_tick", "mppi_server_drain", "mppi_server_autotune", "mppi_server_stats",
    "mppi_server_set_input", "mppi_server_load_test",
    # include/mppi_mlp.h
    "mppi_mlp_create", "mppi_mlp_destroy", "mppi_mlp_num_params", "mppi_mlp_get_params",
    "mppi_mlp_set_params", "mppi_mlp_set_normalization", "mppi_mlp_fit_normalization",
    "mppi_mlp_forward",
    "mppi_mlp_loss_grad", "mppi_mlp_train_step", "mppi_mlp_propose", "mppi_mlp_check_wait",
    "mppi_mlp_propose_step_device",
]

_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libmppi.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} "
                           "(run python -m paper_2609_02020_b300.build)")
    L = C.CDLL(path)
    fp, dp, vp = C.POINTER(C.c_float), C.POINTER(C.c_double), C.c_void_p
    H = C.c_void_p
    sig = {
        "mppi_create": ([C.POINTER(Robot), C.POINTER(Cost), C.POINTER(Config), vp,
                         C.POINTER(C.c_void_p)], C.c_int),
        "mppi_destroy": ([H], C.c_int),
        "mppi_step": ([H, vp, vp, vp, vp, vp, vp], C.c_int),
        "mppi_step_device": ([H, vp, vp, vp], C.c_int),
        "mppi_sync": ([H], C.c_int),
        "mppi_get_costs": ([H, fp], C.c_int),
        "mppi_get_noise": ([H, fp], C.c_int),
        "mppi_get_updated_plan": ([H, fp], C.c_int),
        "mppi_get_stats": ([H, dp], C.c_int),
        "mppi_set_plan": ([H, fp], C.c_int),
        "mppi_get_plan": ([H, fp], C.c_int),
        "mppi_set_iter": ([H, C.c_uint64], C.c_int),
        "mppi_get_iter": ([H, C.POINTER(C.c_uint64)], C.c_int),
        "mppi_rollout_device": ([H, vp, vp, vp], C.c_int),
        "mppi_update_device": ([H, vp, vp, vp, vp, vp], C.c_int),
        "mppi_ee_pose": ([H, fp, fp], C.c_int),
        "mppi_time_kernels": ([H, vp, C.c_int, fp, fp], C.c_int),
        "mppi_noise_words": ([H, C.c_uint64, C.c_uint32, C.c_int, C.c_uint32,
                              C.POINTER(C.c_uint32)], C.c_int),
        "mppi_step_static": ([C.POINTER(Robot), C.POINTER(Cost), C.POINTER(Config), C.c_uint64,
                              vp, vp, vp, vp, vp], C.c_int),
        "mppi_last_error": ([H], C.c_char_p),
        "mppi_version": ([], C.c_char_p),
        "mppi_simulate_device": ([H, C.c_int, vp, vp, C.c_int, vp], C.c_int),
        "mppi_set_plan_device": ([H, vp], C.c_int),
        "mppi_get_plan_device": ([H, vp], C.c_int),
        "mppi_get_updated_plan_device": ([H, vp], C.c_int),
        "mppi_get_correction_device": ([H, vp], C.c_int),
        "mppi_set_proposal_device": ([H, vp, C.c_int], C.c_int),
        "mppi_gravity_torque": ([H, fp, fp], C.c_int),
        "mppi_force_estimate_device": ([H, vp, vp, C.c_int, vp], C.c_int),
        "mppi_set_obstacles": ([H, C.c_int, fp], C.c_int),
        "mppi_get_variant": ([H, C.POINTER(C.c_int)], C.c_int),
        "mppi_measure_fp32_peak": ([C.POINTER(C.c_double)], C.c_int),
        "mppi_set_obstacles_device": ([H, C.c_int, vp], C.c_int),
        "mppi_set_external_wrench": ([H, fp], C.c_int),
        "mppi_set_external_wrench_device": ([H, vp], C.c_int),
        "mppi_pool_create": ([C.c_size_t, C.POINTER(C.c_void_p)], C.c_int),
        "mppi_pool_destroy": ([H], C.c_int),
        "mppi_pool_alloc": ([H, C.c_size_t, C.POINTER(C.c_size_t)], C.c_int),
        "mppi_pool_free": ([H, C.c_size_t], C.c_int),
        "mppi_pool_stats": ([H, C.POINTER(C.c_size_t)], C.c_int),
        "mppi_server_create": ([C.POINTER(ServerConfig), C.POINTER(C.c_void_p)], C.c_int),
        "mppi_server_destroy": ([H], C.c_int),
        "mppi_server_add_problem": ([H, C.POINTER(Robot), C.POINTER(Cost), C.POINTER(Config),
                                     C.POINTER(C.c_int)], C.c_int),
        "mppi_server_set_plan": ([H, C.c_int, fp], C.c_int),
        "mppi_server_get_plan": ([H, C.c_int, fp], C.c_int),
        "mppi_server_get_iter": ([H, C.c_int, C.POINTER(C.c_uint64)], C.c_int),
        "mppi_server_submit": ([H, C.c_int, fp, C.POINTER(C.c_uint64)], C.c_int),
        "mppi_server_poll": ([H, C.c_uint64, fp, C.POINTER(C.c_int)], C.c_int),
        "mppi_server_wait": ([H, C.c_uint64, fp], C.c_int),
        "mppi_server_start": ([H], C.c_int),
        "mppi_server_stop": ([H], C.c_int),
        "mppi_server_tick": ([H, C.POINTER(C.c_int)], C.c_int),
        "mppi_server_drain": ([H], C.c_int),
        "mppi_server_autotune": ([H, C.POINTER(C.c_float)], C.c_int),
        "mppi_server_stats": ([H, dp], C.c_int),
        "mppi_server_set_input": ([H, C.c_int, fp], C.c_int),
        "mppi_server_load_test": ([H, C.c_double, C.c_double, C.c_uint64, dp], C.c_int),
        "mppi_mlp_create": ([C.POINTER(MLPConfig), vp, C.POINTER(C.c_void_p)], C.c_int),
        "mppi_mlp_destroy": ([H], C.c_int),
        "mppi_mlp_num_params": ([H, C.POINTER(C.c_size_t)], C.c_int),
        "mppi_mlp_get_params": ([H, fp], C.c_int),
        "mppi_mlp_set_params": ([H, fp], C.c_int),
        "mppi_mlp_set_normalization": ([H, fp, fp, fp, fp], C.c_int),
        "mppi_mlp_fit_normalization": ([H, vp, vp, C.c_int, C.c_float], C.c_int),
        "mppi_mlp_forward": ([H, vp, C.c_int, vp], C.c_int),
        "mppi_mlp_loss_grad": ([H, vp, vp, C.c_int, fp, fp], C.c_int),
        "mppi_mlp_train_step": ([H, vp, vp, C.c_int, C.c_float, fp], C.c_int),
        "mppi_mlp_propose": ([H, H, vp, C.c_int], C.c_int),
        "mppi_mlp_propose_step_device": ([H, H, vp, C.c_int, vp, vp], C.c_int),
        "mppi_mlp_check_wait": ([H, C.c_longlong], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _f32(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _fp(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _dptr(t):
    """Device pointer of a torch tensor (or None)."""
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def robot_struct(d: dict) -> Robot:
    r = Robot()
    r.n = int(d["n"])
    for name, shape in (("joint_xyz", (NJ, 3)), ("joint_rpy", (NJ, 3)), ("axis", (NJ, 3)),
                        ("com", (NJ, 3)), ("inertia", (NJ, 6))):
        v = np.asarray(d[name], dtype=np.float64).reshape(shape)
        dst = getattr(r, name)
        for i in range(shape[0]):
            for j in range(shape[1]):
                dst[i][j] = v[i, j]
    for name in ("mass", "armature", "damping", "q_min", "q_max", "qd_max", "tau_max"):
        v = np.asarray(d[name], dtype=np.float64).reshape(NJ)
        dst = getattr(r, name)
        for i in range(NJ):
            dst[i] = v[i]
    for name in ("ee_xyz", "gravity"):
        v = np.asarray(d[name], dtype=np.float64).reshape(3)
        dst = getattr(r, name)
        for i in range(3):
            dst[i] = v[i]
    return r


def cost_struct(d: dict) -> Cost:
    c = Cost()
    for a in range(3):
        c.w_pos[a] = float(np.asarray(d["w_pos"])[a])
        c.w_ori[a] = float(np.asarray(d["w_ori"])[a])
    for name in ("w_force", "f_des", "w_reg", "w_qlim", "w_qdlim", "w_tau", "w_posture",
                 "w_terminal", "k_contact", "d_contact"):
        setattr(c, name, float(d.get(name, 0.0)))
    qp = np.asarray(d.get("q_posture", np.zeros(NJ)), dtype=np.float64)
    for j in range(NJ):
        c.q_posture[j] = qp[j]
    c.contact = int(d.get("contact", 0))
    c.force_estimate = int(d.get("force_estimate", 0))
    for name in ("w_force6", "f_des6", "w_reg6"):
        v = np.asarray(d.get(name, np.zeros(6)), dtype=np.float64).reshape(6)
        dst = getattr(c, name)
        for a in range(6):
            dst[a] = v[a]
    c.collision = int(d.get("collision", 0))
    for name in ("w_collision", "d_th_self", "d_th_obs"):
        setattr(c, name, float(d.get(name, 0.0)))
    lr = np.asarray(d.get("link_radius", np.zeros(NJ)), dtype=np.float64).reshape(NJ)
    for j in range(NJ):
        c.link_radius[j] = lr[j]
    obs = np.asarray(d.get("obstacles", np.zeros((0, 7))), dtype=np.float64).reshape(-1, 7)
    if obs.shape[0] > OBS_MAX:
        raise ValueError(f"at most {OBS_MAX} obstacles")
    c.n_obstacles = obs.shape[0]
    for o in range(obs.shape[0]):
        for a in range(7):
            c.obstacles[o][a] = obs[o, a]
    c.ext_wrench = int(d.get("ext_wrench", 0))
    fe = np.asarray(d.get("f_ext", np.zeros(6)), dtype=np.float64).reshape(6)
    for a in range(6):
        c.f_ext[a] = fe[a]
    return c


class MPPI:
    """One controller handle (mppi_create ... mppi_destroy)."""

    def __init__(self, robot: dict, cost: dict, *, dt: float, T: int, K: int, lam: float,
                 sigma, seed: int, reduce_fp64: bool = False, use_graph: bool = True,
                 variant: int = 0, stream=None):
        self.lib = load()
        self.T, self.K = int(T), int(K)
        self._robot = robot_struct(robot)
        self._cost = cost_struct(cost)
        cfg = Config()
        cfg.dt = float(dt)
        cfg.T = self.T
        cfg.K = self.K
        cfg.lambda_ = float(lam)
        s = np.broadcast_to(np.asarray(sigma, dtype=np.float64), (NJ,))
        for j in range(NJ):
            cfg.sigma[j] = float(s[j])
        cfg.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
        cfg.reduce_fp64 = int(bool(reduce_fp64))
        cfg.use_graph = int(bool(use_graph))
        cfg.variant = int(variant)
        self._cfg = cfg
        h = C.c_void_p()
        sp = C.c_void_p(stream.cuda_stream) if stream is not None else None
        rc = self.lib.mppi_create(C.byref(self._robot), C.byref(self._cost), C.byref(cfg), sp,
                                  C.byref(h))
        if rc != OK:
            raise MPPIError(rc, self.lib.mppi_last_error(None).decode())
        self.h = h
        # host staging of mppi_step: inputs packed into one float32 record and
        # the outputs, with their addresses cached so that a call marshals
        # only integers
        self._in = np.zeros(IN_FLOATS, dtype=np.float32)
        self._tau = np.zeros(NJ, dtype=np.float32)
        self._plan = np.zeros((self.T, NJ), dtype=np.float32)
        a = self._in.ctypes.data
        self._a_in = (a, a + 4 * NJ, a + 8 * NJ, a + 4 * (3 * NJ))
        self._a_tau, self._a_plan = self._tau.ctypes.data, self._plan.ctypes.data

    # -- lifetime -----------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            self.lib.mppi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc):
        if rc != OK:
            raise MPPIError(rc, self.lib.mppi_last_error(self.h).decode())
        return rc

    # -- updates ------------------------------------------------------------
    def _stage(self, q, qd, goal, plane):
        b = self._in
        b[0:NJ] = q
        b[NJ:2 * NJ] = qd
        b[2 * NJ:3 * NJ] = goal
        if plane is not None:
            b[3 * NJ:] = plane
        a = self._a_in
        return a[0], a[1], a[2], (a[3] if plane is not None else None)

    def step(self, q, qd, goal, plane=None, want_plan: bool = True):
        """mppi_step from host arrays -> (tau0 [7], shifted plan [T, 7] or None)."""
        aq, aqd, ag, ap = self._stage(q, qd, goal, plane)
        self._check(self.lib.mppi_step(self.h, aq, aqd, ag, ap, self._a_tau,
                                       self._a_plan if want_plan else None))
        return self._tau.copy(), (self._plan.copy() if want_plan else None)

    def step_status(self, q, qd, goal, plane=None):
        """Like step() but returns (rc, tau0) instead of raising on NONFINITE."""
        aq, aqd, ag, ap = self._stage(q, qd, goal, plane)
        rc = self.lib.mppi_step(self.h, aq, aqd, ag, ap, self._a_tau, None)
        return rc, self._tau.copy()

    def step_device(self, d_in, d_tau0=None, d_plan=None):
        """mppi_step_device on torch CUDA tensors (queued; see sync())."""
        self._check(self.lib.mppi_step_device(self.h, _dptr(d_in), _dptr(d_tau0), _dptr(d_plan)))

    def sync(self) -> int:
        """mppi_sync: waits for the handle's stream; the last update's status."""
        return self.lib.mppi_sync(self.h)

    def rollout_device(self, d_in, d_S, d_noise=None):
        """mppi_rollout_device: the rollouts alone (costs, and the noise when
        d_noise is given) from the inputs at d_in; queued on the stream."""
        self._check(self.lib.mppi_rollout_device(self.h, _dptr(d_in), _dptr(d_S), _dptr(d_noise)))

    def update_device(self, d_S, d_noise, d_plan, d_ustar, d_plan_next):
        """mppi_update_device: Eq. 4 and the shift from caller-supplied costs and
        noise; queued on the stream."""
        self._check(self.lib.mppi_update_device(self.h, _dptr(d_S), _dptr(d_noise), _dptr(d_plan),
                                                _dptr(d_ustar), _dptr(d_plan_next)))

    # -- inspection / state -------------------------------------------------
    def costs(self) -> np.ndarray:
        """The last update's K costs S_k (Eq. 3)."""
        S = np.zeros(self.K, dtype=np.float32)
        self._check(self.lib.mppi_get_costs(self.h, _fp(S)))
        return S

    def noise(self) -> np.ndarray:
        """[T*7, K] as stored by the rollouts."""
        n = np.zeros((self.T * NJ, self.K), dtype=np.float32)
        self._check(self.lib.mppi_get_noise(self.h, _fp(n)))
        return n

    def updated_plan(self) -> np.ndarray:
        """The last update's u* [T][7] before the shift (Eq. 4b)."""
        u = np.zeros((self.T, NJ), dtype=np.float32)
        self._check(self.lib.mppi_get_updated_plan(self.h, _fp(u)))
        return u

    def stats(self) -> np.ndarray:
        """S_min, Z, n_eff and the non-finite count of the last update."""
        s = np.zeros(4, dtype=np.float64)
        self._check(self.lib.mppi_get_stats(self.h, s.ctypes.data_as(C.POINTER(C.c_double))))
        return s

    def set_plan(self, u):
        """Sets the warm start [T][7] the next update samples around."""
        self._check(self.lib.mppi_set_plan(self.h, _fp(_f32(u, self.T * NJ))))

    def get_plan(self) -> np.ndarray:
        """The warm start [T][7] the next update samples around."""
        u = np.zeros((self.T, NJ), dtype=np.float32)
        self._check(self.lib.mppi_get_plan(self.h, _fp(u)))
        return u

    def set_iter(self, it: int):
        """Sets the update counter (the Philox counter's iteration word)."""
        self._check(self.lib.mppi_set_iter(self.h, int(it)))

    def get_iter(self) -> int:
        """The update counter: successful updates so far (or as set)."""
        v = C.c_uint64()
        self._check(self.lib.mppi_get_iter(self.h, C.byref(v)))
        return int(v.value)

    def gravity_torque(self, q) -> np.ndarray:
        out = np.zeros(7, dtype=np.float32)
        self._check(self.lib.mppi_gravity_torque(self.h, _fp(_f32(q, NJ)), _fp(out)))
        return out

    def variant(self) -> int:
        """The rollout kernel this handle runs (1 register, 2 rolled, 3 warp-specialised)."""
        v = C.c_int()
        self._check(self.lib.mppi_get_variant(self.h, C.byref(v)))
        return int(v.value)

    def set_obstacles(self, obs):
        """Obstacle capsules [n][7] (a xyz, b xyz, radius) for the following updates."""
        o = np.ascontiguousarray(np.asarray(obs, dtype=np.float32).reshape(-1, 7))
        self._check(self.lib.mppi_set_obstacles(self.h, int(o.shape[0]), _fp(o.reshape(-1))))

    def set_obstacles_device(self, d_obs):
        """The same from a device tensor [n][7] (stream-ordered)."""
        self._check(self.lib.mppi_set_obstacles_device(self.h, int(d_obs.shape[0]), _dptr(d_obs)))

    def set_external_wrench(self, F):
        """Replaces F_ext of the constant external wrench (force xyz; moment
        about the end-effector point xyz, world frame), stream-ordered."""
        self._check(self.lib.mppi_set_external_wrench(self.h, _fp(_f32(F, 6))))

    def set_external_wrench_device(self, d_F):
        """The same from a device tensor of 6 floats (stream-ordered)."""
        self._check(self.lib.mppi_set_external_wrench_device(self.h, _dptr(d_F)))

    def force_estimate_device(self, d_q, d_v, d_F):
        """Wrench estimates F = Jbar^T (v - g(q)) (Eq. 13): d_q, d_v [n][7] ->
        d_F [n][6] (device tensors; queued on the handle's stream)."""
        n = int(d_q.shape[0])
        self._check(self.lib.mppi_force_estimate_device(self.h, _dptr(d_q), _dptr(d_v), n,
                                                        _dptr(d_F)))

    def ee_pose(self, q) -> np.ndarray:
        out = np.zeros(7, dtype=np.float32)
        self._check(self.lib.mppi_ee_pose(self.h, _fp(_f32(q, NJ)), _fp(out)))
        return out

    def simulate_device(self, d_in, d_tau, d_out, substeps: int = 10):
        """Advance d_in's states ([n][25]) by dt under d_tau ([n][7]) into d_out ([n][14])."""
        self._check(self.lib.mppi_simulate_device(self.h, int(d_in.shape[0]), _dptr(d_in), _dptr(d_tau),
                                                  int(substeps), _dptr(d_out)))

    def set_plan_device(self, d_u):
        self._check(self.lib.mppi_set_plan_device(self.h, _dptr(d_u)))

    def get_plan_device(self, d_u):
        self._check(self.lib.mppi_get_plan_device(self.h, _dptr(d_u)))

    def set_proposal_device(self, d_prop, n_plain: int):
        """Second proposal for the next update: samples k >= n_plain around d_prop."""
        self._check(self.lib.mppi_set_proposal_device(self.h, _dptr(d_prop), int(n_plain)))

    def get_updated_plan_device(self, d_u):
        self._check(self.lib.mppi_get_updated_plan_device(self.h, _dptr(d_u)))

    def correction_device(self, d_out):
        """u* - u of the last update into a device tensor [T, 7] (stream-ordered)."""
        self._check(self.lib.mppi_get_correction_device(self.h, _dptr(d_out)))

    def noise_words(self, it: int, k0: int, count: int, t: int) -> np.ndarray:
        """Raw Philox words [count, 8] of the device generator."""
        out = np.zeros((count, 8), dtype=np.uint32)
        self._check(self.lib.mppi_noise_words(self.h, int(it), int(k0), int(count), int(t),
                                              out.ctypes.data_as(C.POINTER(C.c_uint32))))
        return out

    def time_kernels(self, d_in, iters: int = 10):
        a, b = C.c_float(), C.c_float()
        self._check(self.lib.mppi_time_kernels(self.h, _dptr(d_in), int(iters), C.byref(a),
                                               C.byref(b)))
        return a.value, b.value


def step_static(robot: dict, cost: dict, *, dt: float, T: int, K: int, lam: float, sigma,
                seed: int, it: int, d_in, d_plan, d_ustar, d_plan_next, stream=None,
                reduce_fp64: bool = False, variant: int = 0) -> None:
    """mppi_step_static: one update without any device allocation (torch
    CUDA tensors in and out; queued on `stream`, torch's current stream when
    None)."""
    L = load()
    cfg = Config()
    cfg.dt, cfg.T, cfg.K, cfg.lambda_ = float(dt), int(T), int(K), float(lam)
    cfg.reduce_fp64 = int(bool(reduce_fp64))
    cfg.variant = int(variant)
    s = np.broadcast_to(np.asarray(sigma, dtype=np.float64), (NJ,))
    for j in range(NJ):
        cfg.sigma[j] = float(s[j])
    cfg.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    rb, cs = robot_struct(robot), cost_struct(cost)
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    rc = L.mppi_step_static(C.byref(rb), C.byref(cs), C.byref(cfg), int(it), _dptr(d_in),
                            _dptr(d_plan), _dptr(d_ustar), _dptr(d_plan_next),
                            C.c_void_p(stream.cuda_stream))
    if rc != OK:
        raise MPPIError(rc, L.mppi_last_error(None).decode())


def pack_inputs(q, qd, goal, plane=None) -> np.ndarray:
    """The 25-float input record (q, qd, goal, plane) of mppi_step_device."""
    pl = np.array([0.0, 0.0, 1.0, -1.0e9]) if plane is None else plane
    return np.concatenate([_f32(q, NJ), _f32(qd, NJ), _f32(goal, 7), _f32(pl, 4)]).astype(np.float32)


def measure_fp32_peak() -> float:
    """FP32 FMA throughput of the current CUDA device, TFLOP/s."""
    L = load()
    v = C.c_double()
    rc = L.mppi_measure_fp32_peak(C.byref(v))
    if rc != 0:
        raise MPPIError(rc, L.mppi_last_error(None).decode())
    return v.value


def version() -> str:
    return load().mppi_version().decode()


def _config(dt, T, K, lam, sigma, seed, reduce_fp64=False, use_graph=True, variant=0) -> Config:
    cfg = Config()
    cfg.dt, cfg.T, cfg.K, cfg.lambda_ = float(dt), int(T), int(K), float(lam)
    s = np.broadcast_to(np.asarray(sigma, dtype=np.float64), (NJ,))
    for j in range(NJ):
        cfg.sigma[j] = float(s[j])
    cfg.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    cfg.reduce_fp64 = int(bool(reduce_fp64))
    cfg.use_graph = int(bool(use_graph))
    cfg.variant = int(variant)
    return cfg


class Pool:
    """Host-side first-fit pool bookkeeping of include/mppi_serve.h."""

    def __init__(self, nbytes: int):
        self.lib = load()
        h = C.c_void_p()
        rc = self.lib.mppi_pool_create(int(nbytes), C.byref(h))
        if rc != OK:
            raise MPPIError(rc, "mppi_pool_create failed")
        self.h = h

    def alloc(self, nbytes: int):
        """Offset, or None when nothing fits."""
        off = C.c_size_t()
        rc = self.lib.mppi_pool_alloc(self.h, int(nbytes), C.byref(off))
        if rc == ERR_OOM:
            return None
        if rc != OK:
            raise MPPIError(rc, "mppi_pool_alloc failed")
        return int(off.value)

    def free(self, off: int) -> int:
        return self.lib.mppi_pool_free(self.h, int(off))

    def stats(self):
        out = (C.c_size_t * 4)()
        self.lib.mppi_pool_stats(self.h, out)
        return dict(size=out[0], used=out[1], peak=out[2], largest_free=out[3])

    def close(self):
        if getattr(self, "h", None):
            self.lib.mppi_pool_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Batched MPPI server (include/mppi_serve.h)."""

    def __init__(self, *, pool_bytes: int = 1 << 30, max_problems: int = 256,
                 max_batch: int = 256, lanes: int = 2, variant: int = 0, rollout_block: int = 0):
        self.lib = load()
        cfg = ServerConfig()
        cfg.pool_bytes, cfg.max_problems, cfg.max_batch = int(pool_bytes), int(max_problems), int(max_batch)
        cfg.lanes, cfg.variant, cfg.rollout_block = int(lanes), int(variant), int(rollout_block)
        h = C.c_void_p()
        rc = self.lib.mppi_server_create(C.byref(cfg), C.byref(h))
        if rc != OK:
            raise MPPIError(rc, self.lib.mppi_last_error(None).decode())
        self.h = h
        self.T = {}

    def _check(self, rc):
        if rc != OK:
            raise MPPIError(rc, self.lib.mppi_last_error(None).decode())
        return rc

    def add_problem(self, robot: dict, cost: dict, *, dt, T, K, lam, sigma, seed) -> int:
        i = C.c_int()
        rb, cs = robot_struct(robot), cost_struct(cost)
        cfg = _config(dt, T, K, lam, sigma, seed)
        self._check(self.lib.mppi_server_add_problem(self.h, C.byref(rb), C.byref(cs), C.byref(cfg),
                                                     C.byref(i)))
        self.T[i.value] = int(T)
        return i.value

    def set_plan(self, pid: int, u):
        self._check(self.lib.mppi_server_set_plan(self.h, pid, _fp(_f32(u, self.T[pid] * NJ))))

    def get_plan(self, pid: int) -> np.ndarray:
        u = np.zeros((self.T[pid], NJ), dtype=np.float32)
        self._check(self.lib.mppi_server_get_plan(self.h, pid, _fp(u)))
        return u

    def get_iter(self, pid: int) -> int:
        v = C.c_uint64()
        self._check(self.lib.mppi_server_get_iter(self.h, pid, C.byref(v)))
        return int(v.value)

    def set_input(self, pid: int, inp):
        self._check(self.lib.mppi_server_set_input(self.h, pid, _fp(_f32(inp, IN_FLOATS))))

    def submit(self, pid: int, inp) -> int:
        t = C.c_uint64()
        self._check(self.lib.mppi_server_submit(self.h, pid, _fp(_f32(inp, IN_FLOATS)), C.byref(t)))
        return int(t.value)

    def poll(self, ticket: int):
        """(done, status, tau0)"""
        tau0 = np.zeros(NJ, dtype=np.float32)
        d = C.c_int()
        rc = self.lib.mppi_server_poll(self.h, int(ticket), _fp(tau0), C.byref(d))
        if rc not in (OK, ERR_NONFINITE):
            self._check(rc)
        return bool(d.value), rc, tau0

    def wait(self, ticket: int):
        """(status, tau0)"""
        tau0 = np.zeros(NJ, dtype=np.float32)
        rc = self.lib.mppi_server_wait(self.h, int(ticket), _fp(tau0))
        if rc not in (OK, ERR_NONFINITE):
            self._check(rc)
        return rc, tau0

    def start(self):
        self._check(self.lib.mppi_server_start(self.h))

    def stop(self):
        self._check(self.lib.mppi_server_stop(self.h))

    def tick(self) -> int:
        n = C.c_int()
        self._check(self.lib.mppi_server_tick(self.h, C.byref(n)))
        return n.value

    def drain(self):
        self._check(self.lib.mppi_server_drain(self.h))

    def autotune(self) -> float:
        ms = C.c_float()
        self._check(self.lib.mppi_server_autotune(self.h, C.byref(ms)))
        return ms.value

    def stats(self) -> dict:
        o = (C.c_double * 8)()
        self._check(self.lib.mppi_server_stats(self.h, o))
        return dict(completed=o[0], ticks=o[1], mean_batch=o[2], pool_peak=o[3], pool_size=o[4],
                    variant=int(o[5]), block=int(o[6]), rollout_steps=o[7])

    def load_test(self, rate_hz: float, seconds: float, seed: int = 1) -> dict:
        o = (C.c_double * 8)()
        self._check(self.lib.mppi_server_load_test(self.h, float(rate_hz), float(seconds), int(seed), o))
        return dict(completed=o[0], p50_ms=o[1], p99_ms=o[2], mean_ms=o[3], updates_per_s=o[4],
                    rollout_steps_per_s=o[5], mean_batch=o[6], max_queue=o[7])

    def close(self):
        if getattr(self, "h", None):
            self.lib.mppi_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class MLP:
    """Learned-proposal network (include/mppi_mlp.h); device arrays are torch
    CUDA float32 tensors."""

    def __init__(self, n_in: int, n_hidden: int, n_layers: int, n_out: int, *,
                 max_batch: int = 4096, seed: int = 0, beta1=0.9, beta2=0.999, eps=1e-8,
                 stream=None):
        self.lib = load()
        cfg = MLPConfig()
        cfg.n_in, cfg.n_hidden, cfg.n_layers, cfg.n_out = n_in, n_hidden, n_layers, n_out
        cfg.max_batch, cfg.seed = int(max_batch), int(seed)
        cfg.beta1, cfg.beta2, cfg.eps = beta1, beta2, eps
        h = C.c_void_p()
        sp = C.c_void_p(stream.cuda_stream) if stream is not None else None
        rc = self.lib.mppi_mlp_create(C.byref(cfg), sp, C.byref(h))
        if rc != OK:
            raise MPPIError(rc, self.lib.mppi_last_error(None).decode())
        self.h = h
        self.dims = [n_in] + [n_hidden] * n_layers + [n_out]
        n = C.c_size_t()
        self.lib.mppi_mlp_num_params(self.h, C.byref(n))
        self.n_params = int(n.value)

    def _check(self, rc):
        if rc != OK:
            raise MPPIError(rc, self.lib.mppi_last_error(None).decode())

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.n_params, dtype=np.float32)
        self._check(self.lib.mppi_mlp_get_params(self.h, _fp(p)))
        return p

    def set_params(self, p):
        self._check(self.lib.mppi_mlp_set_params(self.h, _fp(_f32(p, self.n_params))))

    def set_normalization(self, mean_in, std_in, mean_out, std_out):
        self._check(self.lib.mppi_mlp_set_normalization(
            self.h, _fp(_f32(mean_in, self.dims[0])), _fp(_f32(std_in, self.dims[0])),
            _fp(_f32(mean_out, self.dims[-1])), _fp(_f32(std_out, self.dims[-1]))))

    def fit_normalization(self, d_x, d_y, floor: float = 1e-3):
        """Standardisation fitted on the device to training rows d_x [n, n_in], d_y [n, n_out]."""
        self._check(self.lib.mppi_mlp_fit_normalization(self.h, _dptr(d_x), _dptr(d_y),
                                                        int(d_x.shape[0]), float(floor)))

    def forward(self, d_x, d_y):
        self._check(self.lib.mppi_mlp_forward(self.h, _dptr(d_x), int(d_x.shape[0]), _dptr(d_y)))

    def loss_grad(self, d_x, d_y):
        loss = C.c_float()
        g = np.zeros(self.n_params, dtype=np.float32)
        self._check(self.lib.mppi_mlp_loss_grad(self.h, _dptr(d_x), _dptr(d_y), int(d_x.shape[0]),
                                                C.byref(loss), _fp(g)))
        return float(loss.value), g

    def train_step(self, d_x, d_y, lr: float, want_loss: bool = False):
        loss = C.c_float()
        self._check(self.lib.mppi_mlp_train_step(self.h, _dptr(d_x), _dptr(d_y), int(d_x.shape[0]),
                                                 float(lr), C.byref(loss) if want_loss else None))
        return float(loss.value) if want_loss else None

    def propose(self, ctl: "MPPI", d_in, n_plain: int = 0):
        """Install the network's plan as ctl's second proposal for its next
        update, keeping n_plain samples around ctl's warm start."""
        self._check(self.lib.mppi_mlp_propose(self.h, ctl.h, _dptr(d_in), int(n_plain)))

    def propose_step_device(self, ctl: "MPPI", d_in, n_plain: int = 0, d_tau0=None, d_plan=None):
        """propose(ctl, d_in, n_plain) and ctl.step_device(d_in, d_tau0, d_plan)
        in one call, the update's plain blocks overlapping the proposal
        (queued; see MPPI.sync())."""
        self._check(self.lib.mppi_mlp_propose_step_device(self.h, ctl.h, _dptr(d_in), int(n_plain),
                                                          _dptr(d_tau0), _dptr(d_plan)))

    def check_wait(self, cycles: int) -> int:
        """Status of one bounded device wait that nothing completes
        (ERR_TIMEOUT when the timeout path works)."""
        return int(self.lib.mppi_mlp_check_wait(self.h, int(cycles)))

    def close(self):
        if getattr(self, "h", None):
            self.lib.mppi_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
