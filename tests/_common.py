"""Shared test helpers: build one workload for both the CUDA path and the oracle.

Inputs come from the seeded generators in ``paper_2609_02020_b300.synth``;
per-update inputs (q, qd, goal, plane) are rounded to float32 first, because
that is what the C ABI takes, and the oracle receives the same rounded values.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_2609_02020_b300 import synth

SEED = 0xC0FFEE


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def parity_cost(scale: float = 0.05) -> dict:
    """Free-space weights scaled so that S is O(10-50) lambda.  FP32 rollouts
    carry a relative cost error of about 2e-7, and the plan moves by about
    sigma * (cost error) / lambda through the weights of Eq. 4a, so the 1e-5
    N m plan tolerance needs S / lambda of a few tens at most."""
    c = synth.cost_free_space()
    for k in ("w_pos", "w_ori"):
        c[k] = np.asarray(c[k]) * scale
    for k in ("w_qlim", "w_qdlim", "w_tau", "w_posture"):
        c[k] = c[k] * scale
    return c


def make_case(seed: int, *, contact: bool = False, cost: dict | None = None, K: int = 256,
              T: int = 18, dt: float = 0.01, lam: float = 1.0, sigma=2.0, armature: float = 0.1,
              penetration: float = 0.02, general: bool = False) -> dict:
    arm = (synth.arm_general if general else synth.arm)(seed, armature=armature)
    q, qd = synth.state(1000 + seed, arm)
    goal = synth.goal(1000 + seed, arm)
    if cost is None:
        cost = synth.cost_contact() if contact else synth.cost_free_space()
    rb = oracle.make_robot(arm)
    q, qd, goal = f32(q), f32(qd), f32(goal)
    if cost.get("contact", 0):
        pe = oracle.fk(rb, q)[3]
        plane = f32(synth.plane_through(pe[2], penetration))
    else:
        plane = f32(synth.NO_PLANE)
    sig = np.broadcast_to(np.asarray(sigma, dtype=np.float64), (7,)).copy()
    return dict(arm=arm, cost=cost, rb=rb, oc=oracle.make_cost(cost), q=q, qd=qd, goal=goal,
                plane=plane, K=K, T=T, dt=dt, lam=lam, sigma=sig, seed=SEED)


def gpu_controller(c: dict, **kw):
    from paper_2609_02020_b300 import mppi
    return mppi.MPPI(c["arm"], c["cost"], dt=c["dt"], T=c["T"], K=c["K"], lam=c["lam"],
                     sigma=c["sigma"], seed=c["seed"], **kw)


def oracle_step(c: dict, plan=None, it: int = 0, want_noise: bool = True, nthreads: int = 8,
                q=None, qd=None):
    T = c["T"]
    plan = np.zeros((T, 7)) if plan is None else f32(plan)
    return oracle.mppi_step(c["rb"], c["oc"], c["dt"], T, c["K"], c["lam"], c["sigma"], c["seed"],
                            it, c["q"] if q is None else q, c["qd"] if qd is None else qd,
                            c["goal"], c["plane"], plan, nthreads=nthreads,
                            want_noise=want_noise)


def noise_ktj(gpu_noise: np.ndarray, T: int, K: int) -> np.ndarray:
    """[T*7, K] as the library stores it -> [K, T, 7] as the oracle uses it."""
    return gpu_noise.reshape(T, 7, K).transpose(2, 0, 1).astype(np.float64)
