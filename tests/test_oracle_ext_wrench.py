"""Pins of the oracle's constant external wrench (Eq. 5-6 as the paper states
them: tau_ext = J^T(q) F_ext, "constant over the prediction horizon").

  * the projection against virtual work, from finite differences of the
    forward kinematics alone (no Jacobian routine): tau_j = f . dp/dq_j +
    m . w_j, w_j the rotation rate of the end-effector frame per unit q_j;
  * constancy over the horizon and superposition: a rollout with the wrench
    and plan u costs what a rollout without it and plan u + tau_ext(q_0)
    costs (the torque-limit term off, since it sees the sampled torque);
  * a zero wrench changes nothing;
  * a planted mistake (the wrench projected at every step's q instead of at
    q_0) is caught by the superposition pin.
"""
import numpy as np
import pytest

import oracle
from paper_2609_02020_b300 import synth
from _common import SEED

pytestmark = pytest.mark.filterwarnings("ignore")


def _case(seed, f_ext, contact=False, **cost_kw):
    arm = synth.arm(seed)
    rb = oracle.make_robot(arm)
    q, qd = synth.state(1000 + seed, arm)
    goal = synth.goal(1000 + seed, arm)
    cost = synth.cost_contact() if contact else synth.cost_free_space()
    cost.update(cost_kw)
    cost["ext_wrench"] = 1
    cost["f_ext"] = np.asarray(f_ext, dtype=np.float64)
    plane = (synth.plane_through(oracle.fk(rb, q)[3][2], 0.02) if contact else synth.NO_PLANE)
    return arm, rb, cost, q, qd, goal, plane


def _log_so3(R):
    c = np.clip(0.5 * (np.trace(R) - 1.0), -1.0, 1.0)
    th = np.arccos(c)
    v = np.array([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]])
    return v * (0.5 if th < 1e-9 else th / (2.0 * np.sin(th)))


@pytest.mark.parametrize("seed", range(4))
def test_projection_matches_virtual_work(seed):
    rng = np.random.default_rng(seed)
    F = rng.normal(0.0, 5.0, 6)
    arm, rb, cost, q, _, _, _ = _case(seed, F)
    tau = oracle.ext_torque(rb, oracle.make_cost(cost), q)
    h = 1e-6
    ref = np.zeros(7)
    for j in range(7):
        dq = np.zeros(7)
        dq[j] = h
        _, _, Rp, pp = oracle.fk(rb, q + dq)
        _, _, Rm, pm = oracle.fk(rb, q - dq)
        dp = (pp - pm) / (2 * h)
        w = _log_so3(Rp @ Rm.T) / (2 * h)
        ref[j] = F[:3] @ dp + F[3:] @ w
    assert np.abs(tau - ref).max() <= 1e-6 * max(1.0, np.abs(ref).max()), (tau, ref)


def _rollout(rb, cost, q, qd, goal, plane, plan, k=0, T=18):
    return oracle.rollout(rb, oracle.make_cost(cost), 0.01, T, np.full(7, 2.0), SEED, 3, k, q, qd,
                          goal, plane, plan)


@pytest.mark.parametrize("contact", [False, True])
@pytest.mark.parametrize("seed", range(3))
def test_constant_over_horizon_by_superposition(seed, contact):
    rng = np.random.default_rng(10 + seed)
    F = rng.normal(0.0, 8.0, 6)
    arm, rb, cost, q, qd, goal, plane = _case(seed, F, contact=contact, w_tau=0.0)
    plan = rng.normal(0.0, 3.0, (18, 7))
    tau0 = oracle.ext_torque(rb, oracle.make_cost(cost), q)
    plain = dict(cost, ext_wrench=0)
    for k in (0, 5, 99):
        a = _rollout(rb, cost, q, qd, goal, plane, plan, k)
        b = _rollout(rb, plain, q, qd, goal, plane, plan + tau0, k)
        assert np.isfinite(a) and abs(a - b) <= 1e-10 * abs(b), (k, a, b)


def test_zero_wrench_changes_nothing():
    arm, rb, cost, q, qd, goal, plane = _case(2, np.zeros(6), contact=True)
    plan = np.random.default_rng(4).normal(0.0, 3.0, (18, 7))
    a = _rollout(rb, cost, q, qd, goal, plane, plan)
    b = _rollout(rb, dict(cost, ext_wrench=0), q, qd, goal, plane, plan)
    assert a == b


def test_superposition_pin_catches_a_per_step_projection():
    # the planted mistake, written here in Python on the oracle's own pieces:
    # projecting the wrench at each step's q moves the cost away from the
    # constant-tau_ext superposition by far more than rounding
    rng = np.random.default_rng(3)
    F = rng.normal(0.0, 8.0, 6)
    arm, rb, cost, q, qd, goal, plane = _case(1, F, w_tau=0.0)
    plan = rng.normal(0.0, 3.0, (18, 7))
    oc_plain = oracle.make_cost(dict(cost, ext_wrench=0))
    sig = np.full(7, 2.0)
    qq, qqd = q.copy(), qd.copy()
    S_wrong = 0.0
    for t in range(18):
        z = oracle.normals(SEED, 3, 0, t)[:7]
        v = plan[t] + sig * z
        tex = oracle.jacobian(rb, qq).T @ F
        qdd = oracle.forward_dynamics(rb, qq, qqd, v + tex)
        qqd = qqd + 0.01 * qdd
        qq = qq + 0.01 * qqd
        S_wrong += oracle.stage_cost(rb, oc_plain, goal, plane, qq, qqd, v)
    S_right = _rollout(rb, cost, q, qd, goal, plane, plan)
    assert abs(S_wrong - S_right) > 1e-6 * abs(S_right)
