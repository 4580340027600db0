"""Pins of the oracle's end-effector wrench estimate (Eq. 12-13).

F_ee = Jbar^T (v - g(q)) with Jbar = M^-1 J^T (J M^-1 J^T)^-1.  Each test
checks it against a property that the dynamically consistent inverse has by
construction, reached through another route than the oracle's own
CRBA + Cholesky evaluation: statics (a wrench held against gravity),
task-space dynamics through the articulated-body algorithm, null-space
torques built with RNEA, the square-Jacobian limit (Jbar^T = J^-T for any
M), and the index of the rollout step at which the cost is charged.
"""
import numpy as np
import pytest

import oracle
from paper_2609_02020_b300 import synth

from test_oracle_pins import random_robot

ZERO7 = np.zeros(7)


def _gravity(rb, q):
    return oracle.rnea(rb, q, np.zeros(rb.n), np.zeros(rb.n))


def _state(seed, d):
    q, _ = synth.state(seed, d)
    return q[: d["n"]]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_static_wrench_is_recovered(seed):
    # tau = g(q) + J^T F holds the arm against gravity while it pushes with F:
    # the estimate must return F for any M
    d = random_robot(100 + seed, armature=0.1)
    rb = oracle.make_robot(d)
    q = _state(seed, d)
    J = oracle.jacobian(rb, q)
    F = np.random.default_rng(seed).normal(0.0, 5.0, 6)
    rc, Fe = oracle.force_estimate(rb, q, _gravity(rb, q) + J.T @ F)
    assert rc == 0
    np.testing.assert_allclose(Fe, F, rtol=0, atol=1e-9 * (1 + np.abs(F).max()))


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_task_acceleration_matches_aba(seed):
    # defining property of Jbar: the estimated wrench, applied at the
    # end-effector, gives the end-effector the same acceleration (at qd = 0)
    # as the torque it was estimated from; accelerations come from the
    # articulated-body algorithm, not from CRBA + Cholesky
    d = random_robot(200 + seed, armature=0.05 * (seed + 1))
    rb = oracle.make_robot(d)
    q = _state(seed + 10, d)
    g = np.random.default_rng(seed)
    v = g.normal(0.0, 20.0, 7)
    rc, Fe = oracle.force_estimate(rb, q, v)
    assert rc == 0
    J = oracle.jacobian(rb, q)
    a_from_tau = J @ oracle.aba(rb, q, ZERO7, v)
    a_from_F = J @ oracle.aba(rb, q, ZERO7, _gravity(rb, q) + J.T @ Fe)
    np.testing.assert_allclose(a_from_F, a_from_tau, rtol=0,
                               atol=1e-9 * (1 + np.abs(a_from_tau).max()))


@pytest.mark.parametrize("seed", [0, 1])
def test_null_space_torque_gives_no_wrench(seed):
    # a torque that accelerates the joints only inside the null space of J
    # (built by RNEA from such an acceleration) produces no end-effector wrench
    d = random_robot(300 + seed, armature=0.1)
    rb = oracle.make_robot(d)
    q = _state(seed + 20, d)
    J = oracle.jacobian(rb, q)
    _, _, Vt = np.linalg.svd(J)
    qdd_null = 3.0 * Vt[-1]
    tau = oracle.rnea(rb, q, ZERO7, qdd_null) + d["armature"] * qdd_null
    rc, Fe = oracle.force_estimate(rb, q, tau)
    assert rc == 0
    assert np.abs(Fe).max() < 1e-9 * (1 + np.abs(tau).max())
    # and adding it to a pushing torque does not change the estimate
    F = np.array([3.0, -1.0, 10.0, 0.2, 0.0, -0.4])
    base = _gravity(rb, q) + J.T @ F
    _, F1 = oracle.force_estimate(rb, q, base + tau - _gravity(rb, q))
    np.testing.assert_allclose(F1, F, atol=1e-8)


def _six_joint(d):
    n = 6
    e = {k: (np.asarray(v)[:n] if isinstance(v, np.ndarray) and v.shape[:1] == (7,) else v)
         for k, v in d.items()}
    e["n"] = n
    return e


@pytest.mark.parametrize("scale", [1.0, 3.0])
def test_square_jacobian_gives_inverse_transpose(scale):
    # with six joints J is square, Jbar = J^-1 and F = J^-T (v - g) for any
    # mass distribution
    d = _six_joint(random_robot(400, armature=0.1))
    d["mass"] = d["mass"] * scale
    rb = oracle.make_robot(d)
    q = _state(5, random_robot(400))[:6]
    J = oracle.jacobian(rb, q)
    assert abs(np.linalg.det(J)) > 1e-4
    v = np.linspace(-8.0, 11.0, 6)
    rc, Fe = oracle.force_estimate(rb, q, v)
    assert rc == 0
    F_ref = np.linalg.solve(J.T, v - _gravity(rb, q))
    np.testing.assert_allclose(Fe, F_ref, rtol=1e-9, atol=1e-9)


def test_singular_configuration_is_reported():
    # the straight arm (q = 0) has its even joint axes on one line: J loses rank
    d = synth.arm(0)
    rb = oracle.make_robot(d)
    rc, Fe = oracle.force_estimate(rb, ZERO7, np.ones(7))
    assert rc == -1 and np.isnan(Fe).all()
    c = oracle.make_cost(dict(synth.cost_free_space(), force_estimate=1, w_force6=np.ones(6)))
    assert np.isnan(oracle.force_estimate_cost(rb, c, ZERO7, np.ones(7)))


def test_force_cost_by_hand():
    d = synth.arm(1)
    rb = oracle.make_robot(d)
    q = _state(1, d)
    J = oracle.jacobian(rb, q)
    F = np.array([1.0, -2.0, 12.0, 0.3, -0.1, 0.2])
    v = _gravity(rb, q) + J.T @ F
    w6 = np.array([0.0, 0.0, 2.0, 0.0, 0.0, 0.0])
    fd = np.array([0.0, 0.0, 10.0, 0.0, 0.0, 0.0])
    wr = np.array([0.5, 0.5, 0.0, 0.0, 0.0, 4.0])
    c = oracle.make_cost(dict(synth.cost_free_space(), force_estimate=1, w_force6=w6, f_des6=fd,
                              w_reg6=wr))
    want = 2.0 * (10.0 - 12.0) ** 2 + 0.5 * 1.0 + 0.5 * 4.0 + 4.0 * 0.04
    assert oracle.force_estimate_cost(rb, c, q, v) == pytest.approx(want, rel=1e-10)


@pytest.mark.parametrize("contact", [0, 1])
def test_rollout_charges_estimate_at_q_t(contact):
    # S(with the estimate) - S(without) = sum_t C_force(q_t, v_t), with q_t
    # from an Euler loop over the oracle's forward dynamics (ABA route); with
    # contact on, the normal-force term of Eq. 12 is replaced, not added
    d = synth.arm(2)
    rb = oracle.make_robot(d)
    q0, qd0 = synth.state(2, d)
    goal = synth.goal(2, d)
    base = dict(synth.cost_contact() if contact else synth.cost_free_space())
    plane = synth.plane_through(0.3) if contact else synth.NO_PLANE
    T, dt = 6, 0.01
    sigma = np.full(7, 2.0)
    plan = np.tile(_gravity(rb, q0), (T, 1))
    w6 = np.array([0.01, 0.01, 0.05, 0.1, 0.1, 0.1])
    fd = np.array([0.0, 0.0, -10.0, 0.0, 0.0, 0.0])
    wr = np.full(6, 1e-3)
    with_est = dict(base, force_estimate=1, w_force6=w6, f_des6=fd, w_reg6=wr)
    without = dict(base, w_force=0.0, w_reg=0.0)
    S1, noise = oracle.rollout(rb, oracle.make_cost(with_est), dt, T, sigma, 7, 3, 11, q0, qd0,
                               goal, plane, plan, want_noise=True)
    S0 = oracle.rollout(rb, oracle.make_cost(without), dt, T, sigma, 7, 3, 11, q0, qd0, goal,
                        plane, plan)
    c1 = oracle.make_cost(with_est)
    q, qd = q0.copy(), qd0.copy()
    extra = 0.0
    for t in range(T):
        v = plan[t] + noise[t]
        extra += oracle.force_estimate_cost(rb, c1, q, v)
        tex = oracle.contact(rb, c1, plane, q, qd)[1] if contact else np.zeros(7)
        qdd = oracle.forward_dynamics(rb, q, qd, v + tex, method=oracle.METHOD_ABA)
        qd = qd + dt * qdd
        q = q + dt * qd
    assert extra > 0.0
    assert S1 - S0 == pytest.approx(extra, rel=1e-9)
