"""Pins of the oracle's collision cost (Eq. 15).

The segment distance behind d_i is checked against brute-force minimisation
over the parameter square, closed forms (crossing, parallel, collinear and
degenerate segments) and its symmetries; the link capsules against the
rigid link lengths and the straight arm's closed-form clearances; the cost
against hand-counted indicator and hinge values; the rollout against a
replay of the trajectory.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation as Rot

import oracle
from paper_2609_02020_b300 import synth

RNG = np.random.default_rng(4242)


def brute_distance(p1, q1, p2, q2, n=401):
    s = np.linspace(0.0, 1.0, n)
    A = p1[None] + s[:, None] * (q1 - p1)[None]
    B = p2[None] + s[:, None] * (q2 - p2)[None]
    D = np.linalg.norm(A[:, None, :] - B[None, :, :], axis=2)
    return D.min()


@pytest.mark.parametrize("case", range(40))
def test_segment_distance_against_brute_force(case):
    g = np.random.default_rng(case)
    p1, q1, p2, q2 = (g.normal(0.0, 0.5, 3) for _ in range(4))
    if case % 5 == 0:            # nearly parallel
        q2 = p2 + (q1 - p1) * 0.7 + g.normal(0, 1e-3, 3)
    d = oracle.segment_distance(p1, q1, p2, q2)
    bf = brute_distance(p1, q1, p2, q2)
    # the grid minimum is an upper bound within the Lipschitz constant times
    # half a grid diagonal of the true minimum
    lip = np.linalg.norm(q1 - p1) + np.linalg.norm(q2 - p2)
    assert d <= bf + 1e-12
    assert d >= bf - lip * (1.0 / 400) * 0.75


def test_segment_distance_closed_forms():
    sd = oracle.segment_distance
    # perpendicular segments crossing at an offset: the offset
    assert sd([0, 0, 0], [1, 0, 0], [0.5, -1, 0.3], [0.5, 1, 0.3]) == pytest.approx(0.3, abs=1e-15)
    # parallel overlapping: the separation
    assert sd([0, 0, 0], [2, 0, 0], [1, 0.25, 0], [3, 0.25, 0]) == pytest.approx(0.25, abs=1e-15)
    # collinear disjoint: the gap
    assert sd([0, 0, 0], [1, 0, 0], [1.5, 0, 0], [4, 0, 0]) == pytest.approx(0.5, abs=1e-15)
    # skew, closest points at two endpoints
    assert sd([0, 0, 0], [1, 0, 0], [2, 1, 0], [3, 1, 0]) == pytest.approx(np.sqrt(2), abs=1e-15)
    # a point (degenerate segment) against a segment and against a point
    assert sd([0.5, 2, 0], [0.5, 2, 0], [0, 0, 0], [1, 0, 0]) == pytest.approx(2.0, abs=1e-15)
    assert sd([1, 2, 2], [1, 2, 2], [0, 0, 0], [0, 0, 0]) == pytest.approx(3.0, abs=1e-15)
    # intersecting segments: zero
    assert sd([-1, 0, 0], [1, 0, 0], [0, -1, 0], [0, 1, 0]) == pytest.approx(0.0, abs=1e-15)


@pytest.mark.parametrize("case", range(10))
def test_segment_distance_symmetries(case):
    g = np.random.default_rng(100 + case)
    p1, q1, p2, q2 = (g.normal(0.0, 0.5, 3) for _ in range(4))
    d = oracle.segment_distance(p1, q1, p2, q2)
    assert oracle.segment_distance(p2, q2, p1, q1) == pytest.approx(d, abs=1e-14)
    assert oracle.segment_distance(q1, p1, q2, p2) == pytest.approx(d, abs=1e-14)
    R = Rot.random(random_state=case).as_matrix()
    t = g.normal(0, 1, 3)
    m = [R @ x + t for x in (p1, q1, p2, q2)]
    assert oracle.segment_distance(*m) == pytest.approx(d, abs=1e-13)


def _coll_cost(mode=1, w=10.0, th_self=0.05, th_obs=0.2, obstacles=None):
    c = synth.cost_free_space()
    c.update(collision=mode, w_collision=w, d_th_self=th_self, d_th_obs=th_obs,
             link_radius=np.full(7, synth.ROD_RADIUS),
             obstacles=np.zeros((0, 7)) if obstacles is None else obstacles)
    return c


def test_link_points_are_rigid_and_straight_arm_clearances():
    d = synth.arm(3)
    rb = oracle.make_robot(d)
    lengths = np.linalg.norm(np.diff(oracle.link_points(rb, np.zeros(7)), axis=0), axis=1)
    np.testing.assert_allclose(lengths, d["length"], atol=1e-15)
    for s in range(4):
        q, _ = synth.state(s, d)
        L = np.linalg.norm(np.diff(oracle.link_points(rb, q), axis=0), axis=1)
        np.testing.assert_allclose(L, d["length"], atol=1e-12)
    # straight arm (q = 0): all links on the z axis; links i and j >= i + 2
    # are (sum of the lengths between them) apart, minus two radii
    c = oracle.make_cost(_coll_cost())
    dist = oracle.collision_distances(rb, c, np.zeros(7))
    want = []
    for i in range(7):
        for j in range(i + 2, 7):
            want.append(d["length"][i + 1:j].sum() - 2 * synth.ROD_RADIUS)
    np.testing.assert_allclose(dist, want, atol=1e-14)


def test_obstacle_clearance_and_indicator_by_hand():
    d = synth.arm(3)
    rb = oracle.make_robot(d)
    P = oracle.link_points(rb, np.zeros(7))
    # a sphere (a = b) beside the middle of link 3 at 0.25 m from its axis
    mid = 0.5 * (P[3] + P[4])
    r_obs = 0.05
    obs = np.array([[mid[0] + 0.25, mid[1], mid[2], mid[0] + 0.25, mid[1], mid[2], r_obs]])
    c = oracle.make_cost(_coll_cost(obstacles=obs))
    dist = oracle.collision_distances(rb, c, np.zeros(7))
    n_self = 15
    assert dist.size == n_self + 7
    assert dist[n_self + 3] == pytest.approx(0.25 - synth.ROD_RADIUS - r_obs, abs=1e-14)
    # the straight arm's self clearances exceed 0.05 only where a whole link
    # lies between; count the indicator hits by hand
    self_hits = sum(1 for x in dist[:n_self] if x < 0.05)
    obs_hits = sum(1 for x in dist[n_self:] if x < 0.2)
    assert obs_hits >= 1
    assert oracle.collision_cost(rb, c, np.zeros(7)) == pytest.approx(10.0 * (self_hits + obs_hits))
    # the squared-hinge reading
    c2 = oracle.make_cost(_coll_cost(mode=2, obstacles=obs))
    want = sum((0.05 - x) ** 2 for x in dist[:n_self] if x < 0.05) + \
        sum((0.2 - x) ** 2 for x in dist[n_self:] if x < 0.2)
    assert oracle.collision_cost(rb, c2, np.zeros(7)) == pytest.approx(10.0 * want, rel=1e-12)


@pytest.mark.parametrize("mode", [1, 2])
def test_rollout_charges_collision_at_next_state(mode):
    # S(with) - S(without) = sum_t C_collision(q_{t+1}) on a replayed trajectory
    d = synth.arm(4)
    rb = oracle.make_robot(d)
    q0, qd0 = synth.state(4, d)
    goal = synth.goal(4, d)
    P = oracle.link_points(rb, q0)
    obs = np.array([np.concatenate([P[5] + [0.1, 0.0, 0.0], P[5] + [0.1, 0.0, 0.2], [0.05]])])
    base = synth.cost_free_space()
    cc = dict(base, **_coll_cost(mode=mode, obstacles=obs))
    T, dt = 8, 0.01
    sigma = np.full(7, 2.0)
    plan = np.tile(oracle.rnea(rb, q0, np.zeros(7), np.zeros(7)), (T, 1))
    S1, noise = oracle.rollout(rb, oracle.make_cost(cc), dt, T, sigma, 9, 1, 5, q0, qd0, goal,
                               synth.NO_PLANE, plan, want_noise=True)
    S0 = oracle.rollout(rb, oracle.make_cost(base), dt, T, sigma, 9, 1, 5, q0, qd0, goal,
                        synth.NO_PLANE, plan)
    c1 = oracle.make_cost(cc)
    q, qd = q0.copy(), qd0.copy()
    extra = 0.0
    for t in range(T):
        qdd = oracle.forward_dynamics(rb, q, qd, plan[t] + noise[t], method=oracle.METHOD_ABA)
        qd = qd + dt * qdd
        q = q + dt * qd
        extra += oracle.collision_cost(rb, c1, q)
    assert extra > 0.0
    assert S1 - S0 == pytest.approx(extra, rel=1e-9, abs=1e-9)
