"""Parity of the wrench-estimate force cost (Eq. 12-13) on the GPU with the
FP64 oracle, through the C ABI.

F = Jbar^T (v - g(q)) is computed in FP32 by an LDL^T solve of M and of the
6 x 6 matrix A = J M^-1 J^T.  A backward-stable solve loses about
u * cond(A) in relative accuracy (u = 2^-24), so the direct comparison of F
allows 8 u cond_2(A) ||F||_inf + 1e-5 N per row (the 8 covers the errors of
forming A and b through the factors of M); rows near a kinematic singularity
(cond_2(A) > 1e4) are excluded there and compared only through costs.
Costs and plans keep the bars of the plain cost: S_k within 1e-4 relative,
plans within 1e-5 N m on workloads FP32 resolves; at heavier weights the
plan bar is a recorded miss, asserted at its measured size.
"""
import numpy as np
import pytest

import oracle
from paper_2609_02020_b300 import synth
from _common import f32, gpu_controller, make_case, oracle_step, parity_cost

pytestmark = pytest.mark.gpu

S_RTOL, S_ATOL = 1e-4, 1e-6
PLAN_TOL = 1e-5
U32 = 2.0 ** -24


def _pairs(n, seed):
    """(q, v) pairs over the joint range, torques around the gravity torque."""
    arm = synth.arm(seed, armature=0.1)
    rb = oracle.make_robot(arm)
    g = np.random.default_rng(seed)
    Q, V = np.zeros((n, 7)), np.zeros((n, 7))
    for i in range(n):
        q, _ = synth.state(10_000 * seed + i, arm)
        Q[i] = q
        V[i] = oracle.rnea(rb, q, np.zeros(7), np.zeros(7)) + g.normal(0.0, 10.0, 7)
    return arm, rb, f32(Q), f32(V)


def _cond_A(rb, arm, q):
    M = oracle.crba(rb, q) + np.diag(arm["armature"])
    J = oracle.jacobian(rb, q)
    return np.linalg.cond(J @ np.linalg.solve(M, J.T))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_force_estimate_matches_oracle(seed):
    import torch
    n = 1000
    arm, rb, Q, V = _pairs(n, seed)
    c = make_case(seed, cost=synth.cost_force_estimate())
    c["arm"] = arm
    with gpu_controller(c) as g:
        dq = torch.tensor(Q, dtype=torch.float32, device="cuda")
        dv = torch.tensor(V, dtype=torch.float32, device="cuda")
        dF = torch.full((n, 6), -1.0, device="cuda")
        g.force_estimate_device(dq, dv, dF)
        torch.cuda.synchronize()
        F = dF.cpu().numpy().astype(np.float64)
    checked = 0
    for i in range(n):
        rc, Fo = oracle.force_estimate(rb, Q[i], V[i])
        assert rc == 0
        kA = _cond_A(rb, arm, Q[i])
        if kA > 1e4:
            continue
        tol = 8 * U32 * kA * np.abs(Fo).max() + 1e-5
        err = np.abs(F[i] - Fo).max()
        assert err <= tol, (i, err, tol, kA)
        checked += 1
    assert checked >= 0.9 * n


def test_force_estimate_recovers_static_wrench():
    # tau = g(q) + J^T F: the device estimate returns F (no oracle involved
    # beyond J and g, which fix the input)
    import torch
    arm, rb, Q, _ = _pairs(64, 5)
    g = np.random.default_rng(5)
    Fw = g.normal(0.0, 10.0, (64, 6))
    V = np.stack([oracle.rnea(rb, Q[i], np.zeros(7), np.zeros(7)) + oracle.jacobian(rb, Q[i]).T @ Fw[i]
                  for i in range(64)])
    c = make_case(5, cost=synth.cost_force_estimate())
    c["arm"] = arm
    with gpu_controller(c) as h:
        dq = torch.tensor(Q, dtype=torch.float32, device="cuda")
        dv = torch.tensor(f32(V), dtype=torch.float32, device="cuda")
        dF = torch.empty((64, 6), device="cuda")
        h.force_estimate_device(dq, dv, dF)
        torch.cuda.synchronize()
        F = dF.cpu().numpy()
    for i in range(64):
        kA = _cond_A(rb, arm, Q[i])
        if kA > 1e4:
            continue
        # the input is rounded to FP32 too: |dv| <= u |v| moves F by cond-scaled u
        tol = 16 * U32 * kA * (np.abs(Fw[i]).max() + np.abs(V[i]).max()) + 1e-5
        assert np.abs(F[i] - Fw[i]).max() <= tol, i


def _hold_plan(c):
    tau_g = oracle.rnea(c["rb"], c["q"], np.zeros(7), np.zeros(7))
    return f32(np.tile(tau_g, (c["T"], 1)))


def _run_fest(c, plan, **kw):
    with gpu_controller(c, **kw) as g:
        g.set_plan(plan.astype(np.float32))
        tau0, nxt = g.step(c["q"], c["qd"], c["goal"], c["plane"])
        out = dict(tau0=tau0, plan=nxt, S=g.costs(), noise=g.noise(), ustar=g.updated_plan())
    o = oracle_step(c, plan=plan)
    return out, o


def _assert_costs(S_gpu, S_orc):
    err = np.abs(S_gpu.astype(np.float64) - S_orc)
    lim = S_RTOL * np.abs(S_orc) + S_ATOL
    bad = np.nonzero(err > lim)[0]
    assert bad.size == 0, f"{bad.size} costs off, worst rel {np.max(err / np.abs(S_orc)):.3e}"


# variant 2: the rolled kernel; 3: the warp-specialised kernel with the
# estimate on a fourth warp
@pytest.mark.parametrize("variant", [2, 3])
@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("contact", [False, True])
def test_fest_costs_match_oracle(seed, contact, variant):
    base = synth.cost_contact() if contact else synth.cost_free_space()
    c = make_case(seed, cost=synth.cost_force_estimate(base=base))
    g, o = _run_fest(c, _hold_plan(c), variant=variant)
    assert np.isfinite(o["S"]).all()
    _assert_costs(g["S"], o["S"])


@pytest.mark.parametrize("variant", [2, 3])
@pytest.mark.parametrize("seed", range(4))
def test_fest_plan_matches_oracle(seed, variant):
    # light force weight: S / lambda of a few tens, as for the plain parity workload
    c = make_case(seed, cost=synth.cost_force_estimate(1e-4, base=parity_cost()))
    g, o = _run_fest(c, _hold_plan(c), variant=variant)
    _assert_costs(g["S"], o["S"])
    assert np.abs(g["ustar"] - o["ustar"]).max() <= PLAN_TOL
    assert np.abs(g["plan"] - o["plan_next"]).max() <= PLAN_TOL


# Recorded miss of the 1e-5 N m plan bar at the heavier force weight
# (W_force 1e-3): S_k is hundreds of lambda with the weights on a few samples,
# where one FP32 ulp of S_k already moves u* by about 1e-5 N m (see the parity
# tests): measured max |du*| 3.8e-6 to 3.9e-5 N m (n_eff 1.0-32).  The
# bound guards the measured size.
HEAVY_MISS_BOUND = 1e-4


@pytest.mark.parametrize("variant", [2, 3])
@pytest.mark.parametrize("seed", range(4))
def test_fest_plan_recorded_miss_at_heavy_weights(seed, variant):
    c = make_case(seed, cost=synth.cost_force_estimate(1e-3))
    g, o = _run_fest(c, _hold_plan(c), variant=variant)
    _assert_costs(g["S"], o["S"])
    assert np.argmin(g["S"]) == np.argmin(o["S"])
    err = max(np.abs(g["ustar"] - o["ustar"]).max(), np.abs(g["plan"] - o["plan_next"]).max())
    print(f"force estimate W=1e-3 seed {seed}: max |du*| {err:.2e} N m, n_eff {o['stats'][2]:.2f}")
    assert err <= HEAVY_MISS_BOUND


@pytest.mark.parametrize("variant", [2, 3])
def test_fest_full_size_sampled(variant):
    # K = 16384, T = 18 in the benchmark's launch shape: sampled samples one by one
    c = make_case(7, cost=synth.cost_force_estimate(), K=16384)
    plan = _hold_plan(c)
    with gpu_controller(c, variant=variant) as g:
        g.set_plan(plan.astype(np.float32))
        g.step(c["q"], c["qd"], c["goal"], c["plane"])
        S = g.costs()
    ks = np.random.default_rng(7).choice(c["K"], 48, replace=False)
    for k in list(ks) + [0, c["K"] - 1]:
        So = oracle.rollout(c["rb"], c["oc"], c["dt"], c["T"], c["sigma"], c["seed"], 0, int(k),
                            c["q"], c["qd"], c["goal"], c["plane"], plan)
        assert abs(S[k] - So) <= S_RTOL * abs(So) + S_ATOL, k


@pytest.mark.parametrize("variant", [2, 3])
def test_fest_full_size_matches_oracle(variant):
    """K = 16384, T = 18 with plane contact and the wrench-estimate cost (the
    `--cost force_estimate` bench workload's sizes): all 16384 costs element
    by element against the oracle's whole update, the best sample, and the
    plan within the heavy-weight bound (S_min ~ 100 lambda here)."""
    import os
    c = make_case(7, cost=synth.cost_force_estimate(base=synth.cost_contact()), K=16384)
    plan = _hold_plan(c)
    o = oracle_step(c, plan=plan, want_noise=False, nthreads=os.cpu_count() or 8)
    with gpu_controller(c, variant=variant) as g:
        g.set_plan(plan.astype(np.float32))
        tau0, nxt = g.step(c["q"], c["qd"], c["goal"], c["plane"])
        S, us = g.costs(), g.updated_plan()
    assert np.isfinite(o["S"]).all()
    _assert_costs(S, o["S"])
    assert np.argmin(S) == np.argmin(o["S"])
    err = max(np.abs(us - o["ustar"]).max(), np.abs(nxt - o["plan_next"]).max())
    print(f"force estimate full size, variant {variant}: max |du*| {err:.2e} N m, "
          f"n_eff {o['stats'][2]:.1f}")
    assert err <= HEAVY_MISS_BOUND


@pytest.mark.parametrize("variant", [2, 3])
@pytest.mark.parametrize("K,T", [(1, 18), (33, 2), (77, 5), (1000, 1)])
def test_fest_ragged_sizes(K, T, variant):
    """Ragged K against the 32-sample blocks (the warp-specialised kernel's
    lanes past K replay sample K - 1 through its four warps) and short T:
    every cost and the best sample.  Around the gravity-holding plan these
    costs are 280-9000 lambda with the weights on one or two samples, the
    heavy-weight regime where the plan bar is a recorded miss, so the plan is
    left to the tests above."""
    c = make_case(3, cost=synth.cost_force_estimate(1e-4, base=parity_cost()), K=K, T=T)
    g, o = _run_fest(c, _hold_plan(c), variant=variant)
    _assert_costs(g["S"], o["S"])
    assert np.argmin(g["S"]) == np.argmin(o["S"])


@pytest.mark.parametrize("variant", [2, 3])
def test_fest_longest_horizon(variant):
    # T = 256 (MPPI_T_MAX) at dt = 1 ms: the warp-specialised kernel's shared
    # memory does not grow with T, the rolled kernel's does (opt-in above 48 KB)
    c = make_case(5, cost=synth.cost_force_estimate(1e-4, base=parity_cost()), K=64, T=256,
                  dt=0.001)
    g, o = _run_fest(c, _hold_plan(c), variant=variant)
    _assert_costs(g["S"], o["S"])
    assert np.argmin(g["S"]) == np.argmin(o["S"])


@pytest.mark.parametrize("variant", [2, 3])
@pytest.mark.parametrize("seed", range(2))
def test_fest_general_geometry(seed, variant):
    # oblique axes and products of inertia (synth.arm_general): the estimate's
    # Jacobian, g(q) and factors of M in the kernels' link frames
    c = make_case(seed, cost=synth.cost_force_estimate(base=synth.cost_contact()), general=True)
    g, o = _run_fest(c, _hold_plan(c), variant=variant)
    assert np.isfinite(o["S"]).all()
    _assert_costs(g["S"], o["S"])
    assert np.argmin(g["S"]) == np.argmin(o["S"])
