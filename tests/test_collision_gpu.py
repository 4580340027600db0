"""Parity of the collision cost (Eq. 15) on the GPU with the FP64 oracle,
through the C ABI.

The squared-hinge form is continuous: S_k within 1e-4 relative, the plan
within 1e-5 N m at light weights, and a recorded miss of that bar, with its
measured size, where S / lambda is hundreds.  The indicator form turns each clearance
into a 0/1 decision; FP32 and FP64 may decide differently for a clearance
within rounding of its threshold.  There the sample's cost may differ by
whole multiples of w_collision, and only for samples whose FP64 trajectory
has such a near-threshold clearance (|d - d_th| <= 1e-4 m, far above the
FP32 error of d); everything else must agree to 1e-4 relative.
"""
import numpy as np
import pytest

import oracle
from paper_2609_02020_b300 import synth
from _common import f32, gpu_controller, make_case, oracle_step, parity_cost

pytestmark = pytest.mark.gpu

S_RTOL, S_ATOL = 1e-4, 1e-6
PLAN_TOL = 1e-5
NEAR = 1e-4


def _obstacles(seed, count=3):
    c = make_case(seed)
    return f32(synth.obstacles_near(oracle.link_points(c["rb"], c["q"]), seed, count))


def _case(seed, mode, K=256, w=10.0, base=None, obstacles=None, **kw):
    obs = _obstacles(seed) if obstacles is None else obstacles
    return make_case(seed, cost=synth.cost_collision(mode, w=w, base=base, obstacles=obs), K=K,
                     **kw)


def _run(c, plan=None, **kw):
    plan = np.zeros((c["T"], 7), np.float32) if plan is None else plan.astype(np.float32)
    with gpu_controller(c, **kw) as g:
        g.set_plan(plan)
        tau0, nxt = g.step(c["q"], c["qd"], c["goal"], c["plane"])
        out = dict(tau0=tau0, plan=nxt, S=g.costs(), noise=g.noise(), ustar=g.updated_plan())
    return out, oracle_step(c, plan=plan)


def _assert_costs(S_gpu, S_orc):
    err = np.abs(S_gpu.astype(np.float64) - S_orc)
    lim = S_RTOL * np.abs(S_orc) + S_ATOL
    bad = np.nonzero(err > lim)[0]
    assert bad.size == 0, f"{bad.size} costs off, worst rel {np.max(err / np.abs(S_orc)):.3e}"


def _near_threshold(c, plan, noise_k):
    """Whether the FP64 trajectory of one sample meets a clearance within
    NEAR of its threshold (replayed with the oracle's dynamics)."""
    rb, oc = c["rb"], c["oc"]
    n_self = 15
    q, qd = c["q"].copy(), c["qd"].copy()
    for t in range(c["T"]):
        qdd = oracle.forward_dynamics(rb, q, qd, plan[t] + noise_k[t])
        qd = qd + c["dt"] * qdd
        q = q + c["dt"] * qd
        d = oracle.collision_distances(rb, oc, q)
        th = np.where(np.arange(d.size) < n_self, oc.d_th_self, oc.d_th_obs)
        if np.min(np.abs(d - th)) <= NEAR:
            return True
    return False


# variant 0 runs the collision cost on the warp-specialised kernel's two
# extra warps at these sizes, variant 2 on the rolled kernel
@pytest.mark.parametrize("variant", [0, 2])
@pytest.mark.parametrize("seed", range(4))
def test_hinge_costs_match_oracle(seed, variant):
    c = _case(seed, 2)
    g, o = _run(c, variant=variant)
    _assert_costs(g["S"], o["S"])


@pytest.mark.parametrize("variant", [0, 2])
@pytest.mark.parametrize("seed", range(4))
def test_indicator_costs_match_oracle(seed, variant):
    w = 10.0
    c = _case(seed, 1, w=w)
    g, o = _run(c, variant=variant)
    # the workload exercises the indicator: it changes the cost of every sample
    o0 = oracle_step(make_case(seed))
    assert np.all(o["S"] - o0["S"] >= w)
    delta = g["S"].astype(np.float64) - o["S"]
    m = np.rint(delta / w)
    rest = np.abs(delta - m * w)
    assert np.all(rest <= S_RTOL * np.abs(o["S"]) + S_ATOL)
    plan = np.zeros((c["T"], 7))
    for k in np.nonzero(m)[0]:
        assert abs(m[k]) <= 2 and _near_threshold(c, plan, o["noise"][k]), k


@pytest.mark.parametrize("seed", range(3))
def test_hinge_plan_matches_oracle(seed):
    # light weights: S / lambda of a few tens, where FP32 resolves the plan
    c = _case(seed, 2, w=0.5, base=parity_cost())
    g, o = _run(c)
    _assert_costs(g["S"], o["S"])
    assert np.abs(g["ustar"] - o["ustar"]).max() <= PLAN_TOL
    assert np.abs(g["plan"] - o["plan_next"]).max() <= PLAN_TOL


# Recorded miss of the 1e-5 N m plan bar at the heavier collision weight
# (w = 10): S_k is hundreds of lambda with the weights on a few samples, where
# one FP32 ulp of S_k already moves u* by about 1e-5 N m (see the parity
# tests): measured max |du*| 5.8e-6 to 2.4e-5 N m (n_eff 1.2-4.3).  The
# bound guards the measured size.
HEAVY_MISS_BOUND = 1e-4


@pytest.mark.parametrize("seed", range(3))
def test_hinge_plan_recorded_miss_at_heavy_weights(seed):
    c = _case(seed, 2, w=10.0)
    g, o = _run(c)
    _assert_costs(g["S"], o["S"])
    assert np.argmin(g["S"]) == np.argmin(o["S"])
    err = max(np.abs(g["ustar"] - o["ustar"]).max(), np.abs(g["plan"] - o["plan_next"]).max())
    print(f"collision hinge w=10 seed {seed}: max |du*| {err:.2e} N m, n_eff {o['stats'][2]:.2f}")
    assert err <= HEAVY_MISS_BOUND


@pytest.mark.parametrize("device", [False, True])
def test_obstacles_replaced_between_updates(device):
    # created without obstacles; the second update (CUDA graph replay) must
    # see the obstacles set in between, the third none again
    import torch
    seed = 1
    obs = _obstacles(seed)
    c0 = _case(seed, 2, obstacles=np.zeros((0, 7)))
    c1 = _case(seed, 2, obstacles=obs)
    with gpu_controller(c0) as g:
        g.step(c0["q"], c0["qd"], c0["goal"], c0["plane"])
        S0 = g.costs()
        plan1 = g.get_plan()
        if device:
            d_obs = torch.tensor(obs, dtype=torch.float32, device="cuda")
            torch.cuda.synchronize()
            g.set_obstacles_device(d_obs)  # d_obs stays alive until the step has run
        else:
            g.set_obstacles(obs)
        g.step(c0["q"], c0["qd"], c0["goal"], c0["plane"])
        S1 = g.costs()
        plan2 = g.get_plan()
        g.set_obstacles(np.zeros((0, 7)))
        g.step(c0["q"], c0["qd"], c0["goal"], c0["plane"])
        S2 = g.costs()
    _assert_costs(S0, oracle_step(c0)["S"])
    _assert_costs(S1, oracle_step(c1, plan=plan1, it=1)["S"])
    _assert_costs(S2, oracle_step(c0, plan=plan2, it=2)["S"])


def test_collision_with_force_estimate():
    # both optional terms in one kernel
    seed = 2
    base = synth.cost_force_estimate(1e-3)
    c = _case(seed, 2, base=base)
    tau_g = oracle.rnea(c["rb"], c["q"], np.zeros(7), np.zeros(7))
    g, o = _run(c, plan=f32(np.tile(tau_g, (c["T"], 1))))
    _assert_costs(g["S"], o["S"])


def test_collision_full_size_sampled():
    # K = 16384, T = 18 in the benchmark's launch shape: sampled samples one by one
    c = _case(5, 2, K=16384)
    with gpu_controller(c) as g:
        assert g.variant() == 3
        g.step(c["q"], c["qd"], c["goal"], c["plane"])
        S = g.costs()
    plan = np.zeros((c["T"], 7))
    ks = np.random.default_rng(5).choice(c["K"], 40, replace=False)
    for k in list(ks) + [0, c["K"] - 1]:
        So = oracle.rollout(c["rb"], c["oc"], c["dt"], c["T"], c["sigma"], c["seed"], 0, int(k),
                            c["q"], c["qd"], c["goal"], c["plane"], plan)
        assert abs(S[k] - So) <= S_RTOL * abs(So) + S_ATOL, k


def test_long_horizon_shared_memory_opt_in():
    # T = 256 with both optional terms needs more than 48 KB of shared memory
    c = _case(0, 2, base=synth.cost_force_estimate(1e-4), T=256, dt=0.001, K=64)
    tau_g = oracle.rnea(c["rb"], c["q"], np.zeros(7), np.zeros(7))
    g, o = _run(c, plan=f32(np.tile(tau_g, (c["T"], 1))))
    _assert_costs(g["S"], o["S"])


@pytest.mark.parametrize("variant", [3, 2])
@pytest.mark.parametrize("K,T", [(1, 18), (33, 2), (77, 5), (1000, 1)])
def test_hinge_ragged_sizes(K, T, variant):
    """Ragged K against the 32-sample blocks (on the warp-specialised kernel
    the lanes past K replay sample K - 1 through all five warps) and short T;
    both collision warps' pair sets and the culled pairs included."""
    c = _case(1, 2, K=K, T=T)
    g, o = _run(c, variant=variant)
    _assert_costs(g["S"], o["S"])


@pytest.mark.parametrize("variant", [3, 2])
def test_hinge_general_geometry(variant):
    # off-axis joint offsets: the link capsules' rigid lengths come from the
    # general joint positions (synth.arm_general)
    c0 = make_case(1, general=True)
    obs = f32(synth.obstacles_near(oracle.link_points(c0["rb"], c0["q"]), 1, 3))
    c = make_case(1, cost=synth.cost_collision(2, w=10.0, obstacles=obs), general=True)
    g, o = _run(c, variant=variant)
    _assert_costs(g["S"], o["S"])
