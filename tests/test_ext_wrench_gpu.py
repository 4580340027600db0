"""The paper's constant external wrench (Eq. 5-6: tau_ext = J(q_0)^T F_ext,
constant over the horizon) on the GPU against the FP64 oracle, through the C
ABI: per-sample costs within 1e-4 relative and, at the parity weights, the
plan within 1e-5 N m, on all three rollout kernels; the wrench replaced
between updates (host and device setters, CUDA graph replay); the calls that
do not take it refuse it.
"""
import numpy as np
import pytest

import oracle
from paper_2609_02020_b300 import mppi, synth
from _common import gpu_controller, make_case, oracle_step, parity_cost

pytestmark = pytest.mark.gpu

S_RTOL, S_ATOL = 1e-4, 1e-6
PLAN_TOL = 1e-5


def _wrench(seed, scale=10.0):
    g = np.random.default_rng(500 + seed)
    return np.concatenate([g.normal(0.0, scale, 3), g.normal(0.0, 0.1 * scale, 3)])


def _with_wrench(cost, F):
    c = dict(cost)
    c.update(ext_wrench=1, f_ext=np.asarray(F, dtype=np.float64))
    return c


def _assert_costs(S_gpu, S_orc):
    err = np.abs(S_gpu.astype(np.float64) - S_orc)
    bad = np.nonzero(err > S_RTOL * np.abs(S_orc) + S_ATOL)[0]
    assert bad.size == 0, f"{bad.size} costs off, worst rel {np.max(err / np.abs(S_orc)):.3e}"


def _step(c, **kw):
    with gpu_controller(c, **kw) as g:
        tau0, plan = g.step(c["q"], c["qd"], c["goal"], c["plane"])
        return dict(tau0=tau0, plan=plan, S=g.costs(), ustar=g.updated_plan())


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("seed", range(4))
def test_costs_and_plan_match_oracle(seed, variant):
    c = make_case(seed, cost=_with_wrench(parity_cost(), _wrench(seed)))
    g = _step(c, variant=variant)
    o = oracle_step(c)
    _assert_costs(g["S"], o["S"])
    err = max(np.abs(g["ustar"] - o["ustar"]).max(), np.abs(g["plan"] - o["plan_next"]).max())
    print(f"external wrench seed {seed} variant {variant}: max |du*| {err:.2e} N m")
    assert err <= PLAN_TOL
    # the wrench moves the rollouts: the costs differ from the plain ones
    plain = oracle_step(make_case(seed, cost=parity_cost()))
    assert np.abs(plain["S"] - o["S"]).max() > 1e-3 * np.abs(o["S"]).max()


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("seed", range(2))
def test_costs_match_oracle_with_contact_and_estimate(seed, variant):
    """With the plane contact too, and (rolled and warp-specialised kernels)
    the wrench-estimate cost of Eq. 12-13: the paper's own combination of a
    measured wrench in the dynamics and the estimate in C_force."""
    cost = _with_wrench(synth.cost_contact(), _wrench(seed))
    if variant != 1:
        cost = synth.cost_force_estimate(base=cost)
    c = make_case(seed, cost=cost)
    g = _step(c, variant=variant)
    o = oracle_step(c)
    _assert_costs(g["S"], o["S"])
    assert np.argmin(g["S"]) == np.argmin(o["S"])


@pytest.mark.parametrize("device", [False, True])
def test_wrench_replaced_between_updates(device):
    import torch
    F1, F2 = _wrench(1), _wrench(2)
    c = make_case(3, cost=_with_wrench(parity_cost(), F1))
    with gpu_controller(c) as g:
        assert g.variant() == 3
        _, plan1 = g.step(c["q"], c["qd"], c["goal"], c["plane"])
        if device:
            g.set_external_wrench_device(torch.tensor(F2, dtype=torch.float32, device="cuda"))
        else:
            g.set_external_wrench(F2)
        _, plan2 = g.step(c["q"], c["qd"], c["goal"], c["plane"])
        S2, us2 = g.costs(), g.updated_plan()
    c2 = make_case(3, cost=_with_wrench(parity_cost(), np.asarray(F2, np.float32)))
    o2 = oracle_step(c2, plan=plan1, it=1)
    _assert_costs(S2, o2["S"])
    assert np.abs(us2 - o2["ustar"]).max() <= PLAN_TOL
    # the update used F2, not F1 (their costs differ by tens of lambda here)
    o1 = oracle_step(make_case(3, cost=_with_wrench(parity_cost(), np.asarray(F1, np.float32))),
                     plan=plan1, it=1)
    assert np.abs(o1["S"] - S2).max() > 1.0


def test_calls_that_do_not_take_it_refuse_it():
    import torch
    cost = _with_wrench(parity_cost(), _wrench(0))
    c = make_case(0, cost=cost, K=64, T=4)
    d_in = torch.tensor(mppi.pack_inputs(c["q"], c["qd"], c["goal"], c["plane"]), device="cuda")
    d_p = torch.zeros(c["T"], 7, device="cuda")
    d_u, d_n = torch.zeros_like(d_p), torch.zeros_like(d_p)
    with pytest.raises(mppi.MPPIError) as e:
        mppi.step_static(c["arm"], cost, dt=c["dt"], T=c["T"], K=c["K"], lam=c["lam"],
                         sigma=c["sigma"], seed=c["seed"], it=0, d_in=d_in, d_plan=d_p,
                         d_ustar=d_u, d_plan_next=d_n)
    assert e.value.code == mppi.ERR_INVALID_ARG
    with mppi.Server(pool_bytes=1 << 26, max_problems=4) as srv:
        with pytest.raises(mppi.MPPIError) as e:
            srv.add_problem(c["arm"], cost, dt=c["dt"], T=c["T"], K=c["K"], lam=c["lam"],
                            sigma=c["sigma"], seed=c["seed"])
        assert e.value.code == mppi.ERR_INVALID_ARG
    with gpu_controller(make_case(0, cost=parity_cost(), K=64, T=4)) as g:
        with pytest.raises(mppi.MPPIError) as e:
            g.set_external_wrench(np.zeros(6))
        assert e.value.code == mppi.ERR_INVALID_ARG
    with gpu_controller(c) as g:
        with pytest.raises(mppi.MPPIError) as e:
            g.set_external_wrench(np.array([0, 0, np.nan, 0, 0, 0]))
        assert e.value.code == mppi.ERR_INVALID_ARG
    bad = dict(cost, f_ext=np.array([0, 0, np.inf, 0, 0, 0]))
    with pytest.raises(mppi.MPPIError):
        gpu_controller(make_case(0, cost=bad, K=64, T=4))


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("K,T", [(1, 18), (33, 2), (77, 5)])
def test_ragged_sizes(K, T, variant):
    c = make_case(2, cost=_with_wrench(parity_cost(), _wrench(2)), K=K, T=T)
    g = _step(c, variant=variant)
    o = oracle_step(c)
    _assert_costs(g["S"], o["S"])
    assert np.abs(g["ustar"] - o["ustar"]).max() <= PLAN_TOL


@pytest.mark.parametrize("variant", [1, 2, 3])
def test_general_geometry(variant):
    c = make_case(0, cost=_with_wrench(parity_cost(), _wrench(0)), general=True)
    g = _step(c, variant=variant)
    o = oracle_step(c)
    _assert_costs(g["S"], o["S"])
    assert np.abs(g["ustar"] - o["ustar"]).max() <= PLAN_TOL
