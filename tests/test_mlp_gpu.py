"""The learned proposal's BF16 tensor-core kernels against the FP64 oracle.

Tolerance: the oracle rounds to BF16 at the same points as the kernels
(weights, layer inputs, loss gradient, back-propagated deltas), so the sides
differ by FP32 accumulation order and by the rare BF16 rounding decision that
this order flips.  A flip moves one element by 2^-8 relative, which shifts a
whole tensor by about 1e-4 in relative Frobenius norm.  The bounds below are
2e-3 (forward) and 5e-3 (each gradient tensor).
"""
import numpy as np
import pytest

import oracle
from paper_2609_02020_b300 import mppi, synth

pytestmark = pytest.mark.gpu

DIMS = [147, 256, 256, 256, 126]
RNG = np.random.default_rng(11)


def rel_fro(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def layer_slices(dims):
    out, off = [], 0
    for l in range(1, len(dims)):
        nw = dims[l] * dims[l - 1]
        out.append((f"W{l}", slice(off, off + nw)))
        out.append((f"b{l}", slice(off + nw, off + nw + dims[l])))
        off += nw + dims[l]
    return out


def net(**kw):
    return mppi.MLP(147, 256, 3, 126, max_batch=256, seed=kw.pop("seed", 3), **kw)


def test_forward_matches_oracle():
    import torch
    m = net()
    P = m.get_params().astype(np.float64)
    X = RNG.normal(size=(100, 147)).astype(np.float32)
    dX = torch.tensor(X, device="cuda")
    dY = torch.zeros(100, 126, device="cuda")
    m.forward(dX, dY)
    torch.cuda.synchronize()  # the network's work is queued on its own stream
    ref = oracle.mlp_forward(DIMS, P, X.astype(np.float64), bf16=True)
    assert rel_fro(dY.cpu().numpy(), ref) <= 2e-3


@pytest.mark.parametrize("n", [1, 77, 256])
def test_gradients_match_oracle(n):
    import torch
    m = net(seed=5)
    P = m.get_params().astype(np.float64)
    X = RNG.normal(size=(n, 147)).astype(np.float32)
    Yt = RNG.normal(size=(n, 126)).astype(np.float32)
    loss, g = m.loss_grad(torch.tensor(X, device="cuda"), torch.tensor(Yt, device="cuda"))
    lo, go = oracle.mlp_loss_grad(DIMS, P, X.astype(np.float64), Yt.astype(np.float64), bf16=True)
    assert abs(loss - lo) <= 1e-3 * lo
    for name, sl in layer_slices(DIMS):
        assert rel_fro(g[sl], go[sl]) <= 5e-3, name
    # and against the unrounded FP64 gradient the BF16 error is of the BF16 order
    _, g64 = oracle.mlp_loss_grad(DIMS, P, X.astype(np.float64), Yt.astype(np.float64), bf16=False)
    assert rel_fro(g, g64) <= 3e-2


def test_standardisation_is_applied():
    import torch
    m = net(seed=6)
    P = m.get_params().astype(np.float64)
    mi, si = RNG.normal(size=147), RNG.uniform(0.5, 2.0, 147)
    mo, so = RNG.normal(size=126), RNG.uniform(0.5, 2.0, 126)
    m.set_normalization(mi, si, mo, so)
    X = RNG.normal(size=(40, 147)).astype(np.float32) * 3
    dY = torch.zeros(40, 126, device="cuda")
    m.forward(torch.tensor(X, device="cuda"), dY)
    torch.cuda.synchronize()
    Xs = (X.astype(np.float64) - mi.astype(np.float32)) / si.astype(np.float32)
    ref = oracle.mlp_forward(DIMS, P, Xs, bf16=True) * so.astype(np.float32) + mo.astype(np.float32)
    assert rel_fro(dY.cpu().numpy(), ref) <= 2e-3


def test_training_fits_a_teacher_network():
    import torch
    teacher = oracle.mlp_num_params(DIMS)
    Pt = RNG.normal(0, 0.08, teacher)
    X = RNG.normal(size=(4096, 147))
    Y = oracle.mlp_forward(DIMS, Pt, X)
    m = net(seed=9)
    dX = torch.tensor(X, dtype=torch.float32, device="cuda")
    dY = torch.tensor(Y, dtype=torch.float32, device="cuda")
    first = m.train_step(dX[:256], dY[:256], 1e-3, want_loss=True)
    for it in range(600):
        i = (it * 256) % 4096
        m.train_step(dX[i:i + 256], dY[i:i + 256], 1e-3)
    last = m.train_step(dX[:256], dY[:256], 1e-3, want_loss=True)
    assert last < 0.2 * first


def test_propose_installs_the_network_plan_as_second_proposal():
    """propose(ctl, d_in, n_plain) gives the same update as installing the
    nominal plan plus the network's output by hand with set_proposal_device
    (costs, tau0 and plan within FP32 rounding of the fused kernel)."""
    import torch
    arm = synth.arm(0)
    q, qd = synth.state(1000, arm)
    goal = synth.goal(1000, arm)
    T = 18
    kw = dict(dt=0.01, T=T, K=512, lam=1.0, sigma=2.0, seed=1)
    plan0 = RNG.normal(0, 3, (T, 7)).astype(np.float32)
    m = net(seed=4)
    d_in = torch.tensor(mppi.pack_inputs(q, qd, goal), device="cuda")
    x = np.concatenate([mppi.pack_inputs(q, qd, goal)[:21], plan0.ravel()])[None]
    dY = torch.zeros(1, 126, device="cuda")
    m.forward(torch.tensor(x, device="cuda"), dY)
    torch.cuda.synchronize()
    res = []
    for by_hand in (False, True):
        ctl = mppi.MPPI(arm, synth.cost_free_space(), **kw)
        ctl.set_plan(plan0)
        if by_hand:
            # the network predicts the correction to the nominal plan
            ctl.set_proposal_device(dY.view(T, 7) + torch.tensor(plan0, device="cuda"), 200)
        else:
            m.propose(ctl, d_in, 200)
        tau0, plan = ctl.step(q, qd, goal)
        res.append((tau0, plan, ctl.costs()))
        ctl.close()
    for a, b in zip(res[0], res[1]):
        assert np.allclose(a, b, rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("variant", [0, 2])
@pytest.mark.parametrize("K,n_plain", [(512, 200), (2048, 0), (2048, 1000), (2048, 2048),
                                       (16384, 8192), (16384, 5001)])
def test_fused_propose_step_matches_the_two_calls(K, n_plain, variant):
    """propose_step_device gives, bit for bit, the updates of propose followed
    by step_device: tau0, the shifted plan, u* and the costs over three
    warm-started updates.  Variant 0 is the warp-specialised kernel (the
    small-K and the default instantiation), whose plain blocks overlap the
    proposal; the rolled kernel (variant 2) waits for it as usual."""
    import torch
    arm = synth.arm(0)
    T = 18
    m = net(seed=5)
    g = np.random.default_rng(K + n_plain)
    plan0 = g.normal(0, 3, (T, 7)).astype(np.float32)
    states = [synth.state(1100 + i, arm) for i in range(3)]
    goal = synth.goal(1100, arm)
    res = []
    for fused in (False, True):
        ctl = mppi.MPPI(arm, synth.cost_contact(), dt=0.01, T=T, K=K, lam=1.0, sigma=2.0,
                        seed=3, variant=variant)
        assert variant == 2 or ctl.variant() == 3
        ctl.set_plan(plan0)
        out = []
        for q, qd in states:
            d_in = torch.tensor(mppi.pack_inputs(q, qd, goal), device="cuda")
            d_tau = torch.zeros(7, device="cuda")
            if fused:
                m.propose_step_device(ctl, d_in, n_plain, d_tau)
            else:
                m.propose(ctl, d_in, n_plain)
                ctl.step_device(d_in, d_tau)
            assert ctl.sync() == mppi.OK
            out.append((d_tau.cpu().numpy(), ctl.get_plan(), ctl.updated_plan(), ctl.costs()))
        res.append(out)
        ctl.close()
    for a_step, b_step in zip(*res):
        for a, b in zip(a_step, b_step):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("cost", ["force_estimate", "collision"])
def test_fused_propose_step_with_the_optional_costs(cost):
    """With the wrench-estimate or collision cost the warp-specialised rollout
    waits for the proposal kernel as usual; the one call still gives the two
    calls' update bit for bit."""
    import torch
    arm = synth.arm(1)
    T, K, n_plain = 18, 2048, 1000
    c = (synth.cost_force_estimate() if cost == "force_estimate" else
         synth.cost_collision(obstacles=[[0.3, 0.0, 0.5, 0.3, 0.15, 0.55, 0.05],
                                         [0.0, 0.35, 0.4, 0.1, 0.35, 0.4, 0.04]]))
    m = net(seed=6)
    q, qd = synth.state(1200, arm)
    d_in = torch.tensor(mppi.pack_inputs(q, qd, synth.goal(1200, arm)), device="cuda")
    res = []
    for fused in (False, True):
        ctl = mppi.MPPI(arm, c, dt=0.01, T=T, K=K, lam=1.0, sigma=2.0, seed=2)
        assert ctl.variant() == 3
        d_tau = torch.zeros(7, device="cuda")
        if fused:
            m.propose_step_device(ctl, d_in, n_plain, d_tau)
        else:
            m.propose(ctl, d_in, n_plain)
            ctl.step_device(d_in, d_tau)
        assert ctl.sync() == mppi.OK
        res.append((d_tau.cpu().numpy(), ctl.get_plan(), ctl.costs()))
        ctl.close()
    for a, b in zip(*res):
        assert np.array_equal(a, b)


def test_fused_propose_step_rejects_bad_arguments():
    import torch
    arm = synth.arm(0)
    m = net()
    ctl = mppi.MPPI(arm, synth.cost_free_space(), dt=0.01, T=18, K=256, lam=1.0, sigma=2.0, seed=1)
    try:
        d_in = torch.zeros(25, device="cuda")
        for bad in (-1, 257):
            with pytest.raises(mppi.MPPIError) as e:
                m.propose_step_device(ctl, d_in, bad)
            assert e.value.code == mppi.ERR_INVALID_ARG
        with pytest.raises(mppi.MPPIError) as e:
            m.propose_step_device(ctl, None, 0)
        assert e.value.code == mppi.ERR_INVALID_ARG
        assert ctl.get_iter() == 0  # nothing was queued
    finally:
        ctl.close()
        m.close()


def test_bounded_wait_reports_timeout():
    # one mbarrier wait that nothing completes, given up after about 1 ms of
    # SM clock through the GEMMs' wait helper and error flag: the status is
    # TIMEOUT, the flag is cleared, and the context stays usable
    import torch
    m = net()
    try:
        assert m.check_wait(2_000_000) == mppi.ERR_TIMEOUT
        assert m.check_wait(0) == mppi.ERR_INVALID_ARG
        dX = torch.tensor(RNG.normal(size=(8, 147)).astype(np.float32), device="cuda")
        dY = torch.zeros(8, 126, device="cuda")
        m.forward(dX, dY)
        torch.cuda.synchronize()
        assert torch.isfinite(dY).all()
    finally:
        m.close()
