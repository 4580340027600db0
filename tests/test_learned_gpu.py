"""What the learned proposal gains over the method without it.

The network is trained on the GPU, by the library's own kernels, on
(state, goal, nominal plan) -> correction pairs that plain MPPI at K=16384
produces in closed loop.  Then, on held-out episodes (reachable goals,
gravity-compensated start), MPPI with the learned proposal at K=512 must
track with a clearly lower cost than plain MPPI at the same K=512 (and not
worse than plain MPPI at K=16384).
"""
import numpy as np
import pytest

from paper_2609_02020_b300 import learned, synth

pytestmark = pytest.mark.gpu


def tracking_problem():
    cost = synth.cost_free_space()
    cost["w_pos"] = np.full(3, 100.0)
    cost["w_ori"] = np.full(3, 10.0)
    return learned.Problem(arm=synth.arm(0), cost=cost)


def test_learned_proposal_beats_plain_mppi_at_equal_samples():
    import torch
    prob = tracking_problem()
    s = torch.cuda.Stream()
    X, Y = learned.generate(prob, 30000, K=16384, seed=0, stream=s)
    assert torch.isfinite(X).all() and torch.isfinite(Y).all()
    net, info = learned.train(X, Y, steps=3000, batch=1024, lr=1e-3, stream=s)
    assert info["train_loss"][-1][1] < info["train_loss"][0][1]
    res = {}
    for name, mk in [("plain512", lambda: learned.PlainMPPI(prob, 512, seed=5, stream=s)),
                     ("learned512", lambda: learned.LearnedMPPI(prob, net, 512, seed=5, stream=s)),
                     ("plain16384", lambda: learned.PlainMPPI(prob, 16384, seed=5, stream=s))]:
        c = mk()
        # 12 held-out episodes: closed-loop MPPI is sensitive to rounding, and
        # over 6 episodes the ratio below ranged 0.65-0.88 between builds
        # that differ only in summation order; over 12 it stays near 0.7
        res[name] = learned.evaluate(prob, c, episodes=12, steps=120, seed=1, stream=s)
        c.close()
    assert res["learned512"]["tracking_cost"] < 0.85 * res["plain512"]["tracking_cost"], res
    assert res["learned512"]["tracking_cost"] < 1.05 * res["plain16384"]["tracking_cost"], res
