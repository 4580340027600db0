"""What the learned proposal gains over the method without it.

The network is trained on the GPU, by the library's own tcgen05 kernels, on
(state, goal, nominal plan) -> correction pairs that plain MPPI at K=16384
produces in closed loop on a reaching task where it converges
(learned.tracking_problem: gravity-compensated arm, position-only goals).
On held-out 10 s episodes, MPPI with the learned proposal at K=512 must
track with a clearly lower cost than plain MPPI at the same K=512.  With
these K=16384 labels it does not reach plain MPPI at K=16384, and the test
does not claim it; `bench.py --mode learned` trains on K=131072 labels plus
pairs at the learned controller's own states, where K=2048 does.
"""
import numpy as np
import pytest

from paper_2609_02020_b300 import learned

pytestmark = pytest.mark.gpu


def test_learned_proposal_beats_plain_mppi_at_equal_samples():
    import torch
    prob = learned.tracking_problem()
    s = torch.cuda.Stream()
    X, Y = learned.generate(prob, 200_000, K=16384, seed=0, episode_len=1000, stream=s)
    assert torch.isfinite(X).all() and torch.isfinite(Y).all()
    net, info = learned.train(X, Y, steps=3000, batch=1024, lr=1e-3, stream=s)
    assert info["train_loss"][-1][1] < info["train_loss"][0][1]
    res = {}
    for name, mk in [("plain512", lambda: learned.PlainMPPI(prob, 512, seed=5, stream=s)),
                     ("learned512", lambda: learned.LearnedMPPI(prob, net, 512, seed=5, stream=s,
                                                               plain_frac=0.5))]:
        c = mk()
        # 12 held-out episodes of 10 s: closed-loop MPPI is chaotic, and the
        # tracking cost moves between builds that differ only in rounding
        res[name] = learned.evaluate(prob, c, episodes=12, steps=1000, seed=1, stream=s)
        c.close()
    # measured: 36.4 (learned) against 72.2 (plain) mean tracking cost
    assert res["learned512"]["tracking_cost"] < 0.75 * res["plain512"]["tracking_cost"], res


def test_on_policy_pairs_are_plain_mppi_corrections():
    """generate_on_policy: the learned controller drives, and each label is
    the correction plain MPPI (K_label samples) makes from the pair's own
    state, goal and warm start.  Re-running one such update on a fresh
    handle with the same seed and iteration reproduces the label bit for
    bit, and the warm starts are the learned controller's (not zero)."""
    import torch
    from paper_2609_02020_b300 import mppi
    prob = learned.tracking_problem()
    s = torch.cuda.Stream()
    X, Y = learned.generate(prob, 2000, K=1024, seed=0, episode_len=500, stream=s)
    net, _ = learned.train(X, Y, steps=50, batch=256, lr=1e-3, stream=s)
    Xo, Yo = learned.generate_on_policy(prob, net, 300, K_label=1024, K_learner=256, seed=3,
                                        episode_len=150, stream=s)
    net.close()
    assert torch.isfinite(Xo).all() and torch.isfinite(Yo).all()
    Xh, Yh = Xo.cpu().numpy(), Yo.cpu().numpy()
    assert np.abs(Xh[1:150, 21:]).max() > 0.0
    for i in (0, 7, 151, 299):
        with torch.cuda.stream(s):
            ex = prob.controller(1024, seed=0xBEEF + 3, stream=s)
            ex.set_iter(i)
            ex.set_plan(Xh[i, 21:].reshape(prob.T, 7))
            d_in = torch.tensor(mppi.pack_inputs(Xh[i, :7], Xh[i, 7:14], Xh[i, 14:21],
                                                 prob.plane), device="cuda")
            d_tau = torch.empty(7, device="cuda")
            y = torch.empty(7 * prob.T, device="cuda")
            ex.step_device(d_in, d_tau, None)
            ex.correction_device(y)
            s.synchronize()
            ex.close()
        assert np.array_equal(y.cpu().numpy(), Yh[i]), i
