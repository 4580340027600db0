"""Learned proposal for torque-sampling MPPI.

Pipeline (every numerical step runs in the CUDA library):
  1. ``generate``: closed-loop episodes of plain MPPI (the paper's update)
     on the model used as a plant; every update gives one training pair
     x = (q, qd, goal, nominal plan u) -> y = u* - u (the correction plain
     MPPI makes to its nominal plan).  ``generate_on_policy`` adds pairs at
     the states and warm starts that MPPI with the learned proposal itself
     visits, labelled by plain MPPI (dataset aggregation, Ross et al.,
     AISTATS 2011), so that the network also sees where its own closed loop
     goes.
  2. ``train``: standardise x and y (statistics fitted by the library), then
     Adam on the mean squared error with the library's BF16 tensor-core
     (tcgen05) forward and backward kernels.
  3. ``LearnedMPPI``: each update samples most trajectories around the
     network's plan and the rest around the plain warm start (the fallback);
     the importance weights of Eq. 4a decide between them.
  4. ``evaluate``: closed-loop tracking cost, final position error and
     update latency of any controller on held-out episodes.
The torch tensors here are device buffers handed to the C ABI as pointers.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import mppi, synth


def n_in(T: int) -> int:
    return 21 + 7 * T


@dataclass
class Problem:
    """One arm and cost; the network is trained for this arm.  Episodes start
    at q ~ U(-start_range, start_range) (synth.state when start_range is 0)
    and aim at the end-effector pose of q + N(0, goal_spread) per joint."""
    arm: dict
    cost: dict
    T: int = 18
    dt: float = 0.01
    lam: float = 1.0
    sigma: float = 2.0
    substeps: int = 10
    plane: np.ndarray = field(default_factory=lambda: synth.NO_PLANE.copy())
    start_range: float = 0.0
    goal_spread: float = 0.6

    def controller(self, K: int, seed: int, stream=None) -> mppi.MPPI:
        return mppi.MPPI(self.arm, self.cost, dt=self.dt, T=self.T, K=K, lam=self.lam,
                         sigma=self.sigma, seed=seed, stream=stream)

    def hold_plan(self, helper: mppi.MPPI, q) -> np.ndarray:
        """Initial plan: the gravity-compensation torque at q over the horizon."""
        return np.tile(helper.gravity_torque(q), (self.T, 1)).astype(np.float32)

    def episode_start(self, seed: int, helper: mppi.MPPI):
        """Start state and a reachable goal: the end-effector pose of a
        configuration within N(0, goal_spread) rad per joint of the start (FK
        on the device)."""
        if self.start_range > 0.0:
            g0 = np.random.default_rng([seed, 78])
            q = g0.uniform(-self.start_range, self.start_range, 7)
            qd = g0.normal(0.0, 0.1, 7)
        else:
            q, qd = synth.state(seed, self.arm)
        g = np.random.default_rng([seed, 77])
        qg = np.clip(q + g.normal(0.0, self.goal_spread, 7), self.arm["q_min"], self.arm["q_max"])
        goal = helper.ee_pose(qg).astype(np.float64)
        return q, qd, goal


def tracking_problem(seed: int = 0) -> Problem:
    """The reaching task of the learned-proposal study, on which plain MPPI at
    K=16384 converges: a gravity-compensated arm (the commanded torque comes
    on top of the robot's own gravity compensation, as with a torque-controlled
    Franka arm: gravity 0 in model and plant), joint damping 5 N m s/rad,
    position-only goals (W_pos = 300, W_ori = 0, no posture term) reached
    from q ~ U(-1.2, 1.2) rad with goals 0.2 rad per joint away, sigma = 2 N m,
    lambda = 3."""
    arm = synth.arm(seed, damping=5.0)
    arm["gravity"] = np.zeros(3)
    cost = synth.cost_free_space()
    cost["w_pos"] = np.full(3, 300.0)
    cost["w_ori"] = np.zeros(3)
    cost["w_posture"] = 0.0
    return Problem(arm=arm, cost=cost, sigma=2.0, lam=3.0, start_range=1.2, goal_spread=0.2)


def generate(prob: Problem, n_pairs: int, *, K: int = 16384, seed: int = 0,
             episode_len: int = 200, stream=None):
    """Training pairs from plain MPPI: X [n, 21 + 7T], Y [n, 7T] (device);
    Y is the correction u* - u to the nominal plan held in X[:, 21:]."""
    import torch
    s = stream or torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctl = prob.controller(K, seed=0xD00D + seed, stream=s)
        X = torch.empty(n_pairs, n_in(prob.T), device="cuda")
        Y = torch.empty(n_pairs, 7 * prob.T, device="cuda")
        d_in = torch.empty(1, 25, device="cuda")
        d_tau = torch.empty(1, 7, device="cuda")
        d_x = torch.empty(1, 14, device="cuda")
        i, ep = 0, 0
        while i < n_pairs:
            q, qd, goal = prob.episode_start(1_000_000 * (seed + 1) + ep, ctl)
            d_in.copy_(torch.tensor(mppi.pack_inputs(q, qd, goal, prob.plane))[None])
            ctl.set_plan(prob.hold_plan(ctl, q))
            for _ in range(min(episode_len, n_pairs - i)):
                X[i, :21].copy_(d_in[0, :21])
                ctl.get_plan_device(X[i, 21:])
                ctl.step_device(d_in[0], d_tau[0], None)
                ctl.correction_device(Y[i])  # u* - u, formed by the library
                ctl.simulate_device(d_in, d_tau, d_x, prob.substeps)
                d_in[0, :14].copy_(d_x[0])
                i += 1
            ep += 1
        ctl.sync()
        s.synchronize()
        ctl.close()
    return X, Y


def generate_on_policy(prob: Problem, net: mppi.MLP, n_pairs: int, *, K_label: int,
                       K_learner: int, plain_frac: float = 0.5, seed: int = 0,
                       episode_len: int = 1000, stream=None):
    """Pairs at the states MPPI with the learned proposal visits: the learned
    controller (K_learner samples) drives the plant; at every update plain
    MPPI with K_label samples starts from the same state and the learned
    controller's warm start, and its correction u* - u is the label."""
    import torch
    s = stream or torch.cuda.Stream()
    with torch.cuda.stream(s):
        lc = LearnedMPPI(prob, net, K_learner, seed=0xA11CE + seed, stream=s,
                         plain_frac=plain_frac)
        ex = prob.controller(K_label, seed=0xBEEF + seed, stream=s)
        helper = prob.controller(1, seed=1, stream=s)
        X = torch.empty(n_pairs, n_in(prob.T), device="cuda")
        Y = torch.empty(n_pairs, 7 * prob.T, device="cuda")
        d_in = torch.empty(1, 25, device="cuda")
        d_tau = torch.empty(1, 7, device="cuda")
        d_tau_ex = torch.empty(1, 7, device="cuda")
        d_x = torch.empty(1, 14, device="cuda")
        plan = torch.empty(prob.T * 7, device="cuda")
        i, ep = 0, 0
        while i < n_pairs:
            q, qd, goal = prob.episode_start(3_000_000 * (seed + 1) + ep, helper)
            d_in.copy_(torch.tensor(mppi.pack_inputs(q, qd, goal, prob.plane))[None])
            lc.reset(prob.hold_plan(helper, q))
            for _ in range(min(episode_len, n_pairs - i)):
                X[i, :21].copy_(d_in[0, :21])
                lc.ctl.get_plan_device(plan)
                X[i, 21:].copy_(plan)
                ex.set_plan_device(plan)
                ex.step_device(d_in[0], d_tau_ex[0], None)
                ex.correction_device(Y[i])
                lc.step_device(d_in[0], d_tau[0])
                helper.simulate_device(d_in, d_tau, d_x, prob.substeps)
                d_in[0, :14].copy_(d_x[0])
                i += 1
            ep += 1
        ex.sync()
        s.synchronize()
        lc.close()
        ex.close()
        helper.close()
    return X, Y


def train(X, Y, *, steps: int = 4000, batch: int = 1024, lr: float = 1e-3, hidden: int = 256,
          layers: int = 3, seed: int = 0, val_frac: float = 0.05, stream=None):
    """Trains the proposal network; returns (net, info with train/val loss)."""
    import torch
    s = stream or torch.cuda.Stream()
    n = X.shape[0]
    nval = max(1, int(n * val_frac))
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    with torch.cuda.stream(s):
        perm = torch.randperm(n, device="cuda", generator=g)
        Xv, Yv = X[perm[:nval]].contiguous(), Y[perm[:nval]].contiguous()
        Xt, Yt = X[perm[nval:]].contiguous(), Y[perm[nval:]].contiguous()
        net = mppi.MLP(X.shape[1], hidden, layers, Y.shape[1], max_batch=max(batch, min(nval, 65536)),
                       seed=seed, stream=s)
        net.fit_normalization(Xt, Yt)  # per-feature means and deviations, on the device
        nt = Xt.shape[0]
        losses = []
        t0 = time.perf_counter()
        for it in range(steps):
            idx = torch.randint(0, nt, (batch,), device="cuda", generator=g)
            xb, yb = Xt[idx], Yt[idx]
            lr_t = lr * 0.5 * (1 + math.cos(math.pi * it / steps))
            want = (it % 500 == 0) or it == steps - 1
            l = net.train_step(xb, yb, max(lr_t, 1e-6), want_loss=want)
            if want:
                losses.append((it, l))
        s.synchronize()
        t_train = time.perf_counter() - t0
        vl, _ = net.loss_grad(Xv[:min(nval, 65536)], Yv[:min(nval, 65536)])
    return net, dict(train_loss=losses, val_loss=vl, seconds=t_train, steps=steps, batch=batch,
                     pairs=n)


class LearnedMPPI:
    """MPPI around the network's plan with the plain warm start beside it:
    n_plain of the K samples stay around the warm start (the fallback)."""

    def __init__(self, prob: Problem, net: mppi.MLP, K: int, *, seed: int, plain_frac: float = 0.25,
                 stream=None):
        self.ctl = prob.controller(K, seed=seed, stream=stream)
        self.net = net
        self.n_plain = int(round(K * plain_frac))

    def step_device(self, d_in, d_tau):
        self.net.propose_step_device(self.ctl, d_in, self.n_plain, d_tau)

    def reset(self, plan0):
        self.ctl.set_plan(plan0)

    def close(self):
        self.ctl.close()


class PlainMPPI:
    def __init__(self, prob: Problem, K: int, *, seed: int, stream=None):
        self.ctl = prob.controller(K, seed=seed, stream=stream)

    def step_device(self, d_in, d_tau):
        self.ctl.step_device(d_in, d_tau, None)

    def reset(self, plan0):
        self.ctl.set_plan(plan0)

    def close(self):
        self.ctl.close()


def _rot_angle(q1, q2):
    d = abs(float(np.dot(q1 / np.linalg.norm(q1), q2 / np.linalg.norm(q2))))
    return 2.0 * math.acos(min(1.0, d))


def evaluate(prob: Problem, controller, *, episodes: int, steps: int, seed: int, stream):
    """Closed loop on the model-as-plant: per-episode tracking cost (mean over
    steps of W_pos |dp|^2 + W_ori theta^2 at the plant's states), position and
    orientation errors over the last half, and the device time of each update
    (CUDA events on the controller's stream)."""
    import torch
    w_pos = float(np.mean(prob.cost["w_pos"]))
    w_ori = float(np.mean(prob.cost["w_ori"]))
    costs, pos_err, ori_err, lat_ms, fin_err = [], [], [], [], []
    tail = min(steps, max(1, int(round(1.0 / prob.dt))))  # the last second
    d_in = torch.empty(1, 25, device="cuda")
    d_tau = torch.empty(1, 7, device="cuda")
    d_x = torch.empty(1, 14, device="cuda")
    traj = torch.empty(steps, 14, device="cuda")
    helper = prob.controller(1, seed=1, stream=stream)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    with torch.cuda.stream(stream):
        for e in range(episodes):
            q, qd, goal = prob.episode_start(7_000_000 + seed * 1000 + e, helper)
            d_in.copy_(torch.tensor(mppi.pack_inputs(q, qd, goal, prob.plane))[None])
            controller.reset(prob.hold_plan(helper, q))
            for t in range(steps):
                ev0[t].record(stream)
                controller.step_device(d_in[0], d_tau[0])
                ev1[t].record(stream)
                helper.simulate_device(d_in, d_tau, d_x, prob.substeps)
                d_in[0, :14].copy_(d_x[0])
                traj[t].copy_(d_x[0])
            stream.synchronize()
            lat_ms += [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
            tr = traj.cpu().numpy()
            c, pe, oe, fe = 0.0, [], [], []
            for t in range(steps):
                pose = helper.ee_pose(tr[t, :7])
                dp = float(np.linalg.norm(pose[:3] - goal[:3]))
                th = _rot_angle(pose[3:], goal[3:])
                c += w_pos * dp * dp + w_ori * th * th
                if t >= steps // 2:
                    pe.append(dp)
                    oe.append(th)
                if t >= steps - tail:
                    fe.append(dp)
            costs.append(c / steps)
            pos_err.append(float(np.mean(pe)))
            ori_err.append(float(np.mean(oe)))
            fin_err.append(float(np.mean(fe)))
    helper.close()
    lat = np.array(lat_ms)
    return dict(tracking_cost=float(np.mean(costs)), tracking_cost_per_episode=costs,
                pos_err_m=float(np.mean(pos_err)), ori_err_rad=float(np.mean(ori_err)),
                final_err_m=float(np.median(fin_err)), final_err_per_episode=fin_err,
                within_2cm=float(np.mean(np.array(fin_err) < 0.02)),
                p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)))
