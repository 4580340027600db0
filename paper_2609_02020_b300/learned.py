"""Learned proposal for torque-sampling MPPI.

Pipeline (every numerical step runs in the CUDA library):
  1. ``generate``: closed-loop episodes of plain MPPI (the paper's update)
     on the model used as a plant; every update gives one training pair
     x = (q, qd, goal, nominal plan u) -> y = u* - u (the correction plain
     MPPI makes to its nominal plan).
  2. ``train``: standardise x and y, then Adam on the mean squared error with
     the library's BF16 tensor-core forward and backward kernels.
  3. ``LearnedMPPI``: each update samples most trajectories around the
     network's plan and the rest around the plain warm start (the fallback);
     the importance weights of Eq. 4a decide between them.
  4. ``evaluate``: closed-loop tracking cost and update latency of any
     controller on held-out episodes.
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
    """One arm and cost; the network is trained for this arm."""
    arm: dict
    cost: dict
    T: int = 18
    dt: float = 0.01
    lam: float = 1.0
    sigma: float = 2.0
    substeps: int = 10
    plane: np.ndarray = field(default_factory=lambda: synth.NO_PLANE.copy())

    def controller(self, K: int, seed: int, stream=None) -> mppi.MPPI:
        return mppi.MPPI(self.arm, self.cost, dt=self.dt, T=self.T, K=K, lam=self.lam,
                         sigma=self.sigma, seed=seed, stream=stream)

    def hold_plan(self, helper: mppi.MPPI, q) -> np.ndarray:
        """Initial plan: the gravity-compensation torque at q over the horizon."""
        return np.tile(helper.gravity_torque(q), (self.T, 1)).astype(np.float32)

    def episode_start(self, seed: int, helper: mppi.MPPI):
        """Start state and a reachable goal: the end-effector pose of a
        configuration within N(0, 0.6) rad per joint of the start (FK on the
        device)."""
        q, qd = synth.state(seed, self.arm)
        g = np.random.default_rng([seed, 77])
        qg = np.clip(q + g.normal(0.0, 0.6, 7), self.arm["q_min"], self.arm["q_max"])
        goal = helper.ee_pose(qg).astype(np.float64)
        return q, qd, goal


def generate(prob: Problem, n_pairs: int, *, K: int = 16384, seed: int = 0,
             episode_len: int = 100, stream=None):
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
                ctl.get_updated_plan_device(Y[i])
                Y[i].sub_(X[i, 21:])
                ctl.simulate_device(d_in, d_tau, d_x, prob.substeps)
                d_in[0, :14].copy_(d_x[0])
                i += 1
            ep += 1
        ctl.sync()
        s.synchronize()
        ctl.close()
    return X, Y


def standardisation(X, Y, floor: float = 1e-3):
    mx, sx = X.mean(0), X.std(0).clamp_min(floor)
    my, sy = Y.mean(0), Y.std(0).clamp_min(floor)
    return [t.cpu().numpy() for t in (mx, sx, my, sy)]


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
        net.set_normalization(*standardisation(Xt, Yt))
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
        self.net.propose(self.ctl, d_in, self.n_plain)
        self.ctl.step_device(d_in, d_tau, None)

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
    costs, pos_err, ori_err, lat_ms = [], [], [], []
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
            c, pe, oe = 0.0, [], []
            for t in range(steps):
                pose = helper.ee_pose(tr[t, :7])
                dp = float(np.linalg.norm(pose[:3] - goal[:3]))
                th = _rot_angle(pose[3:], goal[3:])
                c += w_pos * dp * dp + w_ori * th * th
                if t >= steps // 2:
                    pe.append(dp)
                    oe.append(th)
            costs.append(c / steps)
            pos_err.append(float(np.mean(pe)))
            ori_err.append(float(np.mean(oe)))
    helper.close()
    lat = np.array(lat_ms)
    return dict(tracking_cost=float(np.mean(costs)), tracking_cost_per_episode=costs,
                pos_err_m=float(np.mean(pos_err)), ori_err_rad=float(np.mean(ori_err)),
                p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)))
