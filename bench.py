"""Benchmark: rollout-steps/s and MPPI update latency, 7-DoF arm, K=16384, T=18.

One step = one full MPPI update (K rollouts of T steps with dynamics, contact
and costs, then the Eq. 4 update and the shift) of a seeded 7-joint arm with
plane contact, dt = 0.01 s.  Prints one JSON line on rank 0.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--cost contact|force_estimate|collision]
                    [--mode update|serve|learned|sweep|mlp]

`value` times the update on device-resident inputs with CUDA events on the
library's stream, L2 flushed between steps; `e2e` times the public host call
mppi_step (inputs copied from pinned host memory, tau0 and the plan read back)
with a host clock.  `--impl reference` times the FP64 CPU oracle on the host
cores on a bounded sample of the same workload.  With N > 1 (torchrun) every
rank solves its own independent problem (replicas, weak scaling).
`--cost` swaps the update's cost for the same workload with C_force on the
wrench estimate of Eq. 13, or with the collision indicator of Eq. 15 against
three obstacles near the end-effector (the default line is the contact cost).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rollout-steps/s and MPPI update p50/p99 ms, 7-DoF K=16384 T=18, vs plain"
UNIT = "rollout-steps/s"
K_DEFAULT, T_DEFAULT, DT = 16384, 18, 0.01
SIGMA, LAMBDA, SEED = 2.0, 1.0, 0xC0FFEE
L2_FLUSH_BYTES = 256 << 20  # twice the 126 MB L2

# Algorithmic FP32 operations of one rollout-step (one sample advanced by one
# step) of the contact workload, counted by hand on the formulation the
# kernels run (world-frame RNEA + CRBA + LDL^T; an FMA counts 2, structural
# zeros are not counted, special functions - sin/cos, log, sqrt, atan2,
# reciprocals - are listed apart and not counted):
#   forward sweep, 7 links x 380 (frame 90, motion 48, inertia + force 242)
#     + end-effector pose and velocity 75                             2735
#   backward sweep: suffix sums 96, h 91, composite momenta 294, M 315  796
#   LDL^T factor 154 + two triangular solves 91                          245
#   contact force and tau_ext = J^T F_ext (contact active)               124
#   running cost: motion 81, force 7, joint hinges 133, sum 2            223
#   noise: Box-Muller arithmetic 76, v = u + sigma z 14                   90
#   compensated Euler step (Eq. 7), 7 joints x 12                         84
#   this block's share of Eq. 4 (N_b sums: 126 x 2 / 18)                  14
#                                                                 total 4311
# Each term counts the operations of the helpers in csrc/mppi_device.cuh that
# carry it, structural zeros left out.  The executed count of
# the warp-specialised kernel (ncu FADD + FMUL + 2 FFMA, special functions'
# polynomials included) is kept beside it.  The optional cost terms have no
# hand count; their lines use the executed count and say so.
FLOP_PER_ROLLOUT_STEP = {"contact": 4311.0}
FLOP_EXECUTED_PER_ROLLOUT_STEP = {("contact", "rollout_kernel_ws"): 4970.2,
                                  ("force_estimate", "rollout_kernel_ws_fest"): 6159.1,
                                  ("force_estimate", "rollout_kernel_rolled"): 6167.6,
                                  ("collision", "rollout_kernel_ws"): 6500.2}
# DRAM read + write bytes of one rollout launch at K=16384, T=18 per (cost,
# kernel) (ncu dram__bytes_{read,write}.sum, mean of two launches).  The
# 8.3 MB of stored noise stays in L2 and is not written back inside the
# launch.
# Only kernels captured since their last change are listed; the others
# report null.
ROLLOUT_TRAFFIC_BYTES_PER_LAUNCH = {("contact", "rollout_kernel_ws"): 65024,
                                    ("force_estimate", "rollout_kernel_ws_fest"): 72832,
                                    ("force_estimate", "rollout_kernel_rolled"): 67840,
                                    ("collision", "rollout_kernel_ws"): 131072}
COSTS = ("contact", "force_estimate", "collision")
SM_COUNT = 148
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--K", type=int, default=K_DEFAULT)
    ap.add_argument("--T", type=int, default=T_DEFAULT)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true",
                    help="update mode: skip the learned-proposal latency sub-object")
    ap.add_argument("--no-serve", action="store_true",
                    help="update mode: leave out the compact serving measurement")
    ap.add_argument("--budget-s", type=float, default=120.0,
                    help="reference arm: wall-clock budget of the whole run [s]")
    ap.add_argument("--variant", type=int, default=0,
                    help="rollout kernel: 0 library default, 1 unrolled, 2 rolled, "
                         "3 warp-specialised")
    ap.add_argument("--cost", default="contact", choices=list(COSTS),
                    help="update mode: the plane-contact workload (default), or the same with "
                         "C_force on the wrench estimate of Eq. 13, or with the collision "
                         "indicator of Eq. 15 against 3 obstacles")
    ap.add_argument("--mode", default="update", choices=["update", "serve", "learned", "sweep", "mlp"],
                    help="update: the headline single-update benchmark; serve: batched "
                         "serving of 256 problems under Poisson load; learned: train the "
                         "learned proposal and compare it with plain MPPI; sweep: the update "
                         "over K x T with FP32 and FP64 reductions; mlp: the learned "
                         "proposal's network kernels alone")
    ap.add_argument("--pairs", type=int, default=200_000, help="learned mode: training pairs")
    ap.add_argument("--train-steps", type=int, default=3000, help="learned mode: Adam steps")
    ap.add_argument("--label-k", type=int, default=131072,
                    help="learned mode: samples of the plain MPPI that labels the pairs")
    ap.add_argument("--on-policy-rounds", type=int, default=1,
                    help="learned mode: rounds of pairs at the learned controller's own states")
    ap.add_argument("--on-policy-pairs", type=int, default=100_000,
                    help="learned mode: pairs per on-policy round")
    ap.add_argument("--episodes", type=int, default=12, help="learned mode: eval episodes")
    ap.add_argument("--plain-fracs", default="0.5",
                    help="learned mode: comma-separated shares of the samples kept around the "
                         "plain warm start, one set of learned rows each")
    ap.add_argument("--rates", default="2000,5000,10000,20000,100000",
                    help="serve mode: arrival rates [updates/s]")
    ap.add_argument("--seconds", type=float, default=2.0, help="serve mode: seconds per rate")
    ap.add_argument("--problems", type=int, default=256, help="serve mode: problems")
    ap.add_argument("--pool-mb", type=int, default=1024, help="serve mode: scratch pool [MiB]")
    return ap.parse_args()


def max_over_ranks(values, world: int, device: str):
    """Element-wise maximum of `values` over all ranks (the slowest rank's
    times); the identity for a single rank."""
    if world <= 1:
        return list(values)
    import torch
    import torch.distributed as dist
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def workload(rank: int, cost_name: str = "contact"):
    """Arm, cost (without obstacles), state and goal of one rank's problem."""
    from paper_2609_02020_b300 import synth
    arm = synth.arm(rank)
    q, qd = synth.state(1000 + rank, arm)
    goal = synth.goal(1000 + rank, arm)
    cost = synth.cost_contact()
    if cost_name == "force_estimate":
        cost = synth.cost_force_estimate(base=cost)
    elif cost_name == "collision":
        cost = synth.cost_collision(1, base=cost)
    return arm, cost, q, qd, goal


def obstacles(rank: int, arm: dict, p_ee):
    """Three capsule obstacles 0.12-0.3 m from the end-effector point."""
    from paper_2609_02020_b300 import synth
    pts = np.array([[0.0, 0.0, synth.BASE_HEIGHT], np.asarray(p_ee, float)])
    return synth.obstacles_near(pts, 1000 + rank, 3)


COST_TEXT = {"contact": "plane contact",
             "force_estimate": "plane contact and C_force on the wrench estimate (Eq. 13)",
             "collision": "plane contact and the collision indicator (Eq. 15), 3 obstacles"}


def config_dict(K, T, n, cost_name="contact"):
    return {"workload": f"7-DoF seeded arm, one MPPI update with {COST_TEXT[cost_name]}, "
                        f"K={K} T={T} dt={DT} s, sigma={SIGMA} N m, lambda={LAMBDA}",
            "K": K, "T": T, "dt": DT, "cost": cost_name,
            "robots": "synthetic 7-joint arms (seeded)",
            "l2": "flushed between timed steps", "parallelism": f"replicas x{n}"}


def oracle_problem(K: int, T: int, cost_name: str):
    """The oracle's records of rank 0's problem (plane, obstacles included)."""
    import oracle
    from paper_2609_02020_b300 import synth
    arm, cost, q, qd, goal = workload(0, cost_name)
    rb = oracle.make_robot(arm)
    pe = oracle.fk(rb, q)[3]
    if cost_name == "collision":
        cost = dict(cost, obstacles=obstacles(0, arm, pe))
    plane = synth.plane_through(pe[2])
    return rb, oracle.make_cost(cost), q, qd, goal, plane


# ---------------------------------------------------------------------------
# clocks sampled during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
            t0 = time.time()
            while not self.rows and time.time() - t0 < 10.0 and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def mark(self):
        """Index of the next sample: rows from here on fall in the timed region."""
        return len(self.rows)

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, spans=None):
        rows = self.rows if not spans else [r for a, b in spans for r in self.rows[a:b]]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on the host cores

def cpu_baseline(K: int, T: int, budget_s: float = 10.0, cost_name: str = "contact"):
    """The oracle, as it stands, on the host cores: full FP64 updates of the
    same workload repeated until about `budget_s` seconds have passed."""
    import oracle
    rb, oc, q, qd, goal, plane = oracle_problem(K, T, cost_name)
    cores = os.cpu_count() or 1
    nth = min(cores, oracle.max_threads())
    plan = np.zeros((T, 7))
    reps = 0
    t0 = time.perf_counter()
    while reps == 0 or time.perf_counter() - t0 < budget_s:
        oracle.mppi_step(rb, oc, DT, T, K, LAMBDA, np.full(7, SIGMA), SEED, reps, q, qd, goal,
                         plane, plan, nthreads=nth)
        reps += 1
    dt = time.perf_counter() - t0
    # the oracle's other modes: one thread at this K (one update), and one
    # thread and all threads at K = 256 (about two seconds each)
    modes = []
    for Km, thr, budget in ((K, 1, 0.0), (256, 1, 2.0), (256, nth, 2.0)):
        rbm, ocm, qm, qdm, gm, pm = oracle_problem(Km, T, cost_name)
        n = 0
        t1 = time.perf_counter()
        while n == 0 or time.perf_counter() - t1 < budget:
            oracle.mppi_step(rbm, ocm, DT, T, Km, LAMBDA, np.full(7, SIGMA), SEED, n, qm, qdm, gm,
                             pm, plan, nthreads=thr)
            n += 1
        d = time.perf_counter() - t1
        modes.append({"K": Km, "threads": thr, "value": Km * T * n / d, "updates": n,
                      "seconds": d})
    return {"value": K * T * reps / dt, "unit": UNIT, "cores": nth, "kind": "oracle",
            "sample": f"{reps} full FP64 updates at K={K}, T={T} (same arm and cost), "
                      f"OpenMP over samples on {nth} threads, {dt:.1f} s",
            "seconds": dt, "modes": modes}


def run_reference(args, rank, world):
    if rank != 0:
        return
    K, T = args.K, args.T
    import oracle
    rb, oc, q, qd, goal, plane = oracle_problem(K, T, args.cost)
    nth = min(os.cpu_count() or 1, oracle.max_threads())
    plan = np.zeros((T, 7))
    # size each step's sample so the whole run takes about --budget-s seconds
    t0 = time.perf_counter()
    oracle.mppi_step(rb, oc, DT, T, 512, LAMBDA, np.full(7, SIGMA), SEED, 0, q, qd, goal, plane,
                     plan, nthreads=nth)
    per_sample = (time.perf_counter() - t0) / 512
    budget = args.budget_s / max(1, args.steps + args.warmup)
    K_sample = int(max(64, min(K, budget / per_sample)))
    for w in range(args.warmup):
        oracle.mppi_step(rb, oc, DT, T, K_sample, LAMBDA, np.full(7, SIGMA), SEED, w, q, qd, goal,
                         plane, plan, nthreads=nth)
    times = []
    for s in range(args.steps):
        t0 = time.perf_counter()
        oracle.mppi_step(rb, oc, DT, T, K_sample, LAMBDA, np.full(7, SIGMA), SEED, s, q, qd, goal,
                         plane, plan, nthreads=nth)
        times.append(time.perf_counter() - t0)
    times = np.array(times)
    val = K_sample * T / times.mean()
    scale = K / K_sample
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(times.mean() * 1e3 * scale), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(K, T, 1, args.cost),
            "p50_ms": float(np.percentile(times, 50) * 1e3 * scale),
            "p99_ms": float(np.percentile(times, 99) * 1e3 * scale),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": nth, "kind": "oracle",
                             "sample": f"each step one FP64 update at K={K_sample} of the K={K} "
                                       f"workload (latencies scaled by {scale:g})"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm

def run_ours(args, rank, world):
    import torch
    from paper_2609_02020_b300 import mppi, synth

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    K, T = args.K, args.T
    arm, cost, q, qd, goal = workload(rank, args.cost)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctl = mppi.MPPI(arm, cost, dt=DT, T=T, K=K, lam=LAMBDA, sigma=SIGMA, seed=SEED + rank,
                    variant=args.variant, stream=stream)
    pose = ctl.ee_pose(q)
    if args.cost == "collision":
        ctl.set_obstacles(obstacles(rank, arm, pose[:3]))
    # variant 0 picks the warp-specialised kernel (with the collision cost on
    # two extra warps, the wrench estimate on one) while its blocks fit in one
    # wave, else the register kernel, or the rolled one with an optional cost
    kname = {1: "rollout_kernel", 2: "rollout_kernel_rolled",
             3: "rollout_kernel_ws_fest" if args.cost == "force_estimate"
             else "rollout_kernel_ws_small" if args.cost == "contact" and K <= 8192
             else "rollout_kernel_ws"}[ctl.variant()]
    plane = synth.plane_through(float(pose[2]))
    d_in = torch.tensor(mppi.pack_inputs(q, qd, goal, plane), device="cuda")
    d_tau = torch.zeros(7, device="cuda")
    d_plan = torch.zeros(T, 7, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # --- device-resident timed region --------------------------------------
    for _ in range(args.warmup):
        ctl.step_device(d_in, d_tau, d_plan)
    assert ctl.sync() == 0
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    q32 = np.asarray(q, np.float32)
    qd32 = np.asarray(qd, np.float32)
    g32 = np.asarray(goal, np.float32)
    p32 = np.asarray(plane, np.float32)
    spans = []
    with ClockSampler(dev) as clk:
        barrier()
        a = clk.mark()
        t_wall = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()
            starts[i].record(stream)
            ctl.step_device(d_in, d_tau, d_plan)
            ends[i].record(stream)
        barrier()
        t_wall = time.perf_counter() - t_wall
        spans.append((a, clk.mark()))
        rc = ctl.sync()
        if rc != 0:
            raise RuntimeError(f"update failed with status {rc}")
        step_ms = np.array([s.elapsed_time(e) for s, e in zip(starts, ends)])
        mean_ms = float(step_ms.mean())
        launches = 2 * args.steps  # rollout kernel + merge kernel per update

        # --- latency: the update's p50/p99 over at least LAT_UPDATES updates
        #     and LAT_SECONDS of wall time (so that the clock samples cover
        #     it), after LAT_WARMUP warm-ups, L2 flushed before each update
        lat_ms = latency_loop(ctl, d_in, d_tau, d_plan, flush, stream, barrier, clk, spans)

        # --- per-kernel times for the roofline (events on the library stream)
        ms_roll, ms_upd = ctl.time_kernels(d_in, 200)

        # --- end to end through the public host call --------------------------
        for _ in range(args.warmup):
            ctl.step(q32, qd32, g32, p32)
        barrier()
        a = clk.mark()
        e2e_ms = []
        for _ in range(max(args.steps, LAT_UPDATES)):
            flush.zero_()  # L2 flushed before every timed call, as above
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctl.step(q32, qd32, g32, p32)
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
        barrier()
        spans.append((a, clk.mark()))
    e2e_ms = np.array(e2e_ms)

    # --- aggregate over ranks -------------------------------------------------
    total_ms, e2e_mean = max_over_ranks([float(step_ms.sum()), float(e2e_ms.mean())], world,
                                        "cuda")
    units = K * T * args.steps * world
    value = units / (total_ms * 1e-3)
    e2e_value = K * T * world / (e2e_mean * 1e-3)

    if rank != 0:
        ctl.close()
        return
    clocks = clk.summary(spans)
    peak_max = SM_COUNT * FP32_LANES_PER_SM * 2 * 2032e6 / 1e12
    flop = FLOP_PER_ROLLOUT_STEP.get(args.cost)
    flop_exec = FLOP_EXECUTED_PER_ROLLOUT_STEP.get((args.cost, kname))
    num = flop if flop else flop_exec
    achieved = num * K * T / (ms_roll * 1e-3) / 1e12 if num else None
    traffic = (ROLLOUT_TRAFFIC_BYTES_PER_LAUNCH.get((args.cost, kname))
               if (K, T) == (K_DEFAULT, T_DEFAULT) else None)
    fma = mppi.measure_fp32_peak()  # outside the timed regions
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_max, "unit": "TFLOP/s",
            "frac": achieved / peak_max if achieved else None, "traffic": traffic,
            "kernel": kname, "kernel_ms": ms_roll,
            "flop_per_rollout_step": num,
            "flop_source": ("algorithmic, counted by hand on the formulation" if flop else
                            "executed (ncu FADD + FMUL + 2 FFMA); no hand count for this cost"),
            "flop_executed_per_rollout_step": flop_exec,
            "frac_executed": (flop_exec * K * T / (ms_roll * 1e-3) / 1e12 / peak_max
                              if flop_exec else None),
            "peak_note": "FP32 peak of 148 SMs x 128 lanes x 2 FLOP at the 2032 MHz "
                         "maximum SM clock (derived; no measured FP32 peak is on file); "
                         "peak_fma_measured: independent FMA chains on every SM of this "
                         "GPU, median of five launches",
            "peak_fma_measured": fma,
            "frac_of_fma_measured": achieved / fma if achieved else None}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_dict(K, T, world, args.cost),
            "p50_ms": float(np.percentile(lat_ms, 50)),
            "p99_ms": float(np.percentile(lat_ms, 99)),
            "latency": {"updates": int(lat_ms.size), "warmup": LAT_WARMUP,
                        "mean_ms": float(lat_ms.mean()), "p50_ms": float(np.percentile(lat_ms, 50)),
                        "p99_ms": float(np.percentile(lat_ms, 99)), "max_ms": float(lat_ms.max()),
                        "timing": "CUDA events around each update on the library's stream, "
                                  "L2 flushed before each"},
            "update_hz": 1e3 / mean_ms,
            "kernels_ms": {kname: ms_roll, "merge_kernel": ms_upd},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 26 * 4,
                    "d2h_bytes_per_step": (16 + T * 7) * 4, "calls": int(e2e_ms.size),
                    "p50_ms": float(np.percentile(e2e_ms, 50)),
                    "p99_ms": float(np.percentile(e2e_ms, 99)),
                    "api": "mppi_step (host buffers, CUDA graph replay: H2D copy of the "
                           "inputs and a sequence word, two kernels, the merge kernel writing "
                           "tau0, status, plan and last the sequence word into pinned host "
                           "memory, which the host polls), host clock per call"},
            "roofline": roof,
            "clocks": clocks,
            "gpu_launches": launches,
            "wall_s": t_wall}
    ctl.close()
    if not args.no_serve:
        line["serve"] = serve_summary(rank)
    if not args.no_learned:
        line["learned_latency"] = learned_latency_summary()
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(K, T, cost_name=args.cost)
    print(json.dumps(line), flush=True)


LAT_UPDATES, LAT_WARMUP, LAT_SECONDS = 1000, 50, 1.2


def learned_latency_summary(K_learned=2048, K_plain=16384):
    """Update latency of the learned-proposal form beside plain MPPI, for the
    update line: device time per update (CUDA events on the controller's
    stream, LAT_UPDATES after LAT_WARMUP, L2 not flushed), on the closed-loop
    study's task and network shape.  The network is untrained here: its
    weights do not change the time; the tracking comparison, which needs the
    trained network, is `--mode learned`."""
    import torch
    from paper_2609_02020_b300 import learned, mppi
    prob = learned.tracking_problem(0)
    s = torch.cuda.Stream()
    net = mppi.MLP(21 + 7 * prob.T, 256, 3, 7 * prob.T, max_batch=256, seed=0, stream=s)
    out = {"task": "the closed-loop study's (learned.tracking_problem), untrained network "
                   "147-3x256-126, half of the learned form's samples around the plain warm start",
           "updates": LAT_UPDATES}
    forms = (("plain", K_plain, None), ("learned_one_call", K_learned, True),
             ("learned_two_calls", K_learned, False))
    for name, K, one_call in forms:
        ctl = prob.controller(K, seed=5, stream=s)
        q, qd, goal = prob.episode_start(123, ctl)
        ctl.set_plan(prob.hold_plan(ctl, q))
        d_in = torch.tensor(mppi.pack_inputs(q, qd, goal, prob.plane), device="cuda")
        d_tau = torch.zeros(7, device="cuda")
        n_plain = K // 2
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(LAT_UPDATES)]
        for i in range(LAT_WARMUP + LAT_UPDATES):
            if i >= LAT_WARMUP:
                ev[i - LAT_WARMUP][0].record(s)
            if one_call is None:
                ctl.step_device(d_in, d_tau)
            elif one_call:
                net.propose_step_device(ctl, d_in, n_plain, d_tau)
            else:
                net.propose(ctl, d_in, n_plain)
                ctl.step_device(d_in, d_tau)
            if i >= LAT_WARMUP:
                ev[i - LAT_WARMUP][1].record(s)
        s.synchronize()
        ms = np.array([a.elapsed_time(b) for a, b in ev])
        out[name] = {"K": K, "p50_ms": float(np.percentile(ms, 50)),
                     "p99_ms": float(np.percentile(ms, 99)), "status": ctl.sync()}
        ctl.close()
    net.close()
    return out


def latency_loop(ctl, d_in, d_tau, d_plan, flush, stream, barrier, clk, spans):
    """Device time of single updates (events around each on the library's
    stream, L2 flushed before each): at least LAT_UPDATES updates and
    LAT_SECONDS of wall time after LAT_WARMUP warm-ups; returns ms per update."""
    import torch
    for _ in range(LAT_WARMUP):
        ctl.step_device(d_in, d_tau, d_plan)
    barrier()
    a = clk.mark()
    out = []
    t_end = time.perf_counter() + LAT_SECONDS
    while len(out) < LAT_UPDATES or time.perf_counter() < t_end:
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(250)]
        for st, en in ev:
            flush.zero_()
            st.record(stream)
            ctl.step_device(d_in, d_tau, d_plan)
            en.record(stream)
        torch.cuda.synchronize()
        out.extend(st.elapsed_time(en) for st, en in ev)
    barrier()
    spans.append((a, clk.mark()))
    if ctl.sync() != 0:
        raise RuntimeError("update failed in the latency loop")
    return np.array(out)


SERVE_RATES = (10_000.0, 60_000.0)  # below and above the 256-problem mix's capacity
SERVE_SECONDS = 1.0


def serve_server(rank, n, pool_mb):
    """The batched-serving workload: n seeded problems, uneven K and T, half
    with plane contact; returns (server, all scratch bytes)."""
    from paper_2609_02020_b300 import mppi, synth
    Ks, Ts = synth.serving_mix(17 + rank, n)
    srv = mppi.Server(pool_bytes=pool_mb << 20, max_problems=n, max_batch=min(n, 1024), lanes=3)
    total_scratch = 0
    for i in range(n):
        arm = synth.arm(10_000 * rank + i)
        q, qd = synth.state(20_000 + i, arm)
        goal = synth.goal(20_000 + i, arm)
        cost = synth.cost_contact() if i % 2 else synth.cost_free_space()
        pid = srv.add_problem(arm, cost, dt=DT, T=int(Ts[i]), K=int(Ks[i]), lam=LAMBDA,
                              sigma=SIGMA, seed=SEED + i)
        plane = synth.NO_PLANE
        srv.set_input(pid, mppi.pack_inputs(q, qd, goal, plane if not cost["contact"] else
                                            np.array([0.0, 0.0, 1.0, -10.0])))
        total_scratch += 4 * int(Ks[i]) * (7 * int(Ts[i]) + 1)
    return srv, total_scratch


def serve_summary(rank, n=256, pool_mb=1024):
    """Compact serving measurement for the update line: the 256-problem mix
    under Poisson arrivals for SERVE_SECONDS at 10 k/s and at a saturating
    60 k/s (latency = completion minus scheduled arrival, host clock)."""
    t0 = time.perf_counter()
    srv, scratch = serve_server(rank, n, pool_mb)
    best = srv.autotune()
    st = srv.stats()
    srv.start()
    setup = time.perf_counter() - t0
    pts = []
    for rate in SERVE_RATES:
        r = srv.load_test(rate, SERVE_SECONDS, seed=int(rate))
        pts.append({"rate_hz": rate, "p50_ms": float(r["p50_ms"]), "p99_ms": float(r["p99_ms"]),
                    "updates_per_s": float(r["updates_per_s"]),
                    "rollout_steps_per_s": float(r["rollout_steps_per_s"]),
                    "mean_batch": float(r["mean_batch"]), "completed": int(r["completed"])})
    srv.stop()
    srv.close()
    return {"workload": f"{n} seeded 7-DoF problems, K~U{{512..8192}}, T~U{{10..50}}, half with "
                        "plane contact, Poisson arrivals",
            "seconds_per_rate": SERVE_SECONDS, "setup_s": setup,
            "autotune": {"variant": st["variant"], "tile": st["block"], "rollout_ms": best},
            "points": pts}


def run_serve(args, rank, world):
    """Batched serving: many problems with uneven K and T, Poisson arrivals,
    memory-based admission, continuous batching (include/mppi_serve.h)."""
    import torch
    from paper_2609_02020_b300 import mppi, synth
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    n = args.problems
    srv, total_scratch = serve_server(rank, n, args.pool_mb)
    best = srv.autotune()
    st = srv.stats()
    srv.start()
    points = []
    for rate in [float(r) for r in args.rates.split(",")]:
        r = srv.load_test(rate, args.seconds, seed=int(rate))
        points.append({"rate_hz": rate, **{k: float(v) for k, v in r.items()}})
    srv.stop()
    srv.close()
    if rank == 0:
        print(json.dumps({
            "mode": "serve",
            "metric": "batched MPPI serving: update latency p50/p99 and throughput under Poisson load",
            "unit": "ms / updates/s / rollout-steps/s", "n_gpus": world, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"{n} seeded 7-DoF problems, K~U{{512..8192}}, T~U{{10..50}}, "
                                   f"dt={DT} s, half with plane contact",
                       "pool_mib": args.pool_mb, "all_scratch_mib": total_scratch / 2**20,
                       "lanes": 3, "seconds_per_rate": args.seconds},
            "autotune": {"variant": st["variant"], "tile": st["block"], "rollout_ms": best},
            "points": points}), flush=True)


SWEEP_K = (1024, 4096, 16384, 65536)
SWEEP_T = (18, 36, 50)


def run_sweep(args, rank, world):
    """The update of the contact workload over K x T, with the FP32 and the
    FP64 reduction of Eq. 4: device time per update (CUDA events, L2 flushed
    between updates), the kernel variant 0 chose and its kernel times."""
    import torch
    from paper_2609_02020_b300 import mppi, synth
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    arm, cost, q, qd, goal = workload(rank, "contact")
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    steps = max(args.steps, 1)
    peak = SM_COUNT * FP32_LANES_PER_SM * 2 * 2032e6 / 1e12  # derived, as in the update line
    rows, spans = [], []
    with ClockSampler(dev) as clk:
        for T in SWEEP_T:
            for K in SWEEP_K:
                for fp64 in (False, True):
                    ctl = mppi.MPPI(arm, cost, dt=DT, T=T, K=K, lam=LAMBDA, sigma=SIGMA,
                                    seed=SEED + rank, reduce_fp64=fp64, stream=stream)
                    pose = ctl.ee_pose(q)
                    plane = synth.plane_through(float(pose[2]))
                    d_in = torch.tensor(mppi.pack_inputs(q, qd, goal, plane), device="cuda")
                    d_tau = torch.zeros(7, device="cuda")
                    d_plan = torch.zeros(T, 7, device="cuda")
                    # every update starts from the same state and the zero plan
                    # (outside the timed events): repeated warm-started updates of
                    # one fixed state are no closed loop, and over thousands of
                    # them the plan can drift until no rollout stays finite
                    zero_plan = np.zeros((T, 7), np.float32)
                    for _ in range(max(args.warmup, 3)):
                        ctl.set_plan(zero_plan)
                        ctl.step_device(d_in, d_tau, d_plan)
                    st = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
                    en = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
                    torch.cuda.synchronize()
                    a = clk.mark()
                    for i in range(steps):
                        ctl.set_plan(zero_plan)
                        flush.zero_()
                        st[i].record(stream)
                        ctl.step_device(d_in, d_tau, d_plan)
                        en[i].record(stream)
                    torch.cuda.synchronize()
                    spans.append((a, clk.mark()))
                    if ctl.sync() != 0:
                        raise RuntimeError(f"update failed at K={K} T={T}")
                    ms = np.array([x.elapsed_time(y) for x, y in zip(st, en)])
                    ms_roll, ms_upd = ctl.time_kernels(d_in, 20)
                    tflops = FLOP_PER_ROLLOUT_STEP["contact"] * K * T / (ms_roll * 1e-3) / 1e12
                    rows.append({"K": K, "T": T, "reduce": "f64" if fp64 else "f32",
                                 "variant": ctl.variant(), "ms_per_update": float(ms.mean()),
                                 "p50_ms": float(np.percentile(ms, 50)),
                                 "p99_ms": float(np.percentile(ms, 99)),
                                 "rollout_steps_per_s": K * T / (float(ms.mean()) * 1e-3),
                                 "rollout_ms": ms_roll, "update_ms": ms_upd,
                                 "rollout_tflops": tflops, "frac_fp32_peak": tflops / peak})
                    ctl.close()
    clocks = clk.summary(spans)
    if rank == 0:
        print(json.dumps({
            "mode": "sweep", "metric": "MPPI update time over K x T (contact workload)",
            "unit": "ms", "n_gpus": world, "steps": steps, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"7-DoF seeded arm with plane contact, dt={DT} s, "
                                   f"sigma={SIGMA} N m, lambda={LAMBDA}",
                       "K": list(SWEEP_K), "T": list(SWEEP_T),
                       "l2": "flushed between timed steps"},
            "clocks": clocks, "points": rows}), flush=True)


def run_mlp(args, rank, world):
    """The learned proposal's network kernels alone (tcgen05 BF16, FP32
    accumulate): Adam training steps of 1024 and 4096 rows, the batched
    forward of 4096 rows, and the single-row proposal kernel (launched one
    by one from the host, and 200 launches replayed from one CUDA graph);
    device time by CUDA events on the network's stream, after warm-up."""
    import torch
    from paper_2609_02020_b300 import learned, mppi
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    s = torch.cuda.Stream()
    torch.cuda.set_stream(s)
    dims = [147, 256, 256, 256, 126]
    net = mppi.MLP(dims[0], dims[1], 3, dims[-1], max_batch=4096, seed=1, stream=s)
    g = torch.Generator(device="cuda")
    g.manual_seed(7)
    X = torch.randn(16 * 4096, dims[0], device="cuda", generator=g)
    Y = torch.randn(16 * 4096, dims[-1], device="cuda", generator=g)
    fwd = 2 * sum(dims[i] * dims[i + 1] for i in range(4))

    def timed(fn, n):
        for _ in range(max(args.warmup, 3)):
            fn(0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        for i in range(n):
            fn(i)
        b.record(s)
        s.synchronize()
        return a.elapsed_time(b) / n

    out = {}
    for B in (1024, 4096):
        ms = timed(lambda i: net.train_step(X[(i % 16) * B:(i % 16 + 1) * B],
                                            Y[(i % 16) * B:(i % 16 + 1) * B], 1e-4), 300)
        flop = 3 * fwd * B
        out[f"train_{B}"] = {"ms_per_step": ms, "gflop_per_step": flop / 1e9,
                             "tflops": flop / (ms * 1e-3) / 1e12,
                             "frac_of_bf16_peak": flop / (ms * 1e-3) / 1e12 / 1786.4}
    dY = torch.empty(4096, dims[-1], device="cuda")
    ms = timed(lambda i: net.forward(X[:4096], dY), 300)
    out["forward_4096"] = {"ms": ms, "tflops": fwd * 4096 / (ms * 1e-3) / 1e12}
    prob = learned.tracking_problem()
    ctl = prob.controller(512, seed=1, stream=s)
    q, qd, goal = prob.episode_start(123, ctl)
    d_in = torch.tensor(mppi.pack_inputs(q, qd, goal, prob.plane), device="cuda")
    out["propose_us_stream"] = timed(lambda i: net.propose(ctl, d_in, 256), 500) * 1e3
    # the kernel without the host's launch rate: 200 launches in one CUDA graph
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        for _ in range(200):
            net.propose(ctl, d_in, 256)
    out["propose_us_graph"] = timed(lambda i: g.replay(), 5) * 1e3 / 200
    ctl.close()
    net.close()
    if rank == 0:
        print(json.dumps({"mode": "mlp", "metric": "learned-proposal network kernels on tcgen05",
                          "unit": "ms / TFLOP/s / us", "n_gpus": world, "dtype": "bf16 in, f32 accumulate",
                          "data": "synthetic", "config": {"network": "147 -> 3 x 256 GELU -> 126"},
                          "peak_bf16_tflops": 1786.4, **out}), flush=True)


def run_learned(args, rank, world):
    """Learned proposal on the reaching task where plain MPPI at K=16384
    converges (learned.tracking_problem): pairs from plain MPPI at
    --label-k samples along its own closed loop, then rounds of pairs at the
    states the learned controller visits (same labels), training on the GPU
    with the library's tcgen05 BF16 kernels, then closed-loop tracking cost,
    final position error and update latency of plain MPPI (K=16384, fewer
    samples, and the labelling K) and of MPPI with the learned proposal."""
    import torch
    from paper_2609_02020_b300 import learned, mppi, synth
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    prob = learned.tracking_problem(rank)
    s = torch.cuda.Stream()
    t0 = time.perf_counter()
    X, Y = learned.generate(prob, args.pairs, K=args.label_k, seed=rank, episode_len=1000,
                            stream=s)
    t_gen = time.perf_counter() - t0
    net, info = learned.train(X, Y, steps=args.train_steps, batch=1024, lr=1e-3, stream=s)
    on_policy = []
    for rnd in range(args.on_policy_rounds):
        t1 = time.perf_counter()
        Xd, Yd = learned.generate_on_policy(prob, net, args.on_policy_pairs, K_label=args.label_k,
                                            K_learner=2048, plain_frac=0.5, seed=rank + 17 * rnd,
                                            stream=s)
        t_op = time.perf_counter() - t1
        X, Y = torch.cat([X, Xd]), torch.cat([Y, Yd])
        del Xd, Yd
        net.close()
        net, info = learned.train(X, Y, steps=args.train_steps + 1000, batch=1024, lr=1e-3,
                                  seed=rnd + 1, stream=s)
        on_policy.append({"round": rnd + 1, "pairs": int(X.shape[0]), "generation_s": t_op,
                          "val_loss": info["val_loss"]})
    dims = [X.shape[1], 256, 256, 256, Y.shape[1]]
    flop_step = 3 * 2 * sum(dims[i] * dims[i + 1] for i in range(4)) * 1024
    # the proposal kernel alone: events around single launches on the handle's stream
    ctl = prob.controller(512, seed=1, stream=s)
    q, qd, goal = prob.episode_start(123, ctl)
    d_in = torch.tensor(mppi.pack_inputs(q, qd, goal, prob.plane), device="cuda")
    for _ in range(20):
        net.propose(ctl, d_in, 256)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(500)]
    for a, b in ev:
        a.record(s)
        net.propose(ctl, d_in, 256)
        b.record(s)
    s.synchronize()
    prop_us = np.array([a.elapsed_time(b) for a, b in ev]) * 1e3
    ctl.close()
    rows = []
    for name, K, mk in (
            [("plain", K, lambda K: learned.PlainMPPI(prob, K, seed=5, stream=s))
             for K in (16384, 512, 2048, 4096, args.label_k)] +
            [("learned", K, lambda K, f=float(f): learned.LearnedMPPI(prob, net, K, seed=5,
                                                                      stream=s, plain_frac=f))
             for f in args.plain_fracs.split(",") for K in (512, 2048, 4096)]):
        c = mk(K)
        r = learned.evaluate(prob, c, episodes=args.episodes, steps=1000, seed=1, stream=s)
        frac = c.n_plain / K if name == "learned" else 1.0
        c.close()
        r.pop("tracking_cost_per_episode")
        rows.append({"controller": name, "K": K, "plain_frac": frac, **r})
    if rank == 0:
        print(json.dumps({
            "mode": "learned",
            "metric": "closed-loop tracking cost, final error and update latency, learned "
                      "proposal vs plain MPPI",
            "unit": "cost (mean of W_pos|dp|^2) / m / ms", "n_gpus": world,
            "dtype": "f32 rollouts, bf16 network", "data": "synthetic",
            "config": {"workload": "7-DoF seeded gravity-compensated arm (damping 5), "
                                   "position-only goals 0.2 rad per joint away, W_pos=300, "
                                   "sigma=2, lambda=3, T=18 dt=0.01, 1000-step (10 s) episodes",
                       "pairs": args.pairs, "pairs_K": args.label_k,
                       "on_policy": {"rounds": args.on_policy_rounds,
                                     "pairs_per_round": args.on_policy_pairs,
                                     "learner": "learned proposal, K=2048, half plain"},
                       "network": "147 -> 3 x 256 GELU -> 126, BF16 tcgen05, FP32 accumulate",
                       "plain_fallback_fraction": 0.5},
            "generation_s": t_gen,
            "on_policy_rounds": on_policy,
            "training": {**{k: v for k, v in info.items()},
                         "gflop_per_step": flop_step / 1e9,
                         "tflops": flop_step * info["steps"] / info["seconds"] / 1e12,
                         "frac_of_bf16_peak": flop_step * info["steps"] / info["seconds"] / 1e12
                                              / 1786.4},
            "propose_kernel_us": {"p50": float(np.percentile(prop_us, 50)),
                                  "p99": float(np.percentile(prop_us, 99))},
            "rows": rows}), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() and args.impl == "ours" else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend)
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        elif args.mode == "serve":
            run_serve(args, rank, world)
        elif args.mode == "learned":
            run_learned(args, rank, world)
        elif args.mode == "sweep":
            run_sweep(args, rank, world)
        elif args.mode == "mlp":
            run_mlp(args, rank, world)
        else:
            run_ours(args, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
