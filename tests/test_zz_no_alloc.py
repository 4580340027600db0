"""The allocation-free entry point mppi_step_static.

It exists for callers that may not allocate device memory while they run (a
hard-real-time control thread, or a plug-in whose host owns all device
memory).  These tests call it through the C ABI twice in a row (the second
call warm-started from the first call's shifted plan, with iter + 1) and
compare both results with the handle-based path (mppi_step), which keeps its
scratch in buffers allocated by mppi_create: at K = 4096 with contact, and
at the largest K the static array holds (MPPI_STATIC_K_MAX = 65536, T = 4,
light weights) with FP32 and FP64 sums.  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2609_02020_b300 import mppi
from _common import gpu_controller, make_case, parity_cost

pytestmark = pytest.mark.gpu

PLAN_TOL = 1e-5  # N m, the plan tolerance of the parity tests
STATIC_K_MAX = 65536  # MPPI_STATIC_K_MAX in include/mppi.h


def _two_calls_against_handle(c, fp64=False):
    import torch
    with gpu_controller(c, reduce_fp64=fp64) as g:
        g.step(c["q"], c["qd"], c["goal"], c["plane"])
        u1, p1 = g.updated_plan(), g.get_plan()
        g.step(c["q"], c["qd"], c["goal"], c["plane"])
        u2, p2 = g.updated_plan(), g.get_plan()
    kw = dict(dt=c["dt"], T=c["T"], K=c["K"], lam=c["lam"], sigma=c["sigma"], seed=c["seed"],
              reduce_fp64=fp64)
    d_in = torch.tensor(mppi.pack_inputs(c["q"], c["qd"], c["goal"], c["plane"]), device="cuda")
    d_plan = torch.zeros(c["T"], 7, device="cuda")
    d_u1, d_n1 = torch.zeros_like(d_plan), torch.zeros_like(d_plan)
    d_u2, d_n2 = torch.zeros_like(d_plan), torch.zeros_like(d_plan)
    mppi.step_static(c["arm"], c["cost"], it=0, d_in=d_in, d_plan=d_plan, d_ustar=d_u1,
                     d_plan_next=d_n1, **kw)
    mppi.step_static(c["arm"], c["cost"], it=1, d_in=d_in, d_plan=d_n1, d_ustar=d_u2,
                     d_plan_next=d_n2, **kw)
    torch.cuda.synchronize()
    return max(np.abs(d_u1.cpu().numpy() - u1).max(), np.abs(d_n1.cpu().numpy() - p1).max(),
               np.abs(d_u2.cpu().numpy() - u2).max(), np.abs(d_n2.cpu().numpy() - p2).max())


def test_step_static_matches_handle_path_on_two_calls():
    err = _two_calls_against_handle(make_case(2, contact=True, K=4096, T=18))
    print(f"static vs handle, K=4096 T=18: max |du| {err:.2e} N m")
    assert err <= PLAN_TOL


@pytest.mark.parametrize("fp64", [False, True])
def test_step_static_at_its_largest_k(fp64):
    # the most samples the static array holds, where the static update's
    # per-thread sums over K differ most from the handle's block partials;
    # light weights spread the update over hundreds of samples, so that the
    # sums matter (with contact one sample carries it and both agree exactly)
    err = _two_calls_against_handle(make_case(3, cost=parity_cost(), K=STATIC_K_MAX, T=4), fp64)
    print(f"static vs handle, K={STATIC_K_MAX} T=4, fp64={fp64}: max |du| {err:.2e} N m")
    assert err <= PLAN_TOL


def _call_static(K, **extra):
    import torch
    c = make_case(0, K=K, T=4)
    d = torch.zeros(32, device="cuda")
    mppi.step_static(c["arm"], c["cost"], dt=c["dt"], T=c["T"], K=c["K"], lam=c["lam"],
                     sigma=c["sigma"], seed=1, it=0, d_in=d, d_plan=d, d_ustar=d, d_plan_next=d,
                     **extra)


def test_step_static_rejects_k_above_its_limit():
    mppi.load()
    with pytest.raises(mppi.MPPIError) as e:
        _call_static(STATIC_K_MAX + 1)
    assert e.value.code == mppi.ERR_INVALID_ARG and "MPPI_STATIC_K_MAX" in str(e.value)


@pytest.mark.parametrize("variant", [2, 3])
def test_step_static_rejects_other_rollout_kernels(variant):
    with pytest.raises(mppi.MPPIError) as e:
        _call_static(64, variant=variant)
    assert e.value.code == mppi.ERR_INVALID_ARG and "variant" in str(e.value)
