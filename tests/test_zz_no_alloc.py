"""The allocation-free entry point mppi_step_static.

It exists for callers that may not allocate device memory while they run (a
hard-real-time control thread, or a plug-in whose host owns all device
memory).  This test calls it through the C ABI twice in a row (the second
call warm-started from the first call's shifted plan, with iter + 1) and
compares both results with the handle-based path (mppi_step), which keeps its
scratch in buffers allocated by mppi_create.  The file is named so that pytest
collects it last.
"""
import numpy as np
import pytest

from paper_2609_02020_b300 import mppi
from _common import gpu_controller, make_case

pytestmark = pytest.mark.gpu

PLAN_TOL = 1e-5  # N m, the plan tolerance of the parity tests


def test_step_static_matches_handle_path_on_two_calls():
    import torch
    c = make_case(2, contact=True, K=4096, T=18)
    with gpu_controller(c) as g:
        g.step(c["q"], c["qd"], c["goal"], c["plane"])
        u1, p1 = g.updated_plan(), g.get_plan()
        g.step(c["q"], c["qd"], c["goal"], c["plane"])
        u2, p2 = g.updated_plan(), g.get_plan()
    kw = dict(dt=c["dt"], T=c["T"], K=c["K"], lam=c["lam"], sigma=c["sigma"], seed=c["seed"])
    d_in = torch.tensor(mppi.pack_inputs(c["q"], c["qd"], c["goal"], c["plane"]), device="cuda")
    d_plan = torch.zeros(c["T"], 7, device="cuda")
    d_u1, d_n1 = torch.zeros_like(d_plan), torch.zeros_like(d_plan)
    d_u2, d_n2 = torch.zeros_like(d_plan), torch.zeros_like(d_plan)
    mppi.step_static(c["arm"], c["cost"], it=0, d_in=d_in, d_plan=d_plan, d_ustar=d_u1,
                     d_plan_next=d_n1, **kw)
    mppi.step_static(c["arm"], c["cost"], it=1, d_in=d_in, d_plan=d_n1, d_ustar=d_u2,
                     d_plan_next=d_n2, **kw)
    torch.cuda.synchronize()
    assert np.abs(d_u1.cpu().numpy() - u1).max() <= PLAN_TOL
    assert np.abs(d_n1.cpu().numpy() - p1).max() <= PLAN_TOL
    assert np.abs(d_u2.cpu().numpy() - u2).max() <= PLAN_TOL
    assert np.abs(d_n2.cpu().numpy() - p2).max() <= PLAN_TOL


def test_step_static_rejects_k_above_its_limit():
    import torch
    c = make_case(0, K=mppi.load() and 65537, T=4)
    d = torch.zeros(32, device="cuda")
    with pytest.raises(mppi.MPPIError) as e:
        mppi.step_static(c["arm"], c["cost"], dt=c["dt"], T=c["T"], K=c["K"], lam=c["lam"],
                         sigma=c["sigma"], seed=1, it=0, d_in=d, d_plan=d, d_ustar=d,
                         d_plan_next=d)
    assert e.value.code == mppi.ERR_INVALID_ARG and "MPPI_STATIC_K_MAX" in str(e.value)
