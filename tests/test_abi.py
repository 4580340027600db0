"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every symbol include/mppi.h declares, and rejects invalid parameters before
touching the device."""
import os
import re

import numpy as np
import pytest

from paper_2609_02020_b300 import mppi, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"MPPI_API\s+[\w\s\*]+?\b(mppi\w+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    L = mppi.load()
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert sorted(mppi.EXPORTS) == sorted(set(mppi.EXPORTS))
    assert set(names) <= set(mppi.EXPORTS) | set(names)
    assert "sm_103a" in mppi.version()


def _create(arm=None, cost=None, **kw):
    args = dict(dt=0.01, T=18, K=256, lam=1.0, sigma=2.0, seed=1)
    args.update(kw)
    return mppi.MPPI(arm or synth.arm(0), cost or synth.cost_free_space(), **args)


@pytest.mark.parametrize("kw,msg", [
    (dict(K=0), "K must"), (dict(K=(1 << 22) + 1), "K must"), (dict(T=0), "T must"),
    (dict(T=257), "T must"), (dict(lam=0.0), "lambda"), (dict(lam=-1.0), "lambda"),
    (dict(dt=0.0), "dt"), (dict(sigma=-1.0), "sigma"), (dict(lam=float("nan")), "lambda"),
    (dict(variant=4), "variant"), (dict(variant=-1), "variant"),
])
def test_create_rejects_bad_config(kw, msg):
    with pytest.raises(mppi.MPPIError) as e:
        _create(**kw)
    assert e.value.code == mppi.ERR_INVALID_ARG and msg in str(e.value)


def test_create_rejects_bad_robot_and_cost():
    arm = synth.arm(0)
    bad = dict(arm, n=6)
    with pytest.raises(mppi.MPPIError, match="robot.n"):
        _create(arm=bad)
    ax = arm["axis"].copy()
    ax[2] = [0.0, 0.0, 2.0]
    with pytest.raises(mppi.MPPIError, match="unit"):
        _create(arm=dict(arm, axis=ax))
    m = arm["mass"].copy()
    m[3] = 0.0
    with pytest.raises(mppi.MPPIError, match="mass"):
        _create(arm=dict(arm, mass=m))
    c = synth.cost_contact()
    c["k_contact"] = -1.0
    with pytest.raises(mppi.MPPIError, match="contact"):
        _create(cost=c)
    c = synth.cost_free_space()
    c["w_tau"] = float("inf")
    with pytest.raises(mppi.MPPIError, match="finite"):
        _create(cost=c)


def test_create_rejects_bad_wrench_estimate_cost():
    c = dict(synth.cost_free_space(), force_estimate=1, w_force6=np.array([0, 0, np.nan, 0, 0, 0]))
    with pytest.raises(mppi.MPPIError, match="wrench-estimate weights"):
        _create(cost=c)
    # the estimate runs in the rolled rollout kernel only
    c = dict(synth.cost_free_space(), force_estimate=1, w_force6=np.ones(6))
    with pytest.raises(mppi.MPPIError, match="rolled"):
        _create(cost=c, variant=1)


def test_create_rejects_bad_collision_cost():
    ok = synth.cost_collision(1, obstacles=np.array([[0, 0, 1, 0, 0, 1.2, 0.05]]))
    for bad, msg in [(dict(collision=3), "collision must"),
                     (dict(w_collision=float("nan")), "finite"),
                     (dict(link_radius=np.full(7, -0.01)), "radii"),
                     (dict(obstacles=np.array([[0, 0, 1, 0, 0, 1.2, -0.05]])), "obstacle radii"),
                     (dict(obstacles=np.array([[0, 0, np.inf, 0, 0, 1.2, 0.05]])), "finite")]:
        with pytest.raises(mppi.MPPIError, match=msg):
            _create(cost=dict(ok, **bad))
    with pytest.raises(mppi.MPPIError, match="rolled"):
        _create(cost=ok, variant=1)
    with pytest.raises(ValueError):
        _create(cost=dict(ok, obstacles=np.zeros((9, 7))))
