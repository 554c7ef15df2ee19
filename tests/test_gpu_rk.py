"""The Runge-Kutta family of Sec. 2.2 on the GPU vs the FP64 oracle tableaus:
RK3 (Kutta), RK4, RK12 (Heun-Euler), RK23 (Bogacki-Shampine), RKCK
(Cash-Karp) next to the Dormand-Prince path tested elsewhere."""

import numpy as np
import pytest

from oracle import llg
from paper_1102_3069_gb300 import binding as B
from paper_1102_3069_gb300 import inputs

from gpu_util import oracle, solver, to_dev, to_np

pytestmark = pytest.mark.gpu

W = inputs.workload("film_64x16")
METHODS = {"rk3": B.MM_RK3, "rk4": B.MM_RK4, "rk12": B.MM_RK12, "rk23": B.MM_RK23, "rkck": B.MM_RKCK,
           "rkdp": B.MM_RKDP}


def _pair(**over):
    mat = dict(W["material"])
    mat.update(over)
    return (solver(W["shape"], W["cell"], pbc=W["pbc"], **mat),
            oracle(W["shape"], W["cell"], pbc=W["pbc"], **mat))


def _m64(m):
    m = m.astype(np.float64)
    return m / np.sqrt((m * m).sum(axis=0, keepdims=True))


@pytest.mark.parametrize("name", sorted(METHODS))
def test_single_step_matches_tableau(name):
    s, p = _pair()
    m = W["m"]
    md = to_dev(m)
    tab = llg.TABLEAUS[name]
    h = 5e-14
    acc, t, _ = B.mm_step(s.ctx, md, METHODS[name], 0.0, h, tol=1.0)
    assert acc and t == pytest.approx(h, rel=1e-12, abs=0.0)
    ref = llg.rk_attempt(p, _m64(m), h, tab)[0]
    assert np.max(np.abs(to_np(md) - ref)) <= 1e-6


@pytest.mark.parametrize("name", ["rk3", "rk4", "rkck"])
def test_fixed_steps_from_smooth_state(name):
    s, p = _pair()
    m = inputs.smooth_tilt(W["shape"])
    md = to_dev(m)
    B.mm_load(s.ctx, md)
    tol = -1.0 if llg.TABLEAUS[name].adaptive else 0.0
    B.mm_advance(s.ctx, METHODS[name], 200, dt_s=5e-14, tol=tol)
    B.mm_store(s.ctx, md)
    st = B.mm_get_stats(s.ctx)
    assert st["accepted"] == 200 and st["status"] == 0
    ref = llg.rk_fixed(p, _m64(m), 5e-14, 200, llg.TABLEAUS[name])
    err = float(np.max(np.abs(to_np(md) - ref)))
    print(name, "200 fixed steps max|dm|", err)
    assert err <= 1e-5


@pytest.mark.parametrize("name", ["rk12", "rk23", "rkck"])
def test_adaptive_run_matches_oracle(name):
    s, p = _pair()
    m = inputs.smooth_tilt(W["shape"])
    md = to_dev(m)
    B.mm_load(s.ctx, md)
    tol = 1e-5 if name == "rk12" else 1e-6
    B.mm_advance(s.ctx, METHODS[name], 200000, dt_s=1e-13, tol=tol, t_end_s=2e-10)
    B.mm_store(s.ctx, md)
    st = B.mm_get_stats(s.ctx)
    assert st["done"] == 1 and st["status"] == 0
    assert st["t"] == pytest.approx(2e-10, rel=1e-12, abs=0.0)
    ref = llg.TableauStepper(p, _m64(m), llg.TABLEAUS[name], h0=1e-13, tol=tol)
    ref.run_until(2e-10)
    mg = to_np(md)
    print(name, "steps gpu", st["accepted"], st["rejected"], "oracle", ref.accepted, ref.rejected,
          "max|dm|", np.max(np.abs(mg - ref.m)))
    assert abs(st["accepted"] - ref.accepted) <= 0.02 * ref.accepted + 2
    assert np.max(np.abs(mg - ref.m)) <= 1e-4


def test_thermal_rk4_steps_match_oracle():
    s, p = _pair(temperature=300.0, seed=99, alpha=0.05)
    m = W["m"]
    md = to_dev(m)
    B.mm_load(s.ctx, md, 0.0, 0)
    dt = 20e-15
    B.mm_advance(s.ctx, B.MM_RK4, 5, dt_s=dt)
    B.mm_store(s.ctx, md)
    ref = llg.rk_fixed(p, _m64(m), dt, 5, llg.TABLEAUS["rk4"])
    assert np.max(np.abs(to_np(md) - ref)) <= 2e-6


def test_adaptive_methods_refuse_thermal_noise():
    s, _ = _pair(temperature=300.0)
    B.mm_load(s.ctx, to_dev(W["m"]))
    for meth in (B.MM_RK12, B.MM_RK23, B.MM_RKCK):
        with pytest.raises(B.MMError) as e:
            B.mm_advance(s.ctx, meth, 1, dt_s=1e-13, tol=1e-6)
        assert e.value.code == B.MM_EINVAL
