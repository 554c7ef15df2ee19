"""The torque bound of mm_advance for the methods whose last stage is not the
new state, against the oracle (Sec. 2.2; relaxation stops once
max_i |m_i x H_i|/Ms falls below the bound).

Euler, Heun and the tableaus without first-same-as-last (RK4, RK12 and
Cash-Karp with fixed steps here) judge the state a step starts from.  The run
must stop at the first state of the oracle's trajectory whose torque is below
the bound, keep that state, and report its torque.  The bound is placed
halfway (geometrically) between the torques of two successive oracle states,
far from both, so that float32 rounding cannot move the crossing.

Also: where a fixed-step run ends relative to t_end.
"""

import numpy as np
import pytest

from oracle import llg
from paper_1102_3069_gb300 import binding as B
from paper_1102_3069_gb300 import inputs

from gpu_util import oracle, solver, to_dev, to_np

pytestmark = pytest.mark.gpu

W = inputs.workload("film_64x16")
MAT = dict(W["material"], alpha=0.5)
DT = 1e-13
NMAX = 160


def _unit64(m):
    m = m.astype(np.float64)
    return m / np.sqrt((m * m).sum(axis=0, keepdims=True))


def _oracle_trajectory(p, m0, step_fn):
    ms, tq = [m0], [p.torque(m0)]
    m = m0
    for _ in range(NMAX):
        m = step_fn(p, m)
        ms.append(m)
        tq.append(p.torque(m))
    return ms, np.array(tq)


def _bound(tq, target=40):
    """A bound between tq[n-1] and tq[n] for the first n >= target where the
    torque falls by at least 0.5 % in one step; returns (n, bound)."""
    for n in range(target, len(tq)):
        if tq[n] < 0.995 * tq[:n].min():
            return n, float(np.sqrt(tq[n] * tq[:n].min()))
    raise AssertionError("torque does not fall along the trajectory")


STEPS = {
    "euler": (B.MM_EULER, 0.0, lambda p, m: llg.euler_step(p, m, DT)),
    "heun": (B.MM_HEUN, 0.0, lambda p, m: llg.heun_step(p, m, DT)),
    "rk4": (B.MM_RK4, 0.0, lambda p, m: llg.rk_fixed(p, m, DT, 1, llg.TABLEAUS["rk4"])),
    "rk12": (B.MM_RK12, -1.0, lambda p, m: llg.rk_fixed(p, m, DT, 1, llg.TABLEAUS["rk12"])),
    "rkck": (B.MM_RKCK, -1.0, lambda p, m: llg.rk_fixed(p, m, DT, 1, llg.TABLEAUS["rkck"])),
}


@pytest.mark.parametrize("name", sorted(STEPS))
def test_stop_on_torque_bound_keeps_the_first_state_below_it(name):
    method, tol, fn = STEPS[name]
    s = solver(W["shape"], W["cell"], pbc=W["pbc"], **MAT)
    p = oracle(W["shape"], W["cell"], pbc=W["pbc"], **MAT)
    m = inputs.smooth_tilt(W["shape"])
    ms, tq = _oracle_trajectory(p, _unit64(m), fn)
    n, bound = _bound(tq)
    md = to_dev(m)
    B.mm_load(s.ctx, md)
    B.mm_advance(s.ctx, method, NMAX, dt_s=DT, tol=tol, torque_tol=bound)
    B.mm_store(s.ctx, md)
    st = B.mm_get_stats(s.ctx)
    print(name, "oracle crossing at", n, "gpu accepted", st["accepted"], "torque", st["max_torque"], tq[n])
    assert st["done"] == 1 and st["status"] == 0
    assert st["accepted"] == n
    assert st["t"] == pytest.approx(n * DT, rel=1e-9, abs=0.0)
    assert st["max_torque"] == pytest.approx(tq[n], rel=1e-4, abs=0.0)
    assert float(np.max(np.abs(to_np(md) - ms[n]))) <= 1e-5
    # a second call finds the bound met at once and keeps the state
    B.mm_advance(s.ctx, method, 5, dt_s=DT, tol=tol, torque_tol=bound)
    st2 = B.mm_get_stats(s.ctx)
    assert st2["accepted"] == n and st2["done"] == 1


@pytest.mark.parametrize("name", ["euler", "heun"])
def test_torque_stop_then_plain_steps_continue_from_the_kept_state(name):
    """After a torque stop the next run (no bound) steps from the kept state:
    the spectrum of the rejected new state must not be reused."""
    method, tol, fn = STEPS[name]
    s = solver(W["shape"], W["cell"], pbc=W["pbc"], **MAT)
    p = oracle(W["shape"], W["cell"], pbc=W["pbc"], **MAT)
    m = inputs.smooth_tilt(W["shape"])
    ms, tq = _oracle_trajectory(p, _unit64(m), fn)
    n, bound = _bound(tq)
    md = to_dev(m)
    B.mm_load(s.ctx, md)
    B.mm_advance(s.ctx, method, NMAX, dt_s=DT, tol=tol, torque_tol=bound)
    B.mm_advance(s.ctx, method, 3, dt_s=DT, tol=tol)
    B.mm_store(s.ctx, md)
    st = B.mm_get_stats(s.ctx)
    assert st["accepted"] == n + 3
    assert float(np.max(np.abs(to_np(md) - ms[n + 3]))) <= 1e-5


@pytest.mark.parametrize("method,t_last", [(B.MM_EULER, 4.0), (B.MM_HEUN, 4.0), (B.MM_RK4, 3.5), (B.MM_RK3, 3.5)])
def test_fixed_step_run_ends_at_t_end(method, t_last):
    """Euler and Heun keep dt and stop at the first step at or past t_end;
    the tableau methods shorten their last step to end exactly there."""
    s = solver(W["shape"], W["cell"], pbc=W["pbc"], **MAT)
    md = to_dev(W["m"])
    B.mm_load(s.ctx, md)
    B.mm_advance(s.ctx, method, 50, dt_s=DT, t_end_s=3.5 * DT)
    st = B.mm_get_stats(s.ctx)
    assert st["done"] == 1 and st["accepted"] == 4
    assert st["t"] == pytest.approx(t_last * DT, rel=1e-9, abs=0.0)
