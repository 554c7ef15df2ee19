"""The one-launch cluster evaluation of small 2-D grids (MM_LAYOUT_CLUSTER):
H_eff, torque and energy against the FP64 oracle element by element, steps of
every method against the oracle and against the multi-kernel passes, every
term (exchange, uniaxial and cubic anisotropy, per-cell axes, Zeeman, thermal
field, spin-transfer torque), open and periodic x/y axes, ragged sizes and
each cluster size from 1 to 16 CTAs."""

import numpy as np
import pytest

from oracle import llg
from paper_1102_3069_gb300 import binding as B
from paper_1102_3069_gb300 import inputs

from gpu_util import HEFF_REL_L2, HEFF_REL_MAX, oracle, rel_l2, rel_max, solver, to_dev, to_np

pytestmark = pytest.mark.gpu

MAT = dict(Ms=8e5, Aex=1.3e-11, Ku=5e3, easy_axis=(1.0, 2.0, 3.0), alpha=0.1, B=(0.01, -0.02, 0.03))
CELL = (4e-9, 3e-9, 2e-9)

# (shape, pbc): cluster sizes 1 (<= 1024 cells), 2, 4, 8 and 16; odd and ragged
# sizes; a single row; periodic x, y and both
SHAPES = [((2, 1, 1), (0, 0, 0)), ((7, 1, 1), (0, 0, 0)), ((3, 5, 1), (0, 0, 0)), ((33, 7, 1), (0, 0, 0)),
          ((64, 16, 1), (0, 0, 0)), ((32, 32, 1), (0, 0, 0)), ((48, 40, 1), (0, 0, 0)),
          ((100, 37, 1), (0, 0, 0)), ((100, 80, 1), (0, 0, 0)), ((128, 128, 1), (0, 0, 0)),
          ((250, 64, 1), (0, 0, 0)), ((200, 256, 1), (0, 0, 0)), ((32, 8, 1), (1, 0, 0)),
          ((40, 16, 1), (0, 1, 0)), ((64, 64, 1), (1, 1, 0)), ((512, 8, 1), (1, 0, 0))]


def _cluster_solver(shape, pbc=(0, 0, 0), images=2, **mat):
    # the cluster launch needs power-of-two FFT lengths (the default rule may pick 2^a {3,5,7})
    s = solver(shape, CELL, pbc=pbc, images=images, fft_lengths=B.MM_FFT_POW2, **mat)
    B.mm_set_pass_layout(s.ctx, B.MM_LAYOUT_CLUSTER)
    return s


@pytest.mark.parametrize("shape,pbc", SHAPES)
def test_cluster_heff_matches_oracle(shape, pbc):
    m = inputs.random_unit(shape, 11)
    s = _cluster_solver(shape, pbc, **MAT)
    h, tq, e = s.heff(to_dev(m), torque=True, energy=True)
    p = oracle(shape, CELL, pbc=pbc, images=2, **MAT)
    m64 = m.astype(np.float64)
    t = p.terms(m64)
    H = t["d"] + t["ex"] + t["an"] + t["z"]
    Hg = to_np(h)
    assert rel_l2(Hg, H) <= HEFF_REL_L2, rel_l2(Hg, H)
    assert rel_max(Hg, H) <= HEFF_REL_MAX, rel_max(Hg, H)
    assert rel_l2(to_np(tq), llg.ll_rhs(m64, H, p.alpha)) <= 2 * HEFF_REL_L2
    E = p.energy(m64)
    assert abs(e - E) <= 2e-6 * abs(E), (e, E)
    # the one launch is what ran
    t1 = B.pass_times(s.ctx, lambda: s.heff(to_dev(m)))
    assert set(t1) == {"k_small"} and t1["k_small"]["launches"] == 1


def test_cluster_heff_every_term():
    """Cubic anisotropy, per-cell easy axes and the spin-transfer torque in
    the cluster launch (64 x 48, four CTAs), against the oracle."""
    shape = (64, 48, 1)
    K1, K2, c1, c2 = 4.8e4, -1.5e4, (1.0, 1.0, 0.0), (-1.0, 1.0, 0.5)
    P, xi, j = 0.56, 0.05, (1e12, -4e11, 0.0)
    axes = inputs.tilted_axes(shape, 5, max_deg=180.0)
    m = inputs.random_unit(shape, 4)
    mat = dict(MAT, Ku=4e4)
    s = _cluster_solver(shape, **mat)
    ax = to_dev(axes)                       # kept alive: the library holds the pointer
    B.mm_set_anisotropy_axes(s.ctx, ax)
    B.mm_set_cubic_anisotropy(s.ctx, K1, K2, c1, c2)
    B.mm_set_stt(s.ctx, P, xi, j)
    h, tq, e = s.heff(to_dev(m), torque=True, energy=True)
    p = llg.Problem(shape, CELL, mat["Ms"], mat["Aex"], mat["alpha"], Ku=mat["Ku"], u=axes.astype(np.float64),
                    B=mat["B"], K1=K1, K2=K2, c1=c1, c2=c2, images=2, stt_P=P, stt_xi=xi, stt_j=j)
    m64 = m.astype(np.float64)
    assert rel_l2(to_np(h), p.heff(m64)) <= HEFF_REL_L2
    assert rel_max(to_np(h), p.heff(m64)) <= HEFF_REL_MAX
    assert rel_l2(to_np(tq), p.rhs(m64)) <= 2 * HEFF_REL_L2
    E = p.energy(m64)
    assert abs(e - E) <= 2e-6 * abs(E), (e, E)


def test_cluster_thermal_field_matches_oracle():
    shape, cell = (40, 24, 1), (3e-9, 3e-9, 3e-9)
    mat = dict(Ms=1.1e6, Aex=2e-11, alpha=0.05, temperature=300.0, seed=123456789)
    m = inputs.random_unit(shape, 3)
    s = solver(shape, cell, images=2, fft_lengths=B.MM_FFT_POW2, **mat)
    B.mm_set_pass_layout(s.ctx, B.MM_LAYOUT_CLUSTER)
    dt = 50e-15
    p = oracle(shape, cell, images=2, **mat)
    for step in (0, 7, 2 ** 33 + 5):
        B.mm_set_thermal_clock(s.ctx, step, dt)
        h, _, _ = s.heff(to_dev(m))
        t = p.terms(m.astype(np.float64), step=step, dt=dt)
        H = t["d"] + t["ex"] + t["z"] + t["th"]
        assert rel_l2(to_np(h), H) <= 2e-6
        assert rel_max(to_np(h) - (t["d"] + t["ex"] + t["z"]), t["th"]) <= 2e-5


def _m64(m):
    m = m.astype(np.float64)
    return m / np.sqrt((m * m).sum(axis=0, keepdims=True))


@pytest.mark.parametrize("method,dt", [(B.MM_EULER, 1e-14), (B.MM_HEUN, 5e-14), (B.MM_RKDP, 1e-13),
                                       (B.MM_RK4, 5e-14), (B.MM_RKCK, 1e-13)])
@pytest.mark.parametrize("shape,pbc", [((64, 16, 1), (0, 0, 0)), ((100, 37, 1), (0, 0, 0)),
                                       ((64, 64, 1), (1, 1, 0))])
def test_cluster_step_matches_oracle(method, dt, shape, pbc):
    mat = dict(MAT, alpha=0.02)
    m = inputs.random_unit(shape, 5)
    s = _cluster_solver(shape, pbc, **mat)
    p = oracle(shape, CELL, pbc=pbc, images=2, **mat)
    md = to_dev(m)
    acc, t, _ = B.mm_step(s.ctx, md, method, 0.0, dt, tol=1.0)
    assert acc and t == pytest.approx(dt, rel=1e-12, abs=0.0)
    m0 = _m64(m)
    if method == B.MM_EULER:
        ref = llg.euler_step(p, m0, dt)
    elif method == B.MM_HEUN:
        ref = llg.heun_step(p, m0, dt)
    elif method == B.MM_RKDP:
        ref = llg.rkdp_stages(p, m0, dt)[0]
    else:
        name = {B.MM_RK4: "rk4", B.MM_RKCK: "rkck"}[method]
        ref = llg.rk_attempt(p, m0, dt, llg.TABLEAUS[name])[0]
    assert np.max(np.abs(to_np(md) - ref)) <= 1e-6


@pytest.mark.parametrize("method,dt,tol", [(B.MM_RKDP, 1e-13, -1.0), (B.MM_EULER, 1e-14, 0.0),
                                           (B.MM_HEUN, 2e-14, 0.0), (B.MM_RK4, 5e-14, 0.0)])
@pytest.mark.parametrize("shape", [(40, 12, 1), (128, 128, 1)])
def test_cluster_and_multi_kernel_trajectories_agree(method, dt, tol, shape):
    """20 fixed steps from a smooth start with the cluster launch and with the
    fused multi-kernel passes: the same trajectory up to float32 rounding.
    (With an adaptive step, rounding-level differences in the error estimate
    move the step size and with it the trajectory; the adaptive runs are
    compared with the oracle instead, below and in test_gpu_steps.py.)"""
    import torch
    cell = (4e-9, 4e-9, 3e-9)
    mat = dict(Ms=8e5, Aex=1.3e-11, Ku=2e4, easy_axis=(0.3, 0.0, 1.0), alpha=0.2, B=(0.0, 0.01, 0.02))
    outs = []
    for layout in (B.MM_LAYOUT_CLUSTER, B.MM_LAYOUT_FUSED):
        s = solver(shape, cell, fft_lengths=B.MM_FFT_POW2, **mat)
        B.mm_set_pass_layout(s.ctx, layout)
        md = to_dev(inputs.smooth_tilt(shape))
        B.mm_load(s.ctx, md)
        B.mm_advance(s.ctx, method, 20, dt_s=dt, tol=tol)
        B.mm_store(s.ctx, md)
        outs.append((md, B.mm_get_stats(s.ctx)))
    torch.cuda.synchronize()
    assert float((outs[0][0] - outs[1][0]).abs().max()) < 2e-6
    for k in ("accepted", "rejected", "evals"):
        assert outs[0][1][k] == outs[1][1][k], k
    assert outs[0][1]["t"] == pytest.approx(outs[1][1]["t"], rel=1e-9)


def test_cluster_thermal_heun_steps_match_oracle():
    w = inputs.workload("film_64x16")
    mat = dict(w["material"], temperature=300.0, seed=77, alpha=0.05)
    s = solver(w["shape"], w["cell"], **mat)
    B.mm_set_pass_layout(s.ctx, B.MM_LAYOUT_CLUSTER)
    p = oracle(w["shape"], w["cell"], **mat)
    md = to_dev(w["m"])
    dt = 20e-15
    ref = _m64(w["m"])
    t = 0.0
    for k in range(5):
        acc, t, _ = B.mm_step(s.ctx, md, B.MM_HEUN, t, dt)
        ref = llg.heun_step(p, ref, dt, step=k)
    assert np.max(np.abs(to_np(md) - ref)) <= 2e-6


def test_cluster_relax_and_torque_stop():
    """Relaxation (Dormand-Prince to max torque < 1e-4) and an Euler run
    stopped by the torque bound, through the cluster launch."""
    w = inputs.workload("film_64x16")
    mat = dict(w["material"], alpha=1.0)
    s = solver(w["shape"], w["cell"], **mat)
    B.mm_set_pass_layout(s.ctx, B.MM_LAYOUT_CLUSTER)
    md = to_dev(w["m"])
    n, tq = B.mm_relax(s.ctx, md, 1e-4, 1e-6, 50000)
    assert tq < 1e-4 and n > 0
    p = oracle(w["shape"], w["cell"], **mat)
    assert p.torque(to_np(md)) < 2e-4          # the float32 state re-evaluated in float64
    B.mm_load(s.ctx, md)
    B.mm_advance(s.ctx, B.MM_EULER, 100, dt_s=1e-14, torque_tol=1.0)
    st = B.mm_get_stats(s.ctx)
    assert st["done"] and st["accepted"] == 0 and st["max_torque"] < 1e-4


def test_cluster_layout_refused_where_it_does_not_apply():
    # 3-D; x padded to 1280 = 5 * 256; a half spectrum too large for 16 CTAs
    for shape in [(8, 8, 2), (600, 7, 1), (300, 300, 1)]:
        s = solver(shape, CELL, images=2, **MAT)
        with pytest.raises(B.MMError) as e:
            B.mm_set_pass_layout(s.ctx, B.MM_LAYOUT_CLUSTER)
        assert e.value.code == B.MM_EINVAL
        s.close()


def test_cluster_run_is_one_launch_and_auto_keeps_the_multi_kernel_passes():
    """With MM_LAYOUT_CLUSTER every evaluation is one launch of the cluster
    kernel (counted per evaluation while per-pass timing is on); the automatic
    layout keeps the multi-kernel passes (measured faster)."""
    shape = (64, 16, 1)
    s = solver(shape, CELL, **MAT)
    md = to_dev(inputs.random_unit(shape, 2))
    B.mm_load(s.ctx, md)
    t = B.pass_times(s.ctx, lambda: B.mm_advance(s.ctx, B.MM_RKDP, 3, dt_s=1e-13, tol=-1.0))
    assert "k_small" not in t
    B.mm_set_pass_layout(s.ctx, B.MM_LAYOUT_CLUSTER)
    B.mm_load(s.ctx, md)
    t = B.pass_times(s.ctx, lambda: B.mm_advance(s.ctx, B.MM_RKDP, 3, dt_s=1e-13, tol=-1.0))
    assert set(t) == {"k_small"}
    assert t["k_small"]["launches"] == B.mm_get_stats(s.ctx)["evals"] == 19


def test_cluster_adaptive_run_matches_oracle():
    """Adaptive Dormand-Prince over 0.1 ns from a smooth state through the
    cluster launch: the final state and the number of accepted steps against
    the oracle's own adaptive run."""
    shape = (48, 40, 1)
    mat = dict(MAT, alpha=0.2)
    m = inputs.smooth_tilt(shape)
    s = _cluster_solver(shape, **mat)
    p = oracle(shape, CELL, images=2, **mat)
    md = to_dev(m)
    B.mm_load(s.ctx, md)
    B.mm_advance(s.ctx, B.MM_RKDP, 100000, dt_s=1e-13, tol=1e-6, t_end_s=1e-10)
    B.mm_store(s.ctx, md)
    st = B.mm_get_stats(s.ctx)
    assert st["done"] == 1 and st["status"] == 0
    assert st["t"] == pytest.approx(1e-10, rel=1e-12, abs=0.0)
    ref = llg.Stepper(p, _m64(m), h0=1e-13, tol=1e-6)
    ref.run_until(1e-10)
    assert abs(st["accepted"] - ref.accepted) <= 0.02 * ref.accepted + 2
    assert float(np.max(np.abs(to_np(md) - ref.m))) <= 1e-4
