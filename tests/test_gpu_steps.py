"""GPU time steps (Euler, Heun, Dormand-Prince; fixed and adaptive; relaxation)
vs the FP64 oracle, plus the failure paths (non-finite state, step-size
underflow, unreached torque bound) reported as status codes."""

import numpy as np
import pytest

from oracle import llg
from paper_1102_3069_gb300 import binding as B
from paper_1102_3069_gb300 import inputs

from gpu_util import oracle, solver, to_dev, to_np

pytestmark = pytest.mark.gpu

W = inputs.workload("film_64x16")


def _pair(w=W, demag=True, **over):
    mat = dict(w["material"])
    mat.update(over)
    s = solver(w["shape"], w["cell"], pbc=w["pbc"], demag=demag, **mat)
    p = oracle(w["shape"], w["cell"], pbc=w["pbc"], demag=demag, **mat)
    return s, p


def _m64(m):
    m = m.astype(np.float64)
    return m / np.sqrt((m * m).sum(axis=0, keepdims=True))


@pytest.mark.parametrize("method,dt", [(B.MM_EULER, 1e-14), (B.MM_HEUN, 5e-14), (B.MM_RKDP, 1e-13)])
def test_single_step(method, dt):
    s, p = _pair()
    m = W["m"]
    md = to_dev(m)
    acc, t, dt_next = B.mm_step(s.ctx, md, method, 0.0, dt, tol=1.0)
    assert acc
    assert t == pytest.approx(dt, rel=1e-12, abs=0.0)
    m0 = _m64(m)
    if method == B.MM_EULER:
        ref = llg.euler_step(p, m0, dt)
    elif method == B.MM_HEUN:
        ref = llg.heun_step(p, m0, dt)
    else:
        ref = llg.rkdp_stages(p, m0, dt)[0]
    assert np.max(np.abs(to_np(md) - ref)) <= 1e-6


def test_thermal_heun_steps_match_oracle():
    w = inputs.workload("film_64x16")
    s, p = _pair(w, temperature=300.0, seed=77, alpha=0.05)
    m = w["m"]
    md = to_dev(m)
    dt = 20e-15
    ref = _m64(m)
    t = 0.0
    for k in range(5):
        acc, t, _ = B.mm_step(s.ctx, md, B.MM_HEUN, t, dt)
        ref = llg.heun_step(p, ref, dt, step=k)
    assert np.max(np.abs(to_np(md) - ref)) <= 2e-6


def _fixed_run(m, nsteps, h=1e-13):
    s, p = _pair()
    md = to_dev(m)
    B.mm_load(s.ctx, md)
    B.mm_advance(s.ctx, B.MM_RKDP, nsteps, dt_s=h, tol=-1.0)
    B.mm_store(s.ctx, md)
    st = B.mm_get_stats(s.ctx)
    assert st["accepted"] == nsteps and st["rejected"] == 0
    assert st["t"] == pytest.approx(nsteps * h, rel=1e-12, abs=0.0)
    ref = llg.rkdp_fixed(p, _m64(m), h, nsteps)
    return float(np.max(np.abs(to_np(md) - ref))), float(np.max(np.abs(ref - _m64(m))))


def test_thousand_fixed_rkdp_steps():
    """max |dm| <= 1e-5 after 1000 fixed Dormand-Prince steps of 100 fs on the
    64 x 16 film, from a smooth state whose trajectory is not chaotic (it moves
    by O(1) over the run)."""
    err, moved = _fixed_run(inputs.smooth_tilt(W["shape"]), 1000)
    print("max|dm| after 1000 fixed steps:", err, "state moved by", moved)
    assert moved > 0.5
    assert err <= 1e-5


def test_fixed_rkdp_steps_from_random_state():
    """From random unit vectors (alpha 0.02) the trajectory is chaotic: the FP64
    oracle alone turns a 1e-7 perturbation into 6e-5 after 200 steps and O(1)
    after 700.  The float32 path is held to 1e-5 over the first 50 steps."""
    err, _ = _fixed_run(W["m"], 50)
    print("max|dm| after 50 fixed steps from the random state:", err)
    assert err <= 1e-5


def test_adaptive_run_to_1ns_smooth_state():
    s, p = _pair()
    m = inputs.smooth_tilt(W["shape"])
    md = to_dev(m)
    B.mm_load(s.ctx, md)
    B.mm_advance(s.ctx, B.MM_RKDP, 100000, dt_s=1e-13, tol=1e-6, t_end_s=1e-9)
    B.mm_store(s.ctx, md)
    st = B.mm_get_stats(s.ctx)
    assert st["done"] == 1 and st["status"] == 0
    assert st["t"] == pytest.approx(1e-9, rel=1e-12, abs=0.0)
    ref = llg.Stepper(p, _m64(m), h0=1e-13, tol=1e-6)
    ref.run_until(1e-9)
    mg = to_np(md)
    print("steps gpu", st["accepted"], st["rejected"], "oracle", ref.accepted, ref.rejected,
          "max|dm|", np.max(np.abs(mg - ref.m)))
    assert abs(st["accepted"] - ref.accepted) <= 0.02 * ref.accepted + 2
    assert np.max(np.abs(mg - ref.m)) <= 1e-4


def test_adaptive_run_to_1ns_random_state():
    """The 64 x 16 film from random unit vectors, RKDP tol 1e-6 for 1 ns.  The
    trajectory is chaotic, so only run-level quantities are compared.  The
    oracle itself, restarted from 1e-7 perturbations of this state or rounded
    to float32 after every step, ends with 2809-3101 accepted steps and a
    dissipated energy (E0 - E)/|E0| of 0.9906-0.9964 (measured)."""
    s, p = _pair()
    m = W["m"]
    md = to_dev(m)
    B.mm_load(s.ctx, md)
    B.mm_advance(s.ctx, B.MM_RKDP, 100000, dt_s=1e-13, tol=1e-6, t_end_s=1e-9)
    B.mm_store(s.ctx, md)
    st = B.mm_get_stats(s.ctx)
    assert st["done"] == 1 and st["status"] == 0
    assert st["t"] == pytest.approx(1e-9, rel=1e-12, abs=0.0)
    ref = llg.Stepper(p, _m64(m), h0=1e-13, tol=1e-6)
    ref.run_until(1e-9)
    mg = to_np(md)
    E0, Eg, Eo = p.energy(_m64(m)), p.energy(mg), p.energy(ref.m)
    print("steps gpu", st["accepted"], st["rejected"], "oracle", ref.accepted, ref.rejected,
          "dissipated gpu", (E0 - Eg) / abs(E0), "oracle", (E0 - Eo) / abs(E0))
    assert abs(st["accepted"] - ref.accepted) <= 0.20 * ref.accepted
    assert np.max(np.abs(np.sqrt((mg * mg).sum(axis=0)) - 1.0)) <= 1e-6
    assert Eg < E0 and Eo < E0
    assert abs(Eg - Eo) <= 0.02 * abs(E0 - Eo)


def test_relax_reaches_bound_and_oracle_energy():
    w = dict(W)
    w["shape"] = (32, 8, 1)
    m = inputs.random_unit(w["shape"], 5)
    s, p = _pair(w, alpha=1.0)
    md = to_dev(m)
    steps, tq = B.mm_relax(s.ctx, md, torque_tol=1e-4, err_tol=1e-5, max_steps=20000)
    assert tq < 1e-4
    mg = to_np(md)
    assert p.torque(mg) < 2e-4          # float32 state re-evaluated in float64
    mo, _, _ = llg.relax(p, _m64(m), torque_tol=1e-4, tol=1e-5)
    Eg, Eo = p.energy(mg), p.energy(mo)
    assert Eg <= Eo + 1e-5 * abs(Eo)


def test_nonfinite_state_stops_with_status():
    s, _ = _pair()
    m = W["m"].copy()
    m[:, 0, 3, 5] = np.nan
    md = to_dev(m)
    with pytest.raises(B.MMError) as e:
        B.mm_step(s.ctx, md, B.MM_RKDP, 0.0, 1e-13, tol=1e-6)
    assert e.value.code == B.MM_ENONFINITE


def test_step_size_underflow_is_reported():
    s, _ = _pair()
    md = to_dev(W["m"])
    B.mm_load(s.ctx, md)
    B.mm_advance(s.ctx, B.MM_RKDP, 200, dt_s=1e-13, tol=1e-30)
    st = B.mm_get_stats(s.ctx)
    assert st["status"] == B.MM_ENOTCONVERGED and st["done"] == 1
    assert st["rejected"] > 5 and st["accepted"] == 0


def test_relax_budget_exhausted():
    s, _ = _pair(alpha=1.0)
    md = to_dev(W["m"])
    with pytest.raises(B.MMError) as e:
        B.mm_relax(s.ctx, md, torque_tol=1e-9, err_tol=1e-5, max_steps=10)
    assert e.value.code == B.MM_ENOTCONVERGED


def test_thermal_with_adaptive_method_is_refused():
    s, _ = _pair(temperature=300.0)
    md = to_dev(W["m"])
    B.mm_load(s.ctx, md)
    with pytest.raises(B.MMError) as e:
        B.mm_advance(s.ctx, B.MM_RKDP, 1, dt_s=1e-13, tol=1e-6)
    assert e.value.code == B.MM_EINVAL


def test_eval_without_kernel_is_refused():
    ctx = B.mm_init_geometry(8, 8, 1, 4e-9, 4e-9, 4e-9)
    import torch
    ws = torch.empty(B.mm_workspace_bytes(ctx) + 256, dtype=torch.uint8, device="cuda")
    B.mm_set_workspace(ctx, (ws.data_ptr() + 255) // 256 * 256, B.mm_workspace_bytes(ctx))
    B.mm_set_material(ctx, Ms=8e5, Aex=1.3e-11)
    m = to_dev(inputs.random_unit((8, 8, 1), 0))
    with pytest.raises(B.MMError) as e:
        B.mm_eval_heff(ctx, m, torch.empty_like(m))
    assert e.value.code == B.MM_ESTATE
    B.mm_destroy(ctx)


def test_host_buffer_run_matches_device_run():
    s, _ = _pair()
    mh = W["m"].copy()
    B.mm_run_host(s.ctx, mh, B.MM_RKDP, 5, dt_s=1e-13, tol=1e-6)
    md = to_dev(W["m"])
    B.mm_load(s.ctx, md)
    B.mm_advance(s.ctx, B.MM_RKDP, 5, dt_s=1e-13, tol=1e-6)
    B.mm_store(s.ctx, md)
    assert np.array_equal(mh, md.cpu().numpy())


@pytest.mark.parametrize("method,name", [(B.MM_EULER, "euler"), (B.MM_HEUN, "heun"), (B.MM_RK3, "rk3"),
                                         (B.MM_RK4, "rk4")])
@pytest.mark.parametrize("shape", [(40, 12, 1), (12, 9, 2)])
def test_max_dm_steps_match_oracle(method, name, shape):
    """Fixed maximum variation of m per step (Sec. 2.2): every step's size is
    max_dm / max|dm/dt(m_n)|; m and the accumulated time follow the oracle.
    (40, 12, 1) runs the split x passes, (12, 9, 2) the fused 3-D path."""
    cell = (4e-9, 4e-9, 3e-9)
    mat = dict(Ms=8e5, Aex=1.3e-11, Ku=2e4, easy_axis=(0.3, 0.0, 1.0), alpha=0.2, B=(0.0, 0.01, 0.02))
    s = solver(shape, cell, **mat)
    p = oracle(shape, cell, **mat)
    m = inputs.random_unit(shape, 21)
    md = to_dev(m)
    dm, n = 0.01, 12
    B.mm_set_max_dm(s.ctx, dm)
    B.mm_load(s.ctx, md)
    B.mm_advance(s.ctx, method, n, dt_s=0.0)
    B.mm_store(s.ctx, md)
    st = B.mm_get_stats(s.ctx)
    ref, t, hs = llg.max_dm_run(p, _m64(m), llg.MAXDM_TABLEAUS[name], dm, n)
    assert st["status"] == 0 and st["accepted"] == n
    assert st["evals"] == n * {"euler": 1, "heun": 2, "rk3": 3, "rk4": 4}[name]
    assert st["t"] == pytest.approx(t, rel=1e-4, abs=0.0)
    assert st["dt"] == pytest.approx(hs[-1], rel=1e-4, abs=0.0)          # the last step's size
    assert float(np.max(np.abs(to_np(md) - ref))) < 1e-5
    # a cap below the natural step size binds every step
    cap = 0.5 * min(hs)
    B.mm_load(s.ctx, to_dev(m))
    B.mm_advance(s.ctx, method, 4, dt_s=cap)
    st = B.mm_get_stats(s.ctx)
    assert st["t"] == pytest.approx(4 * cap, rel=1e-12, abs=0.0)
    # back to fixed steps: dt is required again
    B.mm_set_max_dm(s.ctx, 0.0)
    with pytest.raises(B.MMError):
        B.mm_advance(s.ctx, method, 1, dt_s=0.0)


@pytest.mark.parametrize("method,dt,tol", [(B.MM_RKDP, 0.0, 1e-5), (B.MM_RK23, 0.0, 1e-5), (B.MM_HEUN, 2e-14, 0.0)])
def test_checkpoint_resumes_bit_for_bit(method, dt, tol):
    """mm_get_state / mm_set_state: a run stopped after 25 steps and resumed in
    a fresh context ends exactly where an uninterrupted run of 25 + 20 steps
    ends (same m bits, same time, step size and counters)."""
    import torch
    s1, _ = _pair()
    m = to_dev(W["m"])
    first = 1e-13 if dt == 0.0 else dt
    B.mm_load(s1.ctx, m)
    B.mm_advance(s1.ctx, method, 25, dt_s=first, tol=tol)
    m_cp = torch.empty_like(m)
    cp = B.mm_get_state(s1.ctx, m_cp)
    assert cp["accepted"] >= 1 and cp["t"] > 0
    B.mm_advance(s1.ctx, method, 20, dt_s=dt, tol=tol)
    m_a = torch.empty_like(m)
    B.mm_store(s1.ctx, m_a)
    st_a = B.mm_get_stats(s1.ctx)
    s2, _ = _pair()
    B.mm_set_state(s2.ctx, m_cp, cp)
    assert B.mm_get_state(s2.ctx) == cp
    B.mm_advance(s2.ctx, method, 20, dt_s=dt, tol=tol)
    m_b = torch.empty_like(m)
    B.mm_store(s2.ctx, m_b)
    st_b = B.mm_get_stats(s2.ctx)
    torch.cuda.synchronize()
    assert torch.equal(m_a, m_b)
    for k in ("t", "dt", "accepted", "rejected", "step_index"):
        assert st_a[k] == st_b[k], k
    with pytest.raises(B.MMError):
        B.mm_set_state(s2.ctx, m_cp, dict(cp, dt=-1.0))


@pytest.mark.parametrize("method,dt", [(B.MM_RKDP, 1e-13), (B.MM_EULER, 1e-14)])
def test_steps_at_the_largest_fft_length(method, dt):
    """Time steps on a grid padded to 4096 points along x (the shared-memory
    x passes) against the oracle."""
    shape, cell = (2048, 3, 1), (4e-9, 4e-9, 4e-9)
    mat = dict(Ms=8e5, Aex=1.3e-11, Ku=5e3, easy_axis=(1.0, 0.0, 0.0), alpha=0.1, B=(0.0, 0.01, 0.0))
    s = solver(shape, cell, **mat)
    p = oracle(shape, cell, **mat)
    m = inputs.random_unit(shape, 5)
    md = to_dev(m)
    acc, t, _ = B.mm_step(s.ctx, md, method, 0.0, dt, tol=1.0)
    m0 = _m64(m)
    ref = llg.rkdp_stages(p, m0, dt)[0] if method == B.MM_RKDP else llg.euler_step(p, m0, dt)
    assert acc and float(np.max(np.abs(to_np(md) - ref))) < 1e-6


@pytest.mark.parametrize("method,dt,tol", [(B.MM_RKDP, 1e-13, -1.0), (B.MM_EULER, 1e-14, 0.0), (B.MM_HEUN, 2e-14, 0.0)])
@pytest.mark.parametrize("shape", [(40, 12, 1), (20, 70, 3)])
def test_pass_layouts_agree(method, dt, tol, shape):
    """The fused and the split x-pass layouts of a time step give the same
    trajectory up to float32 rounding (a few fixed steps from a non-chaotic
    start; with an adaptive step, rounding-level differences in the error
    estimate move the step size and with it the trajectory)."""
    import torch
    cell = (4e-9, 4e-9, 3e-9)
    mat = dict(Ms=8e5, Aex=1.3e-11, Ku=2e4, easy_axis=(0.3, 0.0, 1.0), alpha=0.2, B=(0.0, 0.01, 0.02))
    outs = []
    for layout in (B.MM_LAYOUT_FUSED, B.MM_LAYOUT_SPLIT):
        s = solver(shape, cell, **mat)
        B.mm_set_pass_layout(s.ctx, layout)
        md = to_dev(inputs.smooth_tilt(shape))
        B.mm_load(s.ctx, md)
        B.mm_advance(s.ctx, method, 8, dt_s=dt, tol=tol)
        B.mm_store(s.ctx, md)
        outs.append((md, B.mm_get_stats(s.ctx)))
    torch.cuda.synchronize()
    assert float((outs[0][0] - outs[1][0]).abs().max()) < 1e-6
    assert outs[0][1]["accepted"] == outs[1][1]["accepted"]
    with pytest.raises(B.MMError):
        B.mm_set_pass_layout(s.ctx, 7)


def test_pass_times_account_for_every_evaluation():
    """Per-pass event timing (mm_profile, mm_pass_times) of steps run without
    the step graph: every evaluation makes exactly one launch that ends in the
    cell terms, so those launches count the evaluations the device state
    reports; reading the times releases them, and a second read with nothing
    new run returns the same totals."""
    s, _ = _pair()
    md = to_dev(W["m"])
    B.mm_load(s.ctx, md)
    B.mm_profile(s.ctx, True)
    B.mm_advance(s.ctx, B.MM_RKDP, 3, dt_s=1e-13, tol=-1.0)
    t1 = B.mm_pass_times(s.ctx)
    st = B.mm_get_stats(s.ctx)
    cell_passes = ("k_xinv_local", "k_xinv_local_fused", "k_local", "k_local_h", "k_small")
    assert sum(v["launches"] for k, v in t1.items() if k in cell_passes) == st["evals"] == 19
    assert all(v["ms_total"] >= 0.0 for v in t1.values()) and sum(v["ms_total"] for v in t1.values()) > 0.0
    assert B.mm_pass_times(s.ctx) == t1
    B.mm_profile(s.ctx, False)


@pytest.mark.parametrize("method,dt,tol", [(B.MM_RKDP, 1e-13, -1.0), (B.MM_EULER, 1e-14, 0.0), (B.MM_HEUN, 2e-14, 0.0)])
@pytest.mark.parametrize("shape", [(40, 12, 1), (250, 64, 1)])
def test_film_term_set_kernel_agrees_with_general_kernel(method, dt, tol, shape):
    """A film with one easy axis and no cubic, thermal or spin-transfer terms
    runs the fused x kernel compiled for that term set; the same film with a
    per-cell easy axis equal to that axis in every cell runs the general
    kernel.  Both follow the same trajectory up to float32 rounding, and the
    first step matches the oracle."""
    import torch
    cell = (4e-9, 4e-9, 3e-9)
    ax = np.array([0.3, 0.0, 1.0]) / np.hypot(0.3, 1.0)
    mat = dict(Ms=8e5, Aex=1.3e-11, Ku=2e4, easy_axis=tuple(ax), alpha=0.2, B=(0.0, 0.01, 0.02))
    m = inputs.smooth_tilt(shape)
    outs = []
    # the library keeps the caller's pointer: the axes array must outlive the runs
    axes = to_dev(np.broadcast_to(ax.astype(np.float32)[:, None, None, None], (3,) + tuple(shape[::-1])).copy())
    for per_cell in (False, True):
        s = solver(shape, cell, **mat)
        B.mm_set_pass_layout(s.ctx, B.MM_LAYOUT_FUSED)      # the multi-kernel passes, not the cluster launch
        if per_cell:
            B.mm_set_anisotropy_axes(s.ctx, axes)
        md = to_dev(m)
        B.mm_load(s.ctx, md)
        B.mm_advance(s.ctx, method, 1, dt_s=dt, tol=tol)
        B.mm_store(s.ctx, md)
        first = to_np(md)
        B.mm_advance(s.ctx, method, 7, dt_s=dt, tol=tol)
        B.mm_store(s.ctx, md)
        outs.append((first, md, B.mm_get_stats(s.ctx)))
    torch.cuda.synchronize()
    assert float(np.max(np.abs(outs[0][0] - outs[1][0]))) < 1e-6
    assert float((outs[0][1] - outs[1][1]).abs().max()) < 1e-6
    assert outs[0][2]["accepted"] == outs[1][2]["accepted"]
    p = oracle(shape, cell, **mat)
    m0 = _m64(m)
    ref = (llg.rkdp_stages(p, m0, dt)[0] if method == B.MM_RKDP else
           llg.euler_step(p, m0, dt) if method == B.MM_EULER else llg.heun_step(p, m0, dt))
    assert float(np.max(np.abs(outs[0][0] - ref))) < 1e-6
