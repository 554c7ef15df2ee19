"""Pins for oracle.llg: Landau-Lifshitz right-hand side and the integrators.

Macrospin closed forms (one cubic cell: its own demag field is parallel to m
and exerts no torque; no exchange partner) with H = B/mu0 along z and
gamma' = gamma0/(1+alpha^2):
    phi(t) = phi0 + gamma' H t,   cos theta(t) = tanh(alpha gamma' H t + atanh cos theta0).
* Larmor: alpha = 0 precession at gamma0 H;
* Kittel: a single flat cell precesses about an in-plane field at
  gamma0 sqrt((H + (Nyy - Nxx) Ms)(H + (Nzz - Nxx) Ms)), its N from Aharoni's
  prism formula;
* uniaxial easy axis along the field (alpha = 0): precession at
  gamma0 (H + 2Ku/(mu0 Ms) cos theta0), which is Kittel's small-angle FMR
  frequency gamma0 (H + H_K) as theta0 -> 0;
* convergence orders 1 (Euler), 2 (Heun), 5 (Dormand-Prince) and order 5 of
  the embedded error estimate;
* energy is conserved without damping up to the integrator's O(h^5) drift
  (the field is the exact energy gradient); energy does not increase under damping; relaxation reaches the torque bound,
  and for a single cell it lands on the Stoner-Wohlfarth equilibrium angle;
* Langevin: an ensemble of uncoupled thermal macrospins in a field has
  <cos theta> = coth x - 1/x, x = mu0 Ms V H / (kB T), which fixes the variance
  of Eq. 6 and the noise interpretation of the Heun scheme.
"""

import numpy as np
import pytest

from oracle import fields as F
from oracle import llg

MS = 8e5
CELL = (4e-9, 4e-9, 4e-9)


def _macrospin(alpha, B=0.05, Ku=0.0):
    return llg.Problem((1, 1, 1), CELL, MS, 1.3e-11, alpha, Ku=Ku, u=(0, 0, 1), B=(0, 0, B))


def _m0(theta, phi):
    return np.array([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)]).reshape(3, 1, 1, 1)


def _exact(alpha, B, theta0, phi0, t):
    H = B / F.MU0
    gp = F.GAMMA0 / (1 + alpha ** 2)
    phi = phi0 + gp * H * t
    ct = np.tanh(alpha * gp * H * t + np.arctanh(np.cos(theta0)))
    st = np.sqrt(1 - ct * ct)
    return np.array([st * np.cos(phi), st * np.sin(phi), ct]).reshape(3, 1, 1, 1)


def test_rhs_direction_and_magnitude():
    # m along x, H along z: precession pushes m towards +y, damping towards +z
    m = _m0(np.pi / 2, 0.0)
    H = np.array([0, 0, 1e5]).reshape(3, 1, 1, 1)
    d = llg.ll_rhs(m, H, 0.1)
    gp = F.GAMMA0 / 1.01
    np.testing.assert_allclose(d.ravel(), [0.0, gp * 1e5, 0.1 * gp * 1e5], rtol=1e-14, atol=1e-6)


@pytest.mark.parametrize("alpha", [0.0, 0.02, 0.5])
def test_macrospin_closed_form_rkdp(alpha):
    B, th0, ph0 = 0.05, 1.0, 0.3
    p = _macrospin(alpha, B)
    h, n = 2e-13, 500
    m = llg.rkdp_fixed(p, _m0(th0, ph0), h, n)
    np.testing.assert_allclose(m, _exact(alpha, B, th0, ph0, h * n), atol=1e-10)


def test_larmor_frequency():
    B = 0.1
    p = _macrospin(0.0, B)
    T = 2 * np.pi / (F.GAMMA0 * B / F.MU0)           # one Larmor period
    n = 400
    m = llg.rkdp_fixed(p, _m0(0.7, 0.0), T / n, n)
    np.testing.assert_allclose(m, _m0(0.7, 0.0), atol=1e-9)


def test_uniaxial_precession_frequency():
    B, Ku, th0 = 0.02, 5e4, 0.4
    p = _macrospin(0.0, B, Ku)
    HK = 2 * Ku / (F.MU0 * MS)
    w = F.GAMMA0 * (B / F.MU0 + HK * np.cos(th0))
    t = 3.0 * 2 * np.pi / w
    n = 600
    m = llg.rkdp_fixed(p, _m0(th0, 0.0), t / n, n)
    np.testing.assert_allclose(m, _m0(th0, 0.0), atol=1e-9)


def test_flat_cell_precesses_at_the_kittel_frequency():
    # one 4 x 4 x 1 nm cell: its self-field (Eq. 2) is -N.M with the prism's
    # demagnetising factors, which Aharoni's closed form gives independently of
    # the oracle; small-angle precession about an in-plane field H along x then
    # has Kittel's frequency  w = gamma0 sqrt((H + (Nyy - Nxx) Ms)(H + (Nzz - Nxx) Ms))
    from closed_forms import aharoni_dz
    cell = (4e-9, 4e-9, 1e-9)
    Nxx, Nyy, Nzz = aharoni_dz(cell[1], cell[2], cell[0]), aharoni_dz(cell[2], cell[0], cell[1]), aharoni_dz(*cell)
    B = 0.05
    H = B / F.MU0
    T = 2 * np.pi / (F.GAMMA0 * np.sqrt((H + (Nyy - Nxx) * MS) * (H + (Nzz - Nxx) * MS)))
    p = llg.Problem((1, 1, 1), cell, MS, 1.3e-11, 0.0, B=(B, 0.0, 0.0))
    m = _m0(np.pi / 2 - 1e-3, 0.0)                  # 1 mrad off the field, towards +z
    n = 400
    h = T / n
    t, ys = [], []
    for i in range(3 * n + 5):
        t.append(i * h)
        ys.append(m[1].item())
        m = llg.rkdp_fixed(p, m, h, 1)
    cross = [t[i] - ys[i] * h / (ys[i + 1] - ys[i]) for i in range(len(ys) - 1) if ys[i] > 0 >= ys[i + 1]]
    assert len(cross) >= 2
    assert np.mean(np.diff(cross)) == pytest.approx(T, rel=1e-6, abs=0.0)


def _order(stepper, hs, T, alpha=0.1, B=0.05):
    p = _macrospin(alpha, B)
    errs = []
    for h in hs:
        n = int(round(T / h))
        m = _m0(1.0, 0.0)
        for k in range(n):
            m = stepper(p, m, h, k)
        errs.append(np.max(np.abs(m - _exact(alpha, B, 1.0, 0.0, n * h))))
    return np.log2(errs[0] / errs[1])


def test_convergence_orders():
    T = 1e-10
    assert _order(llg.euler_step, [1e-12, 5e-13], T) == pytest.approx(1.0, abs=0.15)
    assert _order(llg.heun_step, [2e-12, 1e-12], T) == pytest.approx(2.0, abs=0.15)

    def dp(p, m, h, k):
        return llg.rkdp_stages(p, m, h)[0]

    assert _order(dp, [1e-11, 5e-12], T) == pytest.approx(5.0, abs=0.3)


def test_embedded_error_estimate_is_order_five():
    p = _macrospin(0.1, 0.05)
    m = _m0(1.0, 0.0)
    e1 = llg.rkdp_stages(p, m, 4e-12)[2]
    e2 = llg.rkdp_stages(p, m, 2e-12)[2]
    assert np.log2(e1 / e2) == pytest.approx(5.0, abs=0.3)


def test_adaptive_run_hits_closed_form():
    alpha, B, th0, ph0 = 0.05, 0.05, 1.2, 0.0
    p = _macrospin(alpha, B)
    st = llg.Stepper(p, _m0(th0, ph0), h0=1e-13, tol=1e-9)
    st.run_until(2e-10)
    assert st.t == pytest.approx(2e-10, rel=1e-12, abs=0.0)
    np.testing.assert_allclose(st.m, _exact(alpha, B, th0, ph0, st.t), atol=100 * 1e-9)
    assert st.accepted > 10


def _random_film(alpha, seed=0, shape=(16, 8, 1), B=(0, 0, 0.01)):
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    m = rng.standard_normal((3, nz, ny, nx))
    m /= np.linalg.norm(m, axis=0)
    p = llg.Problem(shape, (4e-9, 4e-9, 4e-9), 8.6e5, 1.3e-11, alpha, B=B)
    return p, m


def test_controller_special_cases():
    # the step-size rule read for Sec. 2.2 (the paper gives none):
    # f = 0.9 (tol/err)^(1/q) clamped to [0.2, 5], at most 1 right after a reject
    tol = 1e-6
    f = llg.controller_factor
    assert f(tol, tol, False) == pytest.approx(0.9, rel=1e-15, abs=0.0)
    assert f(32 * tol, tol, False) == pytest.approx(0.45, rel=1e-15, abs=0.0)    # q = 5: 2^5 -> 1/2
    assert f(0.0, tol, False) == 5.0 and f(1e-30, tol, False) == 5.0
    assert f(1e6 * tol, tol, False) == 0.2
    assert f(1e-9 * tol, tol, True) == 1.0 and f(32 * tol, tol, True) == pytest.approx(0.45, rel=1e-15, abs=0.0)
    st = llg.TableauStepper(_macrospin(0.1), _m0(1.0, 0.0), llg.TABLEAUS["rk23"], tol=tol)
    assert st._factor(8 * tol, False) == pytest.approx(0.45, rel=1e-15, abs=0.0)                 # q = 3
    st = llg.TableauStepper(_macrospin(0.1), _m0(1.0, 0.0), llg.TABLEAUS["rk12"], tol=tol)
    assert st._factor(4 * tol, False) == pytest.approx(0.45, rel=1e-15, abs=0.0)                 # q = 2


def test_energy_never_increases_under_damping():
    p, m = _random_film(0.5)
    st = llg.Stepper(p, m, h0=1e-14, tol=1e-6)
    E = [p.energy(st.m)]
    for _ in range(40):
        if st.step():
            E.append(p.energy(st.m))
    E = np.array(E)
    scale = abs(E[0])
    assert np.all(np.diff(E) <= 1e-6 * scale)
    assert E[-1] < E[0]


def test_undamped_energy_drift_falls_with_the_method_order():
    # with alpha = 0, dm/dt is perpendicular to H_eff, and H_eff is minus the
    # energy gradient (a symmetric magnetostatic kernel, exchange, anisotropy,
    # Zeeman), so the energy is conserved; a Dormand-Prince run drifts only by
    # its local error, O(h^5) over a fixed time
    from paper_1102_3069_gb300 import inputs
    shape = (8, 6, 2)
    p = llg.Problem(shape, (4e-9, 3e-9, 2e-9), MS, 1.3e-11, 0.0, Ku=2e4, u=(0.3, 0.4, 1.0), B=(0.01, -0.02, 0.03))
    m0 = llg.normalize(inputs.smooth_tilt(shape).astype(np.float64))
    E0 = p.energy(m0)
    drift = [abs(p.energy(llg.rkdp_fixed(p, m0, h, int(round(2e-12 / h)))) - E0) / abs(E0) for h in (4e-14, 2e-14)]
    assert drift[1] < 1e-10
    assert np.log2(drift[0] / drift[1]) == pytest.approx(5.0, abs=0.3)


def test_candidate_norm_error_is_of_order_tol():
    p, m = _random_film(0.02, seed=3)
    h = 2e-14
    k1 = p.rhs(m)
    mn = m.copy()
    ks = [k1]
    for s in range(1, 7):
        ms = m.copy()
        for j, a in enumerate(llg.DP_A[s]):
            ms = ms + h * a * ks[j]
        ks.append(p.rhs(ms))
    for j in range(6):
        mn = mn + h * llg.DP_B[j] * ks[j]
    err = llg.rkdp_stages(p, m, h)[2]
    assert np.max(np.abs(np.linalg.norm(mn, axis=0) - 1.0)) < 10 * err + 1e-12


def test_relax_reaches_torque_bound():
    p, m = _random_film(1.0, seed=1, shape=(8, 4, 1))
    E0 = p.energy(m)
    mr, steps, tq = llg.relax(p, m, torque_tol=1e-4, tol=1e-5)
    assert tq < 1e-4
    assert p.torque(mr) < 1e-4
    assert p.energy(mr) < E0
    assert steps > 0


@pytest.mark.parametrize("psi_deg,B", [(30.0, 0.05), (60.0, 0.02), (80.0, 0.1), (45.0, 0.2)])
def test_relax_reaches_the_stoner_wohlfarth_angle(psi_deg, B):
    # one cubic cell (isotropic self-field, no exchange partner) with a uniaxial
    # axis along z and a field at psi from it: the relaxed state lies in the
    # x-z plane at the angle theta with Ku sin(2 theta) = mu0 Ms H sin(psi - theta),
    # found here by bracketing (scipy), independently of the oracle's dynamics
    from scipy.optimize import brentq
    Ku = 5e4
    psi = np.deg2rad(psi_deg)
    p = llg.Problem((1, 1, 1), CELL, MS, 1.3e-11, 1.0, Ku=Ku, u=(0, 0, 1),
                    B=(B * np.sin(psi), 0.0, B * np.cos(psi)))
    H = B / F.MU0
    theta = brentq(lambda th: Ku * np.sin(2 * th) + F.MU0 * MS * H * np.sin(th - psi), 0.0, psi)
    mr, steps, tq = llg.relax(p, _m0(psi, 0.0), torque_tol=1e-9, tol=1e-8)
    assert tq < 1e-9 and steps > 0
    assert abs(np.arctan2(mr[0].item(), mr[2].item()) - theta) < 1e-7
    assert abs(mr[1].item()) < 1e-7


def test_rkdp_refuses_thermal_noise():
    p = llg.Problem((2, 1, 1), CELL, MS, 1e-11, 0.1, T=300.0)
    with pytest.raises(ValueError):
        llg.rkdp_stages(p, _m0(0.5, 0.5).repeat(2, axis=3), 1e-13)


def test_langevin_statistics_of_thermal_macrospins():
    # uncoupled macrospins: no exchange partner effect (A = 0), no demag
    n = 4096
    T, x = 300.0, 2.0
    V = CELL[0] * CELL[1] * CELL[2]
    B = x * F.KB * T / (MS * V)
    dt = 0.02 / (F.GAMMA0 * B / F.MU0)
    p = llg.Problem((n, 1, 1), CELL, MS, 0.0, 1.0, B=(0, 0, B), T=T, seed=42, demag=False)
    m = np.zeros((3, 1, 1, n))
    m[2] = 1.0
    acc, cnt = 0.0, 0
    for k in range(3000):
        m = llg.heun_step(p, m, dt, k)
        if k >= 500 and k % 10 == 0:
            acc += m[2].mean()
            cnt += 1
    expect = 1.0 / np.tanh(x) - 1.0 / x
    assert acc / cnt == pytest.approx(expect, abs=0.01)


@pytest.mark.parametrize("name,order,hs", [("rk3", 3, [4e-12, 2e-12]), ("rk4", 4, [8e-12, 4e-12]),
                                          ("rk12", 2, [2e-12, 1e-12]), ("rk23", 3, [4e-12, 2e-12]),
                                          ("rkck", 5, [1e-11, 5e-12]), ("rkdp", 5, [1e-11, 5e-12])])
def test_tableau_convergence_orders(name, order, hs):
    tab = llg.TABLEAUS[name]

    def st(p, m, h, k):
        return llg.rk_attempt(p, m, h, tab)[0]

    assert _order(st, hs, 1e-10) == pytest.approx(order, abs=0.3)


@pytest.mark.parametrize("name,q", [("rk12", 2), ("rk23", 3), ("rkck", 5)])
def test_embedded_error_orders(name, q):
    p = _macrospin(0.1, 0.05)
    m = _m0(1.0, 0.0)
    tab = llg.TABLEAUS[name]
    e1 = llg.rk_attempt(p, m, 4e-12, tab)[2]
    e2 = llg.rk_attempt(p, m, 2e-12, tab)[2]
    assert np.log2(e1 / e2) == pytest.approx(q, abs=0.3)


def test_tableau_rows_are_consistent():
    # sum_j a_sj = c_s is implied; each row of a first-same-as-last tableau ends in b
    for tab in llg.TABLEAUS.values():
        assert sum(tab.b) == pytest.approx(1.0, abs=1e-15)
        if tab.bstar is not None:
            assert sum(tab.bstar) == pytest.approx(1.0, abs=1e-15)
        if tab.fsal:
            assert tuple(tab.a[-1]) == pytest.approx(tuple(tab.b[:-1]), abs=1e-15)
            assert tab.b[-1] == 0.0


def test_generic_dormand_prince_equals_the_dedicated_one():
    p, m = _random_film(0.05, seed=2, shape=(8, 4, 1))
    a = llg.rk_attempt(p, m, 3e-14, llg.TABLEAUS["rkdp"])
    b = llg.rkdp_stages(p, m, 3e-14)
    assert np.max(np.abs(a[0] - b[0])) < 1e-15
    assert a[2] == pytest.approx(b[2], rel=1e-12, abs=0.0)


@pytest.mark.parametrize("name", ["rk12", "rk23", "rkck"])
def test_adaptive_tableaus_hit_the_closed_form(name):
    alpha, B, th0 = 0.05, 0.05, 1.2
    p = _macrospin(alpha, B)
    st = llg.TableauStepper(p, _m0(th0, 0.0), llg.TABLEAUS[name], h0=1e-13, tol=1e-8)
    st.run_until(1e-10)
    assert st.t == pytest.approx(1e-10, rel=1e-12, abs=0.0)
    np.testing.assert_allclose(st.m, _exact(alpha, B, th0, 0.0, st.t), atol=2e-5)


# ---- fixed maximum variation of m per step (Sec. 2.2) -----------------------

def test_max_dm_step_size_is_the_first_order_variation():
    # Euler with the max-variation rule: the fastest cell moves by dm_max before
    # normalisation, every other cell by less, and h = dm_max / max |dm/dt|
    p = llg.Problem((6, 4, 1), CELL, MS, 1.3e-11, 0.1, Ku=3e4, u=(0, 0.6, 0.8), B=(0.01, 0, 0.02))
    g = np.random.default_rng(3)
    m = llg.normalize(g.standard_normal(p.mshape))
    k1 = p.rhs(m)
    dm = 0.02
    m1, h = llg.max_dm_step(p, m, llg.MAXDM_TABLEAUS["euler"], dm)
    move = np.sqrt(((h * k1) ** 2).sum(axis=0))
    assert move.max() == pytest.approx(dm, rel=1e-14, abs=0.0)
    np.testing.assert_allclose(m1, llg.normalize(m + h * k1), rtol=0, atol=1e-15)
    # the cap wins when it is smaller
    _, hc = llg.max_dm_step(p, m, llg.MAXDM_TABLEAUS["euler"], dm, h_cap=0.5 * h)
    assert hc == 0.5 * h


@pytest.mark.parametrize("name", ["euler", "heun", "rk3", "rk4"])
def test_max_dm_tableaus_equal_the_fixed_step_methods(name):
    # with the same h the max-variation step is the method's own step
    p = _macrospin(0.1)
    m = _m0(1.0, 0.2)
    _, h = llg.max_dm_step(p, m, llg.MAXDM_TABLEAUS[name], 0.01)
    ref = {"euler": lambda: llg.euler_step(p, m, h), "heun": lambda: llg.heun_step(p, m, h),
           "rk3": lambda: llg.rk_fixed(p, m, h, 1, llg.TABLEAUS["rk3"]),
           "rk4": lambda: llg.rk_fixed(p, m, h, 1, llg.TABLEAUS["rk4"])}[name]()
    mn, _ = llg.max_dm_step(p, m, llg.MAXDM_TABLEAUS[name], 0.01)
    np.testing.assert_allclose(mn, ref, atol=1e-15)


@pytest.mark.parametrize("name,order", [("euler", 1), ("heun", 2), ("rk4", 4)])
def test_max_dm_runs_follow_the_closed_form_with_the_method_order(name, order):
    # the macrospin's |dm/dt| = gamma' H sin(theta) sqrt(1+alpha^2) shrinks as it
    # damps, so the steps grow; the state after N steps must match the closed
    # form at the accumulated time, with an error that falls as dm_max^order
    alpha, B, th0, ph0 = 0.1, 0.05, 1.2, 0.3
    p = _macrospin(alpha, B)
    tab = llg.MAXDM_TABLEAUS[name]
    errs = []
    for dm in (0.02, 0.01):
        m, t, hs = llg.max_dm_run(p, _m0(th0, ph0), tab, dm, int(round(4.0 / dm)))
        assert hs[-1] > hs[0]                        # slower precession, larger steps
        errs.append(float(np.abs(m - _exact(alpha, B, th0, ph0, t)).max()))
    assert np.log2(errs[0] / errs[1]) == pytest.approx(order, abs=0.3)
    assert errs[1] < {1: 3e-2, 2: 3e-4, 4: 1e-7}[order]


def test_dissipation_is_the_energy_rate_along_a_trajectory():
    # dE/dt from a one-sided second-order difference of the energy along a
    # Dormand-Prince trajectory equals -mu0 Ms V gamma' alpha sum |m x H|^2
    p = llg.Problem((8, 6, 1), CELL, MS, 1.3e-11, 0.3, Ku=2e4, u=(0.2, 0.4, 1.0), B=(0.01, -0.02, 0.03))
    g = np.random.default_rng(12)
    m0 = llg.normalize(g.standard_normal(p.mshape))
    h = 2e-15
    m1 = llg.rkdp_fixed(p, m0, h, 1)
    m2 = llg.rkdp_fixed(p, m1, h, 1)
    E = [p.energy(x) for x in (m0, m1, m2)]
    dEdt = (-3 * E[0] + 4 * E[1] - E[2]) / (2 * h)
    D = F.dissipation(m0, p.heff(m0), p.Ms, p.V, p.alpha)
    assert D < 0
    assert dEdt == pytest.approx(D, rel=1e-4, abs=0.0)
    # no damping, no dissipation
    p0 = llg.Problem((8, 6, 1), CELL, MS, 1.3e-11, 0.0, Ku=2e4, u=(0.2, 0.4, 1.0), B=(0.01, -0.02, 0.03))
    assert F.dissipation(m0, p0.heff(m0), p0.Ms, p0.V, 0.0) == 0.0
