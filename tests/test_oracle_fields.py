"""Pins for oracle.fields and oracle.philox.

* exchange: uniform state gives zero; a periodic spin wave m = (cos kx, sin kx, 0)
  is an exact eigenvector of the discrete Laplacian with eigenvalue
  -(2 - 2 cos k d)/d^2; at a free boundary a missing neighbour adds nothing
  (checked on a three-cell chain worked by hand);
* a Bloch wall theta = 2 atan(exp(x/D)), D = sqrt(A/K), is an equilibrium of
  exchange + anisotropy up to a residual torque that falls like (d/D)^2;
* exchange energy equals the bond sum A V sum_bonds |m_i - m_j|^2 / d^2;
* anisotropy: |H_an| = 2Ku/(mu0 Ms) cos(theta) along u; energy -Ku V cos^2;
  the same per cell with a different easy axis in every cell;
* Zeeman energy -Ms V m.B;
* demag energy of a uniformly magnetised body: mu0 Ms^2 Vtot N_prism / 2;
* Philox-4x32-10 known-answer vectors (Salmon et al., SC'11, Random123);
* the Gaussian draw has zero mean, unit variance, no cross-correlation.
"""

import numpy as np
import pytest

from oracle import fields as F
from oracle import demag, newell, philox

MS, AEX = 8e5, 1.3e-11


def test_uniform_state_has_no_exchange_field():
    m = np.zeros((3, 3, 4, 5))
    m[1] = 1.0
    for pbc in [(False,) * 3, (True, True, True)]:
        H = F.exchange_field(m, MS, AEX, (4e-9, 3e-9, 2e-9), pbc)
        assert np.max(np.abs(H)) == 0.0


@pytest.mark.parametrize("q", [1, 3, 7])
def test_spin_wave_eigenvalue(q):
    nx, d = 16, 3e-9
    k = 2 * np.pi * q / (nx * d)
    x = np.arange(nx) * d
    m = np.zeros((3, 1, 1, nx))
    m[0, 0, 0] = np.cos(k * x)
    m[1, 0, 0] = np.sin(k * x)
    H = F.exchange_field(m, MS, AEX, (d, 5e-9, 5e-9), (True, False, False))
    lam = -(2 - 2 * np.cos(k * d)) / d ** 2
    expect = 2 * AEX / (F.MU0 * MS) * lam * m
    assert np.max(np.abs(H - expect)) <= 1e-12 * np.max(np.abs(expect))


def test_free_boundary_three_cell_chain():
    d = 2e-9
    m = np.zeros((3, 1, 1, 3))
    m[:, 0, 0, 0] = (1, 0, 0)
    m[:, 0, 0, 1] = (0, 1, 0)
    m[:, 0, 0, 2] = (0, 0, 1)
    H = F.exchange_field(m, MS, AEX, (d, 1e-9, 1e-9))
    c = 2 * AEX / (F.MU0 * MS) / d ** 2
    np.testing.assert_allclose(H[:, 0, 0, 0], c * np.array([-1, 1, 0]), rtol=1e-14)     # only right nbr
    np.testing.assert_allclose(H[:, 0, 0, 1], c * np.array([1, -2, 1]), rtol=1e-14)
    np.testing.assert_allclose(H[:, 0, 0, 2], c * np.array([0, 1, -1]), rtol=1e-14)     # only left nbr


def test_bloch_wall_is_an_equilibrium_to_second_order():
    # the 180-degree wall theta(x) = 2 atan(exp(x/D)), D = sqrt(A/K), balances
    # exchange (Eq. 3) and uniaxial anisotropy (Eq. 4) exactly in the
    # continuum; on the lattice the residual torque falls like (d/D)^2
    A, K = 1.3e-11, 5e5
    D = np.sqrt(A / K)
    HK = 2 * K / (F.MU0 * MS)
    res = []
    for frac in (10, 20, 40):
        d = D / frac
        n = 40 * frac + 1
        x = (np.arange(n) - n // 2) * d
        th = 2 * np.arctan(np.exp(x / D))
        m = np.zeros((3, 1, 1, n))
        m[0, 0, 0], m[2, 0, 0] = np.sin(th), np.cos(th)
        H = F.exchange_field(m, MS, A, (d, d, d)) + F.anisotropy_field(m, MS, K, (0.0, 0.0, 1.0))
        res.append(float(np.linalg.norm(np.cross(m, H, axis=0), axis=0).max()) / HK)
        assert res[-1] <= 0.3 / frac ** 2
    assert np.log2(res[0] / res[1]) == pytest.approx(2.0, abs=0.05)
    assert np.log2(res[1] / res[2]) == pytest.approx(2.0, abs=0.05)


def test_exchange_energy_equals_bond_sum():
    rng = np.random.default_rng(5)
    nx, ny, nz = 6, 5, 3
    cell = (4e-9, 3e-9, 2e-9)
    m = rng.standard_normal((3, nz, ny, nx))
    m /= np.linalg.norm(m, axis=0)
    V = cell[0] * cell[1] * cell[2]
    H = F.exchange_field(m, MS, AEX, cell)
    z = np.zeros_like(m)
    E = F.energy(m, MS, V, z, H, z, z)
    bonds = 0.0
    for axis, d in ((3, cell[0]), (2, cell[1]), (1, cell[2])):
        diff = np.diff(m, axis=axis)
        bonds += (diff ** 2).sum() / d ** 2
    assert E == pytest.approx(AEX * V * bonds, rel=1e-12, abs=0.0)


def test_anisotropy_closed_form():
    Ku = 5e3
    u = np.array([1.0, 2.0, 2.0]) / 3.0
    th = np.linspace(0, np.pi, 7)
    perp = np.array([2.0, -1.0, 0.0]) / np.sqrt(5)
    m = (np.cos(th)[:, None] * u + np.sin(th)[:, None] * perp).T.reshape(3, 1, 1, 7)
    H = F.anisotropy_field(m, MS, Ku, u)
    expect = (2 * Ku / (F.MU0 * MS)) * np.cos(th)[None, :] * u[:, None]
    np.testing.assert_allclose(H.reshape(3, 7), expect, rtol=1e-13, atol=1e-9)
    V = 1e-25
    z = np.zeros_like(m)
    for i in range(7):
        mi = m[:, :, :, i:i + 1]
        Ei = F.energy(mi, MS, V, z[:, :, :, :1], z[:, :, :, :1], H[:, :, :, i:i + 1], z[:, :, :, :1])
        assert Ei == pytest.approx(-Ku * V * np.cos(th[i]) ** 2, rel=1e-12, abs=1e-40)


def test_per_cell_anisotropy_axes_closed_form():
    # each cell has its own easy axis u_i and sits at its own angle theta_i to it:
    # H_an,i = 2Ku/(mu0 Ms) cos(theta_i) u_i, energy -Ku V sum cos^2(theta_i)
    Ku, V = 2e4, 2.7e-26
    g = np.random.default_rng(7)
    n = 11
    u = g.standard_normal((3, n))
    u /= np.linalg.norm(u, axis=0)
    w = np.cross(u, g.standard_normal((3, n)), axis=0)
    w /= np.linalg.norm(w, axis=0)
    th = g.uniform(0, np.pi, n)
    m = np.cos(th) * u + np.sin(th) * w
    H = F.anisotropy_field(m.reshape(3, 1, 1, n), MS, Ku, u.reshape(3, 1, 1, n)).reshape(3, n)
    np.testing.assert_allclose(H, (2 * Ku / (F.MU0 * MS)) * np.cos(th) * u, rtol=1e-12, atol=1e-9)
    z = np.zeros((3, 1, 1, n))
    E = F.energy(m.reshape(3, 1, 1, n), MS, V, z, z, H.reshape(3, 1, 1, n), z)
    assert E == pytest.approx(-Ku * V * np.sum(np.cos(th) ** 2), rel=1e-12, abs=0.0)
    # a uniform axis field of per-cell copies is the uniform-axis result
    Hu = F.anisotropy_field(m.reshape(3, 1, 1, n), MS, Ku, u[:, 0])
    Hc = F.anisotropy_field(m.reshape(3, 1, 1, n), MS, Ku, np.repeat(u[:, :1], n, axis=1).reshape(3, 1, 1, n))
    np.testing.assert_array_equal(Hu, Hc)


def test_zeeman_energy():
    m = np.zeros((3, 1, 1, 2))
    m[:, 0, 0, 0] = (0.6, 0.8, 0.0)
    m[:, 0, 0, 1] = (0.0, 0.0, -1.0)
    B = np.array([0.01, -0.02, 0.03])
    V = 2e-26
    Hz = F.zeeman_field(m, B)
    z = np.zeros_like(m)
    E = F.energy(m, MS, V, z, z, z, Hz)
    assert E == pytest.approx(-MS * V * ((0.6 * 0.01 - 0.8 * 0.02) + (-0.03)), rel=1e-12, abs=0.0)


def test_uniform_body_demag_energy():
    shape, cell = (12, 6, 2), (4e-9, 4e-9, 2e-9)
    nx, ny, nz = shape
    m = np.zeros((3, nz, ny, nx))
    m[0] = 1.0
    V = cell[0] * cell[1] * cell[2]
    Hd = demag.Demag(shape, cell).field(m, MS)
    z = np.zeros_like(m)
    E = F.energy(m, MS, V, Hd, z, z, z)
    Nxx = float(newell.newell_tensor(0, 0, 0, nx * cell[0], ny * cell[1], nz * cell[2])["xx"])
    assert E == pytest.approx(0.5 * F.MU0 * MS ** 2 * V * nx * ny * nz * Nxx, rel=1e-10, abs=0.0)


KAT = [
    ((0x00000000, 0x00000000, 0x00000000, 0x00000000), (0x00000000, 0x00000000),
     (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
    ((0xffffffff, 0xffffffff, 0xffffffff, 0xffffffff), (0xffffffff, 0xffffffff),
     (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
    ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
     (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
]


@pytest.mark.parametrize("ctr,key,expect", KAT)
def test_philox_known_answers(ctr, key, expect):
    got = philox.philox4x32_10(*ctr, *key)
    assert tuple(int(v) for v in got) == expect


def test_gaussian_moments():
    eta = philox.thermal_eta((3, 1, 256, 256), seed=1234, step=7)
    x = eta.reshape(3, -1)
    n = x.shape[1]
    assert np.all(np.abs(x.mean(axis=1)) < 5 / np.sqrt(n))
    assert np.all(np.abs(x.var(axis=1) - 1.0) < 5 * np.sqrt(2.0 / n))
    c = np.corrcoef(x)
    assert np.all(np.abs(c[np.triu_indices(3, 1)]) < 5 / np.sqrt(n))
    # different step or seed -> different numbers (the step's high word counts too)
    assert not np.allclose(eta, philox.thermal_eta((3, 1, 256, 256), seed=1234, step=8))
    assert not np.allclose(eta, philox.thermal_eta((3, 1, 256, 256), seed=1235, step=7))
    assert not np.allclose(eta, philox.thermal_eta((3, 1, 256, 256), seed=1234, step=7 + (1 << 32)))
    # uncorrelated in space and time (Eq. 6): x and y neighbours, the next step
    e = eta.reshape(3, 256, 256)
    nxt = philox.thermal_eta((3, 1, 256, 256), seed=1234, step=8).reshape(3, 256, 256)
    for a, b in ((e[:, :, 1:], e[:, :, :-1]), (e[:, 1:, :], e[:, :-1, :]), (e, nxt)):
        for c in range(3):
            r = np.corrcoef(a[c].ravel(), b[c].ravel())[0, 1]
            assert abs(r) < 5 / np.sqrt(a[c].size), r


def test_uniform_open_interval_exact_in_binary32():
    w = np.array([0, 1, 511, 512, 0xFFFFFFFF], dtype=np.uint64)
    u = philox.uniform_open(w)
    assert np.all(u > 0) and np.all(u < 1)
    assert np.all(u.astype(np.float32).astype(np.float64) == u)


def test_thermal_sigma_units():
    # sigma^2 * gamma0 mu0 Ms V dt = 2 alpha kB T  (Eq. 6)
    s = F.thermal_sigma(0.05, 300.0, 1.1e6, 27e-27, 50e-15)
    assert s * s * F.GAMMA0 * F.MU0 * 1.1e6 * 27e-27 * 50e-15 == pytest.approx(2 * 0.05 * F.KB * 300.0, rel=1e-12, abs=0.0)


def test_cubic_anisotropy_is_minus_energy_gradient():
    rng = np.random.default_rng(9)
    m = rng.standard_normal((3, 1, 2, 3))
    K1, K2 = 4.5e4, -2.1e4
    c1, c2 = (1.0, 1.0, 0.0), (0.0, 0.3, 1.0)
    H = F.cubic_anisotropy_field(m, MS, K1, K2, c1, c2)
    eps = 1e-6
    for comp in range(3):
        d = np.zeros_like(m)
        d[comp] = eps
        g = (F.cubic_energy_density(m + d, K1, K2, c1, c2) - F.cubic_energy_density(m - d, K1, K2, c1, c2)) / (2 * eps)
        np.testing.assert_allclose(H[comp], -g / (F.MU0 * MS), rtol=1e-7, atol=1e-3)


def test_cubic_anisotropy_special_directions():
    K1, K2 = 4.8e4, 1.2e4
    c1, c2, c3 = F.cubic_axes((1.0, 0.0, 0.0), (0.0, 1.0, 0.0))
    m_axis = np.array([1.0, 0, 0]).reshape(3, 1, 1, 1)
    m_111 = (np.ones(3) / np.sqrt(3)).reshape(3, 1, 1, 1)
    m_110 = (np.array([1.0, 1.0, 0.0]) / np.sqrt(2)).reshape(3, 1, 1, 1)
    assert F.cubic_energy_density(m_axis, K1, K2, c1, c2).item() == pytest.approx(0.0, abs=1e-9)
    assert F.cubic_energy_density(m_111, K1, K2, c1, c2).item() == pytest.approx(K1 / 3 + K2 / 27, rel=1e-12, abs=0.0)
    assert F.cubic_energy_density(m_110, K1, K2, c1, c2).item() == pytest.approx(K1 / 4, rel=1e-12, abs=0.0)
    # along a cube axis, [110] and [111] the field is parallel to m (no torque)
    for mm in (m_axis, m_111, m_110):
        H = F.cubic_anisotropy_field(mm, MS, K1, K2, c1, c2)
        assert np.allclose(np.cross(mm, H, axis=0), 0.0, atol=1e-9)
    # the axes are orthonormal and right-handed
    assert np.allclose(np.array([c1, c2, c3]) @ np.array([c1, c2, c3]).T, np.eye(3))
    assert np.allclose(np.cross(c1, c2), c3)


def test_cubic_energy_decreases_under_damping():
    from oracle import llg
    shape = (6, 4, 1)
    rng = np.random.default_rng(3)
    m = rng.standard_normal((3, 1, 4, 6))
    m /= np.linalg.norm(m, axis=0)
    p = llg.Problem(shape, (4e-9, 4e-9, 4e-9), 8e5, 1.3e-11, 0.5, K1=5e4, K2=1e4, c1=(1, 1, 0), c2=(-1, 1, 0))
    st = llg.Stepper(p, m, h0=1e-14, tol=1e-7)
    E = [p.energy(st.m)]
    for _ in range(30):
        if st.step():
            E.append(p.energy(st.m))
    assert np.all(np.diff(E) <= 1e-7 * abs(E[0]))
    assert E[-1] < E[0]


def _spiral(n, k, d):
    x = np.arange(n) * d
    m = np.zeros((3, 1, 1, n))
    m[0, 0, 0] = np.cos(k * x)
    m[1, 0, 0] = np.sin(k * x)
    return m, x


def test_stt_vanishes_for_uniform_state_and_is_perpendicular():
    m = np.zeros((3, 2, 3, 4))
    m[2] = 1.0
    tq = F.stt_torque(m, 0.1, 0.5, 0.05, (1e12, -3e11, 2e11), (4e-9, 3e-9, 2e-9), MS)
    assert np.max(np.abs(tq)) == 0.0
    rng = np.random.default_rng(11)
    m = rng.standard_normal((3, 3, 4, 5))
    m /= np.linalg.norm(m, axis=0)
    tq = F.stt_torque(m, 0.1, 0.5, 0.05, (1e12, -3e11, 2e11), (4e-9, 3e-9, 2e-9), MS, pbc=(True, False, True))
    assert np.max(np.abs((m * tq).sum(axis=0))) <= 1e-9 * np.max(np.abs(tq))


def test_stt_on_a_spiral_has_the_closed_form():
    # m = (cos kx, sin kx, 0), periodic in x: (j.grad)m = j sin(kd)/d (-sin kx, cos kx, 0)
    n, d, q = 32, 2e-9, 3
    k = 2 * np.pi * q / (n * d)
    m, x = _spiral(n, k, d)
    P, xi, alpha, jx = 0.6, 0.05, 0.02, 1e12
    tq = F.stt_torque(m, alpha, P, xi, (jx, 0.0, 0.0), (d, 1e-9, 1e-9), MS, pbc=(True, False, False))
    c = jx * np.sin(k * d) / d
    u = c * np.stack([-np.sin(k * x), np.cos(k * x), np.zeros(n)])
    zhat = np.stack([np.zeros(n), np.zeros(n), c * np.ones(n)])
    bj = F.stt_bj(P, xi, MS)
    expect = -bj / (1 + alpha ** 2) * (-u + (xi - alpha) * zhat)
    np.testing.assert_allclose(tq[:, 0, 0, :], expect, rtol=1e-12, atol=1e-12 * np.abs(expect).max())
    assert bj == pytest.approx(P * F.MU_B / (F.E_CHARGE * MS * (1 + xi * xi)), rel=1e-15, abs=0.0)


def test_current_derivative_on_an_open_three_cell_chain():
    # central differences inside; at a free end the missing neighbour is the
    # cell itself, so the end cells take half the one-sided difference
    d, jx = 2e-9, 3e11
    m = np.zeros((3, 1, 1, 3))
    m[:, 0, 0, 0] = (1, 0, 0)
    m[:, 0, 0, 1] = (0, 1, 0)
    m[:, 0, 0, 2] = (0, 0, 1)
    u = F.current_derivative(m, (jx, 0.0, 0.0), (d, 1e-9, 1e-9))
    c = jx / (2 * d)
    np.testing.assert_allclose(u[:, 0, 0, 0], c * np.array([-1, 1, 0]), rtol=1e-14)     # (m1 - m0)
    np.testing.assert_allclose(u[:, 0, 0, 1], c * np.array([-1, 0, 1]), rtol=1e-14)     # (m2 - m0)
    np.testing.assert_allclose(u[:, 0, 0, 2], c * np.array([0, -1, 1]), rtol=1e-14)     # (m2 - m1)


def test_adiabatic_stt_advects_a_spiral():
    # xi = alpha and no field: dm/dt = b_j/(1+alpha^2) (j.grad)m, a rigid rotation of the
    # spiral about z at rate b_j j sin(kd)/d/(1+alpha^2) - a translation of the texture
    from oracle import llg
    n, d, q = 32, 2e-9, 2
    k = 2 * np.pi * q / (n * d)
    m, x = _spiral(n, k, d)
    P, alpha, jx = 0.7, 0.1, 2e12
    p = llg.Problem((n, 1, 1), (d, 1e-9, 1e-9), MS, 0.0, alpha, pbc=(True, False, False), demag=False,
                    stt_P=P, stt_xi=alpha, stt_j=(jx, 0.0, 0.0))
    w = F.stt_bj(P, alpha, MS) * jx * np.sin(k * d) / d / (1 + alpha ** 2)
    T = 0.4 / w
    mT = llg.rkdp_fixed(p, m, T / 200, 200)
    exact, _ = _spiral(n, k, d)
    exact = np.stack([np.cos(k * x + w * T), np.sin(k * x + w * T), np.zeros(n)])
    np.testing.assert_allclose(mT[:, 0, 0, :], exact, atol=1e-9)
