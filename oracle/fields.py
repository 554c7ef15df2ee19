"""Local effective-field terms, total H_eff and the micromagnetic energy (FP64).

Paper: Sec. 2.1 lists five contributions to H_eff (magnetostatic, exchange,
applied, anisotropy, thermal).

* exchange (Sec. 2.1.2, Eq. 3): H_ex = 2A/(mu0 Ms) lap(m), discretised with the
  6-neighbour scheme that drops to 4 neighbours when nz = 1.  A missing
  neighbour at an open boundary contributes nothing (free/Neumann boundary);
  periodic axes wrap.
* uniaxial anisotropy (Sec. 2.1.3, Eq. 4, phi = Ku sin^2 theta):
  H_an = 2 Ku/(mu0 Ms) (m . u) u, Ku > 0 an easy axis u (unit vector).
* cubic anisotropy (Sec. 2.1.3, Eq. 5): phi = K1 (a1^2 a2^2 + a2^2 a3^2 + a1^2 a3^2)
  + K2 a1^2 a2^2 a3^2 with direction cosines a_i = m . c_i to the orthonormal
  cubic axes c1, c2, c3 = c1 x c2; H_cub = -(1/(mu0 Ms)) dphi/dm
  = -(2/(mu0 Ms)) sum_i a_i [K1 (a_j^2 + a_k^2) + K2 a_j^2 a_k^2] c_i.
  phi is quartic, so its energy is summed directly (not as -mu0 Ms m.H/2).
* Zeeman: H_z = B / mu0 for an applied flux density B in tesla.
* spin-transfer torque (Sec. 2.1.4, Eq. 7, Zhang & Li): a torque, not a field:
  dm/dt += -b_j/(1+alpha^2) [m x (m x (j.grad)m) + (xi - alpha) m x (j.grad)m],
  b_j = P mu_B / (e Ms (1 + xi^2)); (j.grad)m by central differences with the
  free-boundary rule of the exchange stencil (a missing neighbour = the cell).
* thermal (Sec. 2.1.3, Eq. 6): H_th = eta sqrt(2 alpha kB T / (gamma0 mu0 Ms V dt)),
  eta ~ N(0,1) per cell, component and step (drawn by ``philox``).

Energy (not printed in the paper; the standard micromagnetic energy whose
variational derivative is the field above):
    E = - mu0 Ms V sum_i [ 1/2 m.(H_d + H_ex + H_an) + m.H_z ].

m: (3, nz, ny, nx) float64, unit vectors.  Fields in A/m, energy in J.
Pins: tests/test_oracle_fields.py (uniform state, spin-wave eigenvalue,
free-boundary chains for exchange and the current derivative, the Bloch wall
as an equilibrium to second order, closed-form anisotropy, energy = sum of
bond energies, cubic field = minus the energy gradient, the spin-transfer
torque on a spiral) and tests/test_oracle_llg.py (Langevin statistics).
"""

import numpy as np

MU0 = 4.0e-7 * np.pi          # H/m
KB = 1.380649e-23             # J/K
MU_B = 9.2740100783e-24       # J/T, Bohr magneton
E_CHARGE = 1.602176634e-19    # C
GAMMA0 = 2.211e5              # m/(A s): gamma acting on H in A/m (a reading)


def exchange_field(m, Ms, Aex, cell, pbc=(False, False, False)):
    """H_ex = 2A/(mu0 Ms) sum_axes sum_{existing nbr j} (m_j - m_i) / d_axis^2."""
    m = np.asarray(m, float)
    H = np.zeros_like(m)
    pref = 2.0 * Aex / (MU0 * Ms)
    # array axes: 3 -> x, 2 -> y, 1 -> z
    for axis, d, per in ((3, cell[0], pbc[0]), (2, cell[1], pbc[1]), (1, cell[2], pbc[2])):
        n = m.shape[axis]
        if n == 1 and not per:
            continue
        for shift in (1, -1):
            nb = np.roll(m, shift, axis=axis)           # value of the neighbour
            diff = nb - m
            if not per:
                # the neighbour of the first/last cell is missing: no contribution
                sl = [slice(None)] * 4
                sl[axis] = 0 if shift == 1 else n - 1
                diff[tuple(sl)] = 0.0
            H += diff / (d * d)
    return pref * H


def anisotropy_field(m, Ms, Ku, u):
    """H_an = 2 Ku/(mu0 Ms) (m.u) u; u shape (3,) or (3, nz, ny, nx), unit length."""
    m = np.asarray(m, float)
    u = np.asarray(u, float)
    if u.ndim == 1:
        u = u.reshape(3, 1, 1, 1)
    mu = (m * u).sum(axis=0, keepdims=True)
    return (2.0 * Ku / (MU0 * Ms)) * mu * u


def cubic_axes(c1, c2):
    """Orthonormal cubic axes from two given directions (Gram-Schmidt; c3 = c1 x c2)."""
    c1 = np.asarray(c1, float) / np.linalg.norm(c1)
    c2 = np.asarray(c2, float)
    c2 = c2 - c1 * (c1 @ c2)
    c2 = c2 / np.linalg.norm(c2)
    return c1, c2, np.cross(c1, c2)


def cubic_energy_density(m, K1, K2, c1, c2):
    """phi of Eq. 5 per cell (J/m^3); m shape (3, ...)."""
    a = [np.tensordot(c, m, axes=(0, 0)) for c in cubic_axes(c1, c2)]
    s = [x * x for x in a]
    return K1 * (s[0] * s[1] + s[1] * s[2] + s[0] * s[2]) + K2 * s[0] * s[1] * s[2]


def cubic_anisotropy_field(m, Ms, K1, K2, c1, c2):
    """H_cub = -(1/(mu0 Ms)) dphi/dm (A/m)."""
    m = np.asarray(m, float)
    cs = cubic_axes(c1, c2)
    a = [np.tensordot(c, m, axes=(0, 0)) for c in cs]
    s = [x * x for x in a]
    H = np.zeros_like(m)
    for i in range(3):
        j, k = (i + 1) % 3, (i + 2) % 3
        dphi = 2.0 * a[i] * (K1 * (s[j] + s[k]) + K2 * s[j] * s[k])
        H -= dphi[None] * cs[i].reshape((3,) + (1,) * (m.ndim - 1))
    return H / (MU0 * Ms)


def zeeman_field(m, B):
    """H_z = B/mu0 (uniform applied flux density B in T)."""
    B = np.asarray(B, float).reshape(3, 1, 1, 1)
    return np.broadcast_to(B / MU0, m.shape).copy()


def thermal_sigma(alpha, T, Ms, V, dt, gamma0=GAMMA0):
    """Standard deviation of each thermal-field component (A/m), Eq. 6."""
    return np.sqrt(2.0 * alpha * KB * T / (gamma0 * MU0 * Ms * V * dt))


def thermal_field(eta, alpha, T, Ms, V, dt, gamma0=GAMMA0):
    """H_th = eta * sigma, eta standard normal with shape of m."""
    return np.asarray(eta, float) * thermal_sigma(alpha, T, Ms, V, dt, gamma0)


def energy(m, Ms, V, Hd, Hex, Han, Hz):
    """E = -mu0 Ms V sum [ 1/2 m.(Hd+Hex+Han) + m.Hz ] (J)."""
    m = np.asarray(m, float)
    e = 0.5 * (m * (Hd + Hex + Han)).sum() + (m * Hz).sum()
    return -MU0 * Ms * V * e


def stt_bj(P, xi, Ms):
    """b_j = P mu_B / (e Ms (1 + xi^2)) of Sec. 2.1.4 (m^3/C: b_j j is a velocity)."""
    return P * MU_B / (E_CHARGE * Ms * (1.0 + xi * xi))


def current_derivative(m, j, cell, pbc=(False, False, False)):
    """(j . grad) m by central differences; at a free boundary the missing
    neighbour is replaced by the cell itself (zero normal derivative)."""
    m = np.asarray(m, float)
    u = np.zeros_like(m)
    for axis, jc, d, per in ((3, j[0], cell[0], pbc[0]), (2, j[1], cell[1], pbc[1]), (1, j[2], cell[2], pbc[2])):
        if jc == 0.0:
            continue
        n = m.shape[axis]
        up = np.roll(m, -1, axis=axis)          # neighbour at +1
        dn = np.roll(m, 1, axis=axis)           # neighbour at -1
        if not per:
            last = [slice(None)] * 4
            first = [slice(None)] * 4
            last[axis] = n - 1
            first[axis] = 0
            up[tuple(last)] = m[tuple(last)]
            dn[tuple(first)] = m[tuple(first)]
        u += jc * (up - dn) / (2.0 * d)
    return u


def stt_torque(m, alpha, P, xi, j, cell, Ms, pbc=(False, False, False)):
    """Zhang-Li spin-transfer torque of Eq. 7 divided by Ms (1/s):
    -b_j/(1+alpha^2) [ m x (m x (j.grad)m) + (xi - alpha) m x (j.grad)m ]."""
    u = current_derivative(m, j, cell, pbc)
    mxu = np.cross(m, u, axis=0)
    return -stt_bj(P, xi, Ms) / (1.0 + alpha * alpha) * (np.cross(m, mxu, axis=0) + (xi - alpha) * mxu)


def torque_max(m, H, Ms):
    """max_i |m_i x H_i| / Ms (dimensionless)."""
    c = np.cross(m, H, axis=0)
    return float(np.sqrt((c * c).sum(axis=0)).max() / Ms)


def dissipation(m, H, Ms, V, alpha, gamma0=GAMMA0):
    """Rate at which damping removes energy (W): with the LL right-hand side of
    Eq. 1 and a field that is minus the energy gradient (no spin-transfer
    torque, no thermal field), dE/dt = H.dm/dt summed = -mu0 Ms V gamma0 alpha
    / (1 + alpha^2) sum_i |m_i x H_i|^2 <= 0."""
    c = np.cross(m, H, axis=0)
    return -MU0 * Ms * V * gamma0 * alpha / (1.0 + alpha * alpha) * float((c * c).sum())
