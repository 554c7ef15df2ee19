"""Planted mistakes in the oracle: each one must make a pin fail.

Every test below swaps one piece of the oracle for a plausibly wrong version
for the duration of that test only (pytest's monkeypatch; the oracle's files
are never edited), runs the pin that guards the piece, and requires the pin
to fail.  The mistakes are the kinds that a restatement of the paper can
make: a flipped sign, a dropped term or factor, a wrong axis, neighbour or
offset, a transposed operand, a perturbed coefficient, a wrong constant.
Nothing here touches the CUDA path.
"""

import numpy as np
import pytest

from oracle import demag, llg, newell, philox
from oracle import fields as F

import test_oracle_demag as TD
import test_oracle_fields as TF
import test_oracle_llg as TL
import test_oracle_newell as TN


def _caught(pin, *args):
    """The pin fails (an assertion of the pin, not an error of this file)."""
    with pytest.raises(AssertionError):
        pin(*args)


def _wrap(monkeypatch, module, name, outer):
    """Replace module.name by outer(original)."""
    monkeypatch.setattr(module, name, outer(getattr(module, name)))


# ---------------------------------------------------------------- exchange (Eq. 3)

def _exchange(skip_axis=None, boundary="free", one_spacing=False):
    """The 6-neighbour exchange field with one knob for each planted mistake:
    skip an axis, read a missing neighbour as the zero vector ("zero") or wrap
    an open axis ("wrap"), or use the x spacing on every axis."""
    def field(m, Ms, Aex, cell, pbc=(False, False, False)):
        m = np.asarray(m, float)
        H = np.zeros_like(m)
        for axis, d, per in ((3, cell[0], pbc[0]), (2, cell[1], pbc[1]), (1, cell[2], pbc[2])):
            if axis == skip_axis:
                continue
            d = cell[0] if one_spacing else d
            n = m.shape[axis]
            if n == 1 and not per:
                continue
            for shift in (1, -1):
                nb = np.roll(m, shift, axis=axis)
                if not per and boundary != "wrap":
                    edge = [slice(None)] * 4
                    edge[axis] = 0 if shift == 1 else n - 1
                    nb[tuple(edge)] = m[tuple(edge)] if boundary == "free" else 0.0
                H += (nb - m) / (d * d)
        return 2.0 * Aex / (F.MU0 * Ms) * H
    return field


def test_unplanted_exchange_variant_is_the_oracle():
    g = np.random.default_rng(0)
    m = g.standard_normal((3, 3, 4, 5))
    for pbc in ((False, False, False), (True, False, True)):
        np.testing.assert_array_equal(_exchange()(m, 8e5, 1.3e-11, (4e-9, 3e-9, 2e-9), pbc),
                                      F.exchange_field(m, 8e5, 1.3e-11, (4e-9, 3e-9, 2e-9), pbc))


def test_exchange_with_flipped_sign(monkeypatch):
    _wrap(monkeypatch, F, "exchange_field", lambda f: lambda *a, **k: -f(*a, **k))
    _caught(TF.test_spin_wave_eigenvalue, 1)


def test_exchange_without_its_factor_two(monkeypatch):
    _wrap(monkeypatch, F, "exchange_field", lambda f: lambda *a, **k: 0.5 * f(*a, **k))
    _caught(TF.test_bloch_wall_is_an_equilibrium_to_second_order)


def test_exchange_without_the_y_axis(monkeypatch):
    monkeypatch.setattr(F, "exchange_field", _exchange(skip_axis=2))
    _caught(TF.test_exchange_energy_equals_bond_sum)


def test_exchange_reading_missing_neighbours_as_zero(monkeypatch):
    monkeypatch.setattr(F, "exchange_field", _exchange(boundary="zero"))
    _caught(TF.test_free_boundary_three_cell_chain)


def test_exchange_wrapping_open_axes(monkeypatch):
    monkeypatch.setattr(F, "exchange_field", _exchange(boundary="wrap"))
    _caught(TF.test_free_boundary_three_cell_chain)


def test_exchange_with_one_spacing_for_all_axes(monkeypatch):
    monkeypatch.setattr(F, "exchange_field", _exchange(one_spacing=True))
    _caught(TF.test_exchange_energy_equals_bond_sum)


# --------------------------------------------------- anisotropy, Zeeman, energy

def test_uniaxial_anisotropy_without_the_factor_two(monkeypatch):
    _wrap(monkeypatch, F, "anisotropy_field", lambda f: lambda *a, **k: 0.5 * f(*a, **k))
    _caught(TF.test_anisotropy_closed_form)


def test_uniaxial_anisotropy_as_a_hard_axis(monkeypatch):
    _wrap(monkeypatch, F, "anisotropy_field", lambda f: lambda *a, **k: -f(*a, **k))
    _caught(TF.test_per_cell_anisotropy_axes_closed_form)


def test_zeeman_field_in_tesla_not_amperes_per_metre(monkeypatch):
    _wrap(monkeypatch, F, "zeeman_field", lambda f: lambda m, B: F.MU0 * f(m, B))
    _caught(TF.test_zeeman_energy)


def _energy(half_on_self=0.5, half_on_zeeman=1.0):
    def energy(m, Ms, V, Hd, Hex, Han, Hz):
        m = np.asarray(m, float)
        return -F.MU0 * Ms * V * (half_on_self * (m * (Hd + Hex + Han)).sum() + half_on_zeeman * (m * Hz).sum())
    return energy


def test_energy_without_the_half_on_self_interactions(monkeypatch):
    monkeypatch.setattr(F, "energy", _energy(half_on_self=1.0))
    _caught(TF.test_exchange_energy_equals_bond_sum)


def test_energy_with_a_half_on_the_zeeman_term(monkeypatch):
    monkeypatch.setattr(F, "energy", _energy(half_on_zeeman=0.5))
    _caught(TF.test_zeeman_energy)


def test_cubic_field_with_flipped_sign(monkeypatch):
    _wrap(monkeypatch, F, "cubic_anisotropy_field", lambda f: lambda *a, **k: -f(*a, **k))
    _caught(TF.test_cubic_anisotropy_is_minus_energy_gradient)


def test_cubic_field_without_the_K2_term(monkeypatch):
    _wrap(monkeypatch, F, "cubic_anisotropy_field",
          lambda f: lambda m, Ms, K1, K2, c1, c2: f(m, Ms, K1, 0.0, c1, c2))
    _caught(TF.test_cubic_anisotropy_is_minus_energy_gradient)


def test_cubic_energy_with_a_repeated_direction_cosine(monkeypatch):
    def density(m, K1, K2, c1, c2):
        a = [np.tensordot(c, m, axes=(0, 0)) for c in F.cubic_axes(c1, c2)]
        s = [x * x for x in a]
        return K1 * (s[0] * s[1] + s[1] * s[2] + s[0] * s[0]) + K2 * s[0] * s[1] * s[2]
    monkeypatch.setattr(F, "cubic_energy_density", density)
    _caught(TF.test_cubic_anisotropy_special_directions)


# ----------------------------------------------------- spin-transfer torque (Eq. 7)

def test_stt_with_the_current_derivative_reversed(monkeypatch):
    _wrap(monkeypatch, F, "current_derivative", lambda f: lambda *a, **k: -f(*a, **k))
    _caught(TF.test_stt_on_a_spiral_has_the_closed_form)


def test_stt_reading_missing_neighbours_as_zero(monkeypatch):
    def derivative(m, j, cell, pbc=(False, False, False)):
        m = np.asarray(m, float)
        u = np.zeros_like(m)
        for axis, jc, d, per in ((3, j[0], cell[0], pbc[0]), (2, j[1], cell[1], pbc[1]), (1, j[2], cell[2], pbc[2])):
            if jc == 0.0:
                continue
            n = m.shape[axis]
            up, dn = np.roll(m, -1, axis=axis), np.roll(m, 1, axis=axis)
            if not per:
                last, first = [slice(None)] * 4, [slice(None)] * 4
                last[axis], first[axis] = n - 1, 0
                up[tuple(last)] = 0.0
                dn[tuple(first)] = 0.0
            u += jc * (up - dn) / (2.0 * d)
        return u
    monkeypatch.setattr(F, "current_derivative", derivative)
    _caught(TF.test_current_derivative_on_an_open_three_cell_chain)


def test_stt_prefactor_without_one_plus_xi_squared(monkeypatch):
    monkeypatch.setattr(F, "stt_bj", lambda P, xi, Ms: P * F.MU_B / (F.E_CHARGE * Ms))
    _caught(TF.test_stt_on_a_spiral_has_the_closed_form)


# ------------------------------------------------------------ thermal field (Eq. 6)

def test_thermal_variance_without_the_factor_two(monkeypatch):
    _wrap(monkeypatch, F, "thermal_sigma", lambda f: lambda *a, **k: f(*a, **k) / np.sqrt(2.0))
    _caught(TL.test_langevin_statistics_of_thermal_macrospins)


def _eta(cell_of=lambda c: c, high_word=True):
    def eta(shape, seed, step):
        _, nz, ny, nx = shape
        cell = cell_of(np.arange(nz * ny * nx, dtype=np.uint64))
        hi = (int(step) >> 32) & 0xFFFFFFFF if high_word else 0
        w = philox.philox4x32_10(cell, int(step) & 0xFFFFFFFF, hi, 0,
                                 int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF)
        u = [philox.uniform_open(x) for x in w]
        r01, r23 = np.sqrt(-2.0 * np.log(u[0])), np.sqrt(-2.0 * np.log(u[2]))
        return np.stack([r01 * np.cos(2 * np.pi * u[1]), r01 * np.sin(2 * np.pi * u[1]),
                         r23 * np.cos(2 * np.pi * u[3])]).reshape(3, nz, ny, nx)
    return eta


def test_unplanted_noise_variant_is_the_oracle():
    np.testing.assert_array_equal(_eta()((3, 2, 5, 7), 99, 3 + (1 << 33)),
                                  philox.thermal_eta((3, 2, 5, 7), 99, 3 + (1 << 33)))


def test_noise_shared_by_neighbouring_cells(monkeypatch):
    monkeypatch.setattr(philox, "thermal_eta", _eta(cell_of=lambda c: c // np.uint64(2)))
    _caught(TF.test_gaussian_moments)


def test_noise_ignoring_the_high_word_of_the_step(monkeypatch):
    monkeypatch.setattr(philox, "thermal_eta", _eta(high_word=False))
    _caught(TF.test_gaussian_moments)


@pytest.mark.parametrize("name,value", [("_W1", 0xBB67AE86), ("_M0", 0xCD9E8D57)])
def test_philox_with_a_wrong_constant(monkeypatch, name, value):
    monkeypatch.setattr(philox, name, np.uint64(value))
    _caught(TF.test_philox_known_answers, *TF.KAT[2])


# --------------------------------------------------- demagnetising tensor (Eq. 2)

def test_newell_f_with_a_flipped_term(monkeypatch):
    def outer(f):
        def f_bad(x, y, z):
            x_, y_, z_ = np.broadcast_arrays(*(np.asarray(v, float) for v in (x, y, z)))
            R = np.sqrt(x_ * x_ + y_ * y_ + z_ * z_)
            return f(x, y, z) - (2 * x_ * x_ - y_ * y_ - z_ * z_) * R / 3.0   # sign of the R/6 term flipped
        return f_bad
    _wrap(monkeypatch, newell, "newell_f", outer)
    # the flipped term cancels in the trace, so by symmetry the cube's self
    # term stays 1/3; the point-dipole quadrature and Aharoni's prism factors,
    # both independent formulas, see it
    _caught(TN.test_closed_form_and_quadrature_agree, (1.0, 1.0, 1.0))
    _caught(TN.test_self_term_is_the_aharoni_prism_factor, (1.0, 2.0, 3.0))


def test_newell_g_without_its_last_term(monkeypatch):
    def outer(g):
        def g_bad(x, y, z):
            x_, y_, z_ = np.broadcast_arrays(*(np.asarray(v, float) for v in (x, y, z)))
            return g(x, y, z) + x_ * y_ * np.sqrt(x_ * x_ + y_ * y_ + z_ * z_) / 3.0   # -xyR/3 dropped
        return g_bad
    _wrap(monkeypatch, newell, "newell_g", outer)
    _caught(TN.test_closed_form_and_quadrature_agree, (1.0, 1.0, 1.0))


def test_newell_g_with_a_flipped_arctangent_term(monkeypatch):
    def outer(g):
        def g_bad(x, y, z):
            x_, y_, z_ = np.broadcast_arrays(*(np.asarray(v, float) for v in (x, y, z)))
            R = np.sqrt(x_ * x_ + y_ * y_ + z_ * z_)
            with np.errstate(divide="ignore", invalid="ignore"):
                t = np.where(z_ * y_ * y_ != 0, z_ * y_ * y_ * np.arctan(x_ * z_ / (y_ * R)), 0.0)
            return g(x, y, z) + t              # the sign of the z y^2/2 arctangent term flipped
        return g_bad
    _wrap(monkeypatch, newell, "newell_g", outer)
    _caught(TN.test_near_field_matches_fine_quadrature, (1.0, 1.0, 1.0), [(2, 1, 1), (2, 2, 2)], 16)


def test_newell_sum_with_a_wrong_centre_weight(monkeypatch):
    monkeypatch.setitem(newell._W, 0, 1.0)
    _caught(TN.test_offsite_trace_is_zero, (4.0, 4.0, 2.0))      # Laplace: the field is divergence-free


# -------------------------------------------- padded kernel and convolution (Sec. 3.2)

def test_kernel_with_negative_offsets_shifted_by_one(monkeypatch):
    def outer(f):
        def offsets(n, L, periodic, images):
            out = f(n, L, periodic, images)
            return out if periodic else [[o + 1 if o < 0 else o for o in lst] for lst in out]
        return offsets
    _wrap(monkeypatch, demag, "_axis_offsets", outer)
    _caught(TD.test_fft_matches_direct_sum_open, (4, 4, 1), (3.0, 3.0, 3.0))


def test_periodic_kernel_without_the_even_length_tie_break(monkeypatch):
    def outer(f):
        def offsets(n, L, periodic, images):
            out = f(n, L, periodic, images)
            if periodic and n % 2 == 0:
                out[n // 2] = out[n // 2][1:]        # one image fewer on the -n/2 side
            return out
        return offsets
    _wrap(monkeypatch, demag, "_axis_offsets", outer)
    _caught(TD.test_kernel_spectrum_is_real, (8, 6, 3), (True, True, False))


def test_convolution_with_transposed_off_diagonal_components(monkeypatch):
    def outer(f):
        def spectrum(K):
            Kh = f(K)
            Kh["xz"], Kh["yz"] = Kh["yz"], Kh["xz"]
            return Kh
        return spectrum
    _wrap(monkeypatch, demag, "kernel_spectrum", outer)
    _caught(TD.test_fft_matches_direct_sum_open, (5, 3, 2), (4.0, 4.0, 2.0))


def _field_fft(yx_sign=1.0):
    """Stages (i)-(iii) of the convolution with the sign of N_xy in the y row as a knob."""
    def field_fft(m, Ms, Khat, L):
        _, nz, ny, nx = m.shape
        Lx, Ly, Lz = L
        M = np.zeros((3, Lz, Ly, Lx))
        M[:, :nz, :ny, :nx] = Ms * m
        Mh = [np.fft.rfftn(M[c], axes=(0, 1, 2)) for c in range(3)]
        K = Khat
        Hh = [-(K["xx"] * Mh[0] + K["xy"] * Mh[1] + K["xz"] * Mh[2]),
              -(yx_sign * K["xy"] * Mh[0] + K["yy"] * Mh[1] + K["yz"] * Mh[2]),
              -(K["xz"] * Mh[0] + K["yz"] * Mh[1] + K["zz"] * Mh[2])]
        H = np.stack([np.fft.irfftn(Hh[c], s=(Lz, Ly, Lx), axes=(0, 1, 2)) for c in range(3)])
        return H[:, :nz, :ny, :nx].copy()
    return field_fft


def test_unplanted_convolution_variant_is_the_oracle():
    d = demag.Demag((5, 4, 3), (4.0, 3.0, 2.0))
    m = np.random.default_rng(4).standard_normal((3, 3, 4, 5))
    np.testing.assert_array_equal(_field_fft()(m, 2.0, d.Khat, d.L), demag.demag_field_fft(m, 2.0, d.Khat, d.L))


def test_demag_product_with_an_asymmetric_row(monkeypatch):
    # N_xy enters the y row with the wrong sign: the field is no longer the
    # gradient of an energy, so an undamped run stops conserving it
    monkeypatch.setattr(demag, "demag_field_fft", _field_fft(yx_sign=-1.0))
    _caught(TL.test_undamped_energy_drift_falls_with_the_method_order)


def test_demag_field_without_the_minus_sign(monkeypatch):
    _wrap(monkeypatch, demag, "demag_field_fft", lambda f: lambda *a, **k: -f(*a, **k))
    _caught(TD.test_uniform_body_mean_field, (16, 8, 1), (4.0, 4.0, 2.0), 0)
    _caught(TL.test_flat_cell_precesses_at_the_kittel_frequency)


def test_padding_shorter_than_2n_minus_1_is_refused(monkeypatch):
    # circular wrap-around instead of a linear convolution: the oracle refuses it
    monkeypatch.setattr(demag, "padded_length", lambda n, periodic: n)
    with pytest.raises(ValueError):
        TD.test_fft_matches_direct_sum_open((4, 4, 1), (3.0, 3.0, 3.0))


# ----------------------------------------- Landau-Lifshitz equation and integrators

def _ll(damping_sign=1.0, with_prefactor=True):
    def rhs(m, H, alpha, gamma0=F.GAMMA0):
        mxH = np.cross(m, H, axis=0)
        pre = gamma0 / (1.0 + alpha * alpha) if with_prefactor else gamma0
        return -pre * (mxH + damping_sign * alpha * np.cross(m, mxH, axis=0))
    return rhs


def test_unplanted_ll_variant_is_the_oracle():
    g = np.random.default_rng(1)
    m, H = g.standard_normal((3, 2, 3, 4)), g.standard_normal((3, 2, 3, 4))
    np.testing.assert_array_equal(_ll()(m, H, 0.3), llg.ll_rhs(m, H, 0.3))


def test_ll_with_anti_damping(monkeypatch):
    monkeypatch.setattr(llg, "ll_rhs", _ll(damping_sign=-1.0))
    _caught(TL.test_energy_never_increases_under_damping)


def test_ll_without_the_one_plus_alpha_squared(monkeypatch):
    monkeypatch.setattr(llg, "ll_rhs", _ll(with_prefactor=False))
    _caught(TL.test_macrospin_closed_form_rkdp, 0.5)


def test_dormand_prince_with_a_perturbed_stage_coefficient(monkeypatch):
    a = [list(row) for row in llg.DP_A]
    a[4][2] *= 1.0 + 1e-3                              # a_53 = 64448/6561
    monkeypatch.setattr(llg, "DP_A", tuple(tuple(row) for row in a))
    _caught(TL.test_macrospin_closed_form_rkdp, 0.02)


def test_dormand_prince_with_a_perturbed_embedded_weight(monkeypatch):
    b = list(llg.DP_BSTAR)
    b[6] *= 1.0 + 1e-2                                 # b*_7 = 1/40
    monkeypatch.setattr(llg, "DP_BSTAR", tuple(b))
    _caught(TL.test_embedded_error_estimate_is_order_five)


def test_heun_corrector_reusing_the_predictor_slope(monkeypatch):
    def heun(p, m, dt, step=0):
        k1 = p.rhs(m, step, dt)
        return llg.normalize(m + 0.5 * dt * (k1 + k1))
    monkeypatch.setattr(llg, "heun_step", heun)
    _caught(TL.test_convergence_orders)


def test_dissipation_with_flipped_sign(monkeypatch):
    _wrap(monkeypatch, F, "dissipation", lambda f: lambda *a, **k: -f(*a, **k))
    _caught(TL.test_dissipation_is_the_energy_rate_along_a_trajectory)


# --------------------------------------- the rest of the Runge-Kutta family (Sec. 2.2)

def _with_tableau(monkeypatch, name, **fields):
    t = llg.TABLEAUS[name]
    kw = dict(a=t.a, b=t.b, bstar=t.bstar, fsal=t.fsal, q=t.q)
    kw.update(fields)
    monkeypatch.setitem(llg.TABLEAUS, name, llg.Tableau(name, **kw))


def test_rk4_with_interior_and_end_weights_swapped(monkeypatch):
    _with_tableau(monkeypatch, "rk4", b=(1 / 3, 1 / 6, 1 / 6, 1 / 3))      # still sums to 1
    _caught(TL.test_tableau_convergence_orders, "rk4", 4, [8e-12, 4e-12])


def test_rk3_with_a_wrong_third_stage(monkeypatch):
    _with_tableau(monkeypatch, "rk3", a=((), (1 / 2,), (0.0, 1.0)))         # c3 = 1 kept, a31 dropped
    _caught(TL.test_tableau_convergence_orders, "rk3", 3, [4e-12, 2e-12])


@pytest.mark.parametrize("name,q", [("rk23", 3), ("rkck", 5)])
def test_embedded_weights_perturbed(monkeypatch, name, q):
    bs = list(llg.TABLEAUS[name].bstar)
    bs[0] *= 1.0 + 1e-2
    _with_tableau(monkeypatch, name, bstar=tuple(bs))
    _caught(TL.test_embedded_error_orders, name, q)


def test_max_variation_rule_on_the_mean_speed(monkeypatch):
    def step(p, m, tab, dm_max, h_cap=None):
        k1 = p.rhs(m)
        h = dm_max / float(np.sqrt((k1 * k1).sum(axis=0)).mean())        # mean instead of max
        if h_cap:
            h = min(h, h_cap)
        return llg.rk_attempt(p, m, h, tab, k1)[0], h
    monkeypatch.setattr(llg, "max_dm_step", step)
    _caught(TL.test_max_dm_step_size_is_the_first_order_variation)


def test_max_variation_rule_ignoring_the_cap(monkeypatch):
    _wrap(monkeypatch, llg, "max_dm_step", lambda f: lambda p, m, tab, dm_max, h_cap=None: f(p, m, tab, dm_max))
    _caught(TL.test_max_dm_step_size_is_the_first_order_variation)


def test_heun_drawing_new_noise_for_the_corrector(monkeypatch):
    def heun(p, m, dt, step=0):
        k1 = p.rhs(m, step, dt)
        k2 = p.rhs(m + dt * k1, step + (1 << 40), dt)         # an independent eta
        return llg.normalize(m + 0.5 * dt * (k1 + k2))
    monkeypatch.setattr(llg, "heun_step", heun)
    _caught(TL.test_langevin_statistics_of_thermal_macrospins)


# ------------------------------------------------ FFT sizes and periodic images (Sec. 3.3)

def test_fft_sizes_rounded_to_powers_of_two(monkeypatch):
    monkeypatch.setattr(demag, "_good_size", lambda n: 1 << max(0, (n - 1).bit_length()))
    _caught(TD.test_padded_length_rule)


def test_periodic_kernel_with_one_image_fewer(monkeypatch):
    def outer(f):
        def offsets(n, L, periodic, images):
            return f(n, L, periodic, images - 1 if periodic else images)
        return offsets
    _wrap(monkeypatch, demag, "_axis_offsets", outer)
    _caught(TD.test_fft_matches_direct_sum_periodic, (4, 3, 1), (True, False, False))


def test_controller_with_a_fourth_root(monkeypatch):
    def factor(err, tol, after_reject):
        f = 5.0 if err == 0.0 else 0.9 * (tol / err) ** 0.25
        f = min(max(f, 0.2), 5.0)
        return min(f, 1.0) if after_reject else f
    monkeypatch.setattr(llg, "controller_factor", factor)
    _caught(TL.test_controller_special_cases)


def test_controller_growing_right_after_a_reject(monkeypatch):
    _wrap(monkeypatch, llg, "controller_factor", lambda f: lambda err, tol, after_reject: f(err, tol, False))
    _caught(TL.test_controller_special_cases)


def test_dormand_prince_normalising_every_stage(monkeypatch):
    # a legitimate variant, but not the reading taken (only the candidate
    # m_{n+1} is renormalised): the generic tableau code, written separately,
    # disagrees with it
    def stages(p, m, h, k1=None):
        k = [p.rhs(m) if k1 is None else k1]
        for s in range(1, 6):
            ms = m.copy()
            for j, a in enumerate(llg.DP_A[s]):
                if a != 0.0:
                    ms = ms + h * a * k[j]
            k.append(p.rhs(llg.normalize(ms)))
        mn = m.copy()
        for j in range(6):
            if llg.DP_B[j] != 0.0:
                mn = mn + h * llg.DP_B[j] * k[j]
        mn = llg.normalize(mn)
        k.append(p.rhs(mn))
        e = sum(h * (llg.DP_B[j] - llg.DP_BSTAR[j]) * k[j] for j in range(7))
        return mn, k, float(np.sqrt((e * e).sum(axis=0)).max())
    monkeypatch.setattr(llg, "rkdp_stages", stages)
    _caught(TL.test_generic_dormand_prince_equals_the_dedicated_one)
