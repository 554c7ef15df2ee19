"""GPU effective field (mm_eval_heff) vs the FP64 oracle, element by element.

Bound: relative L2 error of H_eff <= 1e-6 and element-wise error <= 5e-6 of
max |H| (the FFT's float32 round-off grows like log2 of the padded length).
Shapes span single cells, odd and ragged sizes, several FFT tiles, 2-D and
3-D, open and periodic axes."""

import numpy as np
import pytest

from oracle import fields as F
from oracle import llg
from paper_1102_3069_gb300 import inputs

from gpu_util import HEFF_REL_L2, HEFF_REL_MAX, oracle, rel_l2, rel_max, solver, to_dev, to_np

pytestmark = pytest.mark.gpu

MAT = dict(Ms=8e5, Aex=1.3e-11, Ku=5e3, easy_axis=(1.0, 2.0, 3.0), alpha=0.1, B=(0.01, -0.02, 0.03))

SHAPES = [(1, 1, 1), (2, 1, 1), (1, 7, 1), (3, 5, 1), (5, 3, 2), (7, 8, 3), (8, 8, 1), (33, 7, 1),
          (64, 16, 1), (16, 12, 3), (100, 37, 1), (31, 17, 5), (20, 70, 3), (40, 33, 2)]


def _compare(shape, cell, pbc=(0, 0, 0), images=10, demag=True, seed=0, mat=MAT):
    m = inputs.random_unit(shape, seed)
    s = solver(shape, cell, pbc=pbc, images=images, demag=demag, **mat)
    h, tq, e = s.heff(to_dev(m), torque=True, energy=True)
    p = oracle(shape, cell, pbc=pbc, images=images, demag=demag, **mat)
    m64 = m.astype(np.float64)
    t = p.terms(m64)
    H = t["d"] + t["ex"] + t["an"] + t["z"]
    Hg = to_np(h)
    assert rel_l2(Hg, H) <= HEFF_REL_L2, rel_l2(Hg, H)
    assert rel_max(Hg, H) <= HEFF_REL_MAX, rel_max(Hg, H)
    dm = llg.ll_rhs(m64, H, p.alpha)
    assert rel_l2(to_np(tq), dm) <= 2 * HEFF_REL_L2
    E = F.energy(m64, p.Ms, p.V, t["d"], t["ex"], t["an"], t["z"])
    assert abs(e - E) <= 1e-6 * abs(E) + 1e-30
    return Hg, H


@pytest.mark.parametrize("shape", SHAPES)
def test_heff_open(shape):
    _compare(shape, (4e-9, 3e-9, 2e-9))


@pytest.mark.parametrize("shape,pbc", [((8, 8, 1), (1, 1, 0)), ((16, 4, 4), (1, 1, 0)), ((4, 6, 8), (0, 0, 1)),
                                       ((32, 5, 2), (1, 0, 0))])
def test_heff_periodic(shape, pbc):
    _compare(shape, (3e-9, 3e-9, 3e-9), pbc=pbc, images=3)


@pytest.mark.parametrize("shape", [(1, 1, 1), (33, 7, 1), (16, 12, 3)])
def test_local_terms_without_demag(shape):
    _compare(shape, (4e-9, 3e-9, 2e-9), demag=False)


def test_named_film_64x16():
    w = inputs.workload("film_64x16")
    _compare(w["shape"], w["cell"], mat=w["material"])


def test_energy_of_uniform_body_is_the_prism_value():
    # uniform m along x: E = mu0 Ms^2 Vtot N_xx(prism)/2 (only demag contributes)
    from oracle import newell
    shape, cell = (40, 10, 2), (4e-9, 4e-9, 2e-9)
    m = np.zeros((3, 2, 10, 40), np.float32)
    m[0] = 1.0
    s = solver(shape, cell, Ms=8e5, Aex=1.3e-11)
    _, _, e = s.heff(to_dev(m), energy=True)
    Nxx = float(newell.newell_tensor(0, 0, 0, 160e-9, 40e-9, 4e-9)["xx"])
    V = 40 * 10 * 2 * 4e-9 * 4e-9 * 2e-9
    E = 0.5 * F.MU0 * 8e5 ** 2 * V * Nxx
    assert abs(e - E) <= 5e-6 * E, (e, E)


def test_thermal_field_matches_oracle_bits():
    shape, cell = (24, 10, 2), (3e-9, 3e-9, 3e-9)
    mat = dict(Ms=1.1e6, Aex=2e-11, alpha=0.05, temperature=300.0, seed=123456789)
    m = inputs.random_unit(shape, 3)
    s = solver(shape, cell, demag=False, **mat)
    from paper_1102_3069_gb300 import binding as B
    dt = 50e-15
    for step in (0, 7, 2 ** 33 + 5):
        B.mm_set_thermal_clock(s.ctx, step, dt)
        h, _, _ = s.heff(to_dev(m))
        p = oracle(shape, cell, demag=False, **mat)
        t = p.terms(m.astype(np.float64), step=step, dt=dt)
        H = t["ex"] + t["z"] + t["th"]
        assert rel_l2(to_np(h), H) <= 2e-6
        # the noise itself is the dominant term: check it separately
        Hth_gpu = to_np(h) - (t["ex"] + t["z"])
        assert rel_max(Hth_gpu, t["th"]) <= 2e-5


def test_nonfinite_input_is_reported():
    from paper_1102_3069_gb300 import binding as B
    shape, cell = (8, 4, 1), (4e-9, 4e-9, 4e-9)
    m = inputs.random_unit(shape, 0)
    m[0, 0, 2, 3] = np.nan
    s = solver(shape, cell, **MAT)
    with pytest.raises(B.MMError) as e:
        s.heff(to_dev(m), energy=True)
    assert e.value.code == B.MM_ENONFINITE
    # the context stays usable
    m[0, 0, 2, 3] = 1.0
    s.heff(to_dev(m), energy=True)


@pytest.mark.parametrize("shape", [(33, 7, 1), (16, 12, 3)])
def test_cubic_anisotropy_matches_oracle(shape):
    from paper_1102_3069_gb300 import binding as B
    cell = (4e-9, 3e-9, 2e-9)
    K1, K2, c1, c2 = 4.8e4, -1.5e4, (1.0, 1.0, 0.0), (-1.0, 1.0, 0.5)
    m = inputs.random_unit(shape, 4)
    s = solver(shape, cell, **MAT)
    B.mm_set_cubic_anisotropy(s.ctx, K1, K2, c1, c2)
    h, tq, e = s.heff(to_dev(m), torque=True, energy=True)
    p = llg.Problem(shape, cell, MAT["Ms"], MAT["Aex"], MAT["alpha"], Ku=MAT["Ku"], u=MAT["easy_axis"], B=MAT["B"],
                    K1=K1, K2=K2, c1=c1, c2=c2)
    m64 = m.astype(np.float64)
    H = p.heff(m64)
    assert rel_l2(to_np(h), H) <= HEFF_REL_L2
    assert rel_l2(to_np(tq), llg.ll_rhs(m64, H, p.alpha)) <= 2 * HEFF_REL_L2
    E = p.energy(m64)
    assert abs(e - E) <= 2e-6 * abs(E), (e, E)
    with pytest.raises(B.MMError):
        B.mm_set_cubic_anisotropy(s.ctx, K1, K2, c1, c1)      # parallel axes


@pytest.mark.parametrize("shape,pbc", [((33, 7, 1), (0, 0, 0)), ((16, 12, 3), (1, 0, 0)), ((32, 8, 1), (1, 1, 0))])
def test_spin_transfer_torque_matches_oracle(shape, pbc):
    from paper_1102_3069_gb300 import binding as B
    cell = (4e-9, 3e-9, 2e-9)
    P, xi, j = 0.56, 0.05, (1e12, -4e11, 2e11)
    m = inputs.random_unit(shape, 6)
    s = solver(shape, cell, pbc=pbc, images=2, **MAT)
    B.mm_set_stt(s.ctx, P, xi, j)
    h, tq, _ = s.heff(to_dev(m), torque=True)
    p = llg.Problem(shape, cell, MAT["Ms"], MAT["Aex"], MAT["alpha"], Ku=MAT["Ku"], u=MAT["easy_axis"], B=MAT["B"],
                    pbc=tuple(bool(v) for v in pbc), images=2, stt_P=P, stt_xi=xi, stt_j=j)
    m64 = m.astype(np.float64)
    assert rel_l2(to_np(h), p.heff(m64)) <= HEFF_REL_L2          # a torque, not a field
    ref = p.rhs(m64)
    assert rel_l2(to_np(tq), ref) <= 2 * HEFF_REL_L2


@pytest.mark.parametrize("shape,pbc", [((33, 7, 1), (0, 0, 0)), ((16, 12, 3), (0, 0, 0)), ((64, 16, 1), (0, 0, 0)),
                                       ((16, 8, 4), (1, 1, 0))])
def test_per_cell_easy_axes_match_oracle(shape, pbc):
    """Eq. 4 with a different unit easy axis in every cell (any direction)."""
    from paper_1102_3069_gb300 import binding as B
    cell = (4e-9, 3e-9, 2e-9)
    axes = inputs.tilted_axes(shape, 5, max_deg=180.0)
    m = inputs.random_unit(shape, 9)
    mat = dict(MAT, Ku=4e4)
    s = solver(shape, cell, pbc=pbc, images=2, **mat)
    ax = to_dev(axes)
    B.mm_set_anisotropy_axes(s.ctx, ax)
    h, tq, e = s.heff(to_dev(m), torque=True, energy=True)
    p = oracle(shape, cell, pbc=pbc, images=2, **dict(mat, easy_axis=axes.astype(np.float64)))
    m64 = m.astype(np.float64)
    t = p.terms(m64)
    H = t["d"] + t["ex"] + t["an"] + t["z"]
    assert rel_l2(to_np(h), H) <= HEFF_REL_L2
    assert rel_max(to_np(h), H) <= HEFF_REL_MAX
    assert rel_l2(to_np(tq), llg.ll_rhs(m64, H, p.alpha)) <= 2 * HEFF_REL_L2
    E = p.energy(m64)
    assert abs(e - E) <= 2e-6 * abs(E), (e, E)
    # one Dormand-Prince step with the per-cell axes
    md = to_dev(m)
    acc, _, _ = B.mm_step(s.ctx, md, B.MM_RKDP, 0.0, 1e-13, tol=1.0)
    m0 = m64 / np.sqrt((m64 * m64).sum(axis=0, keepdims=True))
    ref = llg.rkdp_stages(p, m0, 1e-13)[0]
    assert acc and float(np.max(np.abs(to_np(md) - ref))) < 1e-6
    # NULL returns to the single axis of the material
    B.mm_set_anisotropy_axes(s.ctx, None)
    h1, _, _ = s.heff(to_dev(m))
    p1 = oracle(shape, cell, pbc=pbc, images=2, **mat)
    assert rel_l2(to_np(h1), p1.heff(m64)) <= HEFF_REL_L2


@pytest.mark.parametrize("shape,pbc", [((2048, 3, 1), (0, 0, 0)), ((3, 1500, 1), (0, 0, 0)), ((4096, 2, 1), (1, 0, 0)),
                                       ((1025, 4, 2), (0, 0, 0))])
def test_heff_largest_fft_lengths(shape, pbc):
    """The largest padded lengths the library accepts: 4096 along x and along
    y (open axes up to 2048 cells, periodic axes up to 4096), and just past a
    power of two (1025 -> 4096)."""
    _compare(shape, (4e-9, 3e-9, 2e-9), pbc=pbc, images=1)


@pytest.mark.parametrize("shape", [(33, 7, 1), (16, 12, 3), (64, 16, 1)])
def test_dissipation_matches_oracle(shape):
    """The FP64 sum of |m x H|^2 behind mm_stats.dissipation (damping's energy
    rate, Eq. 1) against the oracle."""
    from paper_1102_3069_gb300 import binding as B
    cell = (4e-9, 3e-9, 2e-9)
    m = inputs.random_unit(shape, 14)
    s = solver(shape, cell, **MAT)
    s.heff(to_dev(m), energy=True)
    st = B.mm_get_stats(s.ctx)
    p = oracle(shape, cell, **MAT)
    m64 = m.astype(np.float64)
    D = F.dissipation(m64, p.heff(m64), p.Ms, p.V, p.alpha)
    assert st["dissipation"] < 0
    assert st["dissipation"] == pytest.approx(D, rel=2e-6, abs=0.0)
