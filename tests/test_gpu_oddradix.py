"""FFT lengths with an odd factor (Sec. 3.3: sizes 2^n {1,3,5,7}) against the
oracle.  An open axis of n cells pads to the smallest 2^k or r * 2^l
(r = 3, 5, 7) >= 2n - 1, a periodic axis may have r * 2^l cells; the passes
along that axis then take a first radix-r pass before the power-of-two
passes, and the kernel setup's FP64 FFT does the same.  The oracle pads by its own rule
(any length >= 2n - 1 gives the same linear convolution).

Bounds as everywhere: relative L2 error of H_eff <= 1e-6, element-wise
<= 5e-6 of max |H|; one step within 1e-6 of the oracle."""

import numpy as np
import pytest

from oracle import llg
from paper_1102_3069_gb300 import binding as B
from paper_1102_3069_gb300 import inputs

from gpu_util import HEFF_REL_L2, HEFF_REL_MAX, oracle, rel_l2, rel_max, solver, to_dev, to_np

pytestmark = pytest.mark.gpu

MAT = dict(Ms=8e5, Aex=1.3e-11, Ku=5e3, easy_axis=(1.0, 2.0, 3.0), alpha=0.1, B=(0.01, -0.02, 0.03))


def _unit64(m):
    m = m.astype(np.float64)
    return m / np.sqrt((m * m).sum(axis=0, keepdims=True))


# (shape, pbc, x length the library pads to)
CASES = [((130, 9, 1), (0, 0, 0), 320), ((600, 7, 1), (0, 0, 0), 1280), ((700, 5, 1), (0, 0, 0), 1536),
         ((1700, 3, 1), (0, 0, 0), 3584), ((1500, 2, 1), (0, 0, 0), 3072), ((96, 12, 3), (0, 0, 0), 192),
         ((192, 8, 1), (1, 0, 0), 192), ((320, 4, 2), (1, 0, 0), 320), ((448, 8, 1), (1, 1, 0), 448)]
# odd factors along y (2-D column pass, 3-D y passes) and z (3-D column pass)
CASES_YZ = [((9, 130, 1), (0, 0, 0)), ((5, 600, 1), (0, 0, 0)), ((8, 448, 1), (0, 1, 0)), ((6, 96, 3), (0, 0, 0)),
            ((7, 160, 2), (0, 0, 0)), ((4, 5, 96), (0, 0, 0)), ((6, 4, 130), (0, 0, 0)), ((8, 8, 192), (0, 0, 1)),
            ((96, 130, 40), (0, 0, 0)), ((192, 64, 5), (1, 1, 0))]


@pytest.mark.parametrize("shape,pbc,px", CASES)
def test_heff_at_odd_x_lengths(shape, pbc, px):
    cell = (4e-9, 3e-9, 2e-9)
    m = inputs.random_unit(shape, 31)
    s = solver(shape, cell, pbc=pbc, images=2, **MAT)
    h, tq, e = s.heff(to_dev(m), torque=True, energy=True)
    p = oracle(shape, cell, pbc=pbc, images=2, **MAT)
    m64 = m.astype(np.float64)
    t = p.terms(m64)
    H = t["d"] + t["ex"] + t["an"] + t["z"]
    Hg = to_np(h)
    print(shape, pbc, "x length", px, "rel L2", rel_l2(Hg, H), "rel max", rel_max(Hg, H))
    assert rel_l2(Hg, H) <= HEFF_REL_L2
    assert rel_max(Hg, H) <= HEFF_REL_MAX
    assert rel_l2(to_np(tq), llg.ll_rhs(m64, H, p.alpha)) <= 2 * HEFF_REL_L2
    E = p.energy(m64)
    assert abs(e - E) <= 2e-6 * abs(E), (e, E)


@pytest.mark.parametrize("shape,pbc", CASES_YZ)
def test_heff_at_odd_y_and_z_lengths(shape, pbc):
    cell = (4e-9, 3e-9, 2e-9)
    m = inputs.random_unit(shape, 33)
    s = solver(shape, cell, pbc=pbc, images=2, **MAT)
    h, tq, _ = s.heff(to_dev(m), torque=True)
    p = oracle(shape, cell, pbc=pbc, images=2, **MAT)
    m64 = m.astype(np.float64)
    H = p.heff(m64)
    Hg = to_np(h)
    print(shape, pbc, "rel L2", rel_l2(Hg, H), "rel max", rel_max(Hg, H))
    assert rel_l2(Hg, H) <= HEFF_REL_L2
    assert rel_max(Hg, H) <= HEFF_REL_MAX
    assert rel_l2(to_np(tq), llg.ll_rhs(m64, H, p.alpha)) <= 2 * HEFF_REL_L2


@pytest.mark.parametrize("shape,pbc,method", [((600, 7, 1), (0, 0, 0), B.MM_RKDP), ((96, 12, 3), (0, 0, 0), B.MM_RKDP),
                                              ((192, 8, 1), (1, 0, 0), B.MM_HEUN), ((5, 600, 1), (0, 0, 0), B.MM_RKDP),
                                              ((96, 130, 40), (0, 0, 0), B.MM_RKDP)])
def test_step_at_odd_x_lengths(shape, pbc, method):
    cell = (4e-9, 3e-9, 2e-9)
    m = inputs.random_unit(shape, 32)
    s = solver(shape, cell, pbc=pbc, images=2, **MAT)
    p = oracle(shape, cell, pbc=pbc, images=2, **MAT)
    md = to_dev(m)
    h = 1e-13
    acc, _, _ = B.mm_step(s.ctx, md, method, 0.0, h, tol=1.0)
    ref = llg.rkdp_stages(p, _unit64(m), h)[0] if method == B.MM_RKDP else llg.heun_step(p, _unit64(m), h)
    err = float(np.max(np.abs(to_np(md) - ref)))
    print(shape, "one step max|dm|", err)
    assert acc and err <= 1e-6


def test_several_fused_steps_at_an_odd_x_length():
    """Ten Dormand-Prince steps through the step graph (fused x passes) on the
    600 x 7 film (x padded to 1280) from a smooth state."""
    shape, cell = (600, 7, 1), (4e-9, 3e-9, 2e-9)
    m = inputs.smooth_tilt(shape)
    s = solver(shape, cell, **MAT)
    p = oracle(shape, cell, **MAT)
    md = to_dev(m)
    B.mm_load(s.ctx, md)
    B.mm_advance(s.ctx, B.MM_RKDP, 10, dt_s=5e-14, tol=-1.0)
    B.mm_store(s.ctx, md)
    st = B.mm_get_stats(s.ctx)
    assert st["accepted"] == 10 and st["status"] == 0
    ref = llg.rkdp_fixed(p, _unit64(m), 5e-14, 10)
    err = float(np.max(np.abs(to_np(md) - ref)))
    print("10 fixed RKDP steps at x length 1280: max|dm|", err)
    assert err <= 1e-5


def test_batches_refuse_odd_x_lengths():
    import torch
    s = solver((600, 7, 1), (4e-9, 3e-9, 2e-9), **MAT)
    with pytest.raises(B.MMError):
        B.Batch([s], torch.cuda.current_stream().cuda_stream)
