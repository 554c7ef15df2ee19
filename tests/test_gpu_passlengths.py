"""Pass lengths that no other parity test reaches, checked against the oracle.

* The 4096-point 3-D passes: an open axis of 1500 cells pads to 4096, so
  (4, 1500, 2) runs the 4096-point y forward and inverse passes of a 3-D grid
  and (3, 2, 1500) runs the 4096-point z column pass (Sec. 3.2: one pass of
  1-D transforms per axis).
* The passes of the 256 x 256 x 64 cube workload: periodic x and y of 256
  cells (x and y transforms of 256 points, Sec. 2.1.1 periodic boundaries,
  no padding) and an open z axis of 33 cells, which pads to the same
  128-point z column pass as the cube's 64 cells.  Per-cell easy axes tilted
  up to 30 degrees from z and the 300 K thermal field, as in the cube.  The
  oracle's periodic kernel is built without extra images (offsets wrapped once)
  to keep its build near a minute; the image sums have their own tests.

Bounds as everywhere: relative L2 error of H_eff <= 1e-6 and element-wise
<= 5e-6 of max |H|; one step: max |dm| <= 1e-6 (Dormand-Prince, no noise) or
<= 1e-5 (two thermal Heun steps).
"""

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


@pytest.mark.parametrize("shape", [(4, 1500, 2), (3, 2, 1500)])
def test_4096_point_3d_passes(shape):
    cell = (4e-9, 3e-9, 2e-9)
    m = inputs.random_unit(shape, 21)
    s = solver(shape, cell, **MAT)                 # the 1500-cell axis pads to 4096
    h, tq, e = s.heff(to_dev(m), torque=True, energy=True)
    p = oracle(shape, cell, **MAT)
    m64 = m.astype(np.float64)
    t = p.terms(m64)
    H = t["d"] + t["ex"] + t["an"] + t["z"]
    Hg = to_np(h)
    print(shape, "rel L2", rel_l2(Hg, H), "rel max", rel_max(Hg, H))
    assert rel_l2(Hg, H) <= HEFF_REL_L2
    assert rel_max(Hg, H) <= HEFF_REL_MAX
    assert rel_l2(to_np(tq), llg.ll_rhs(m64, H, p.alpha)) <= 2 * HEFF_REL_L2
    E = p.energy(m64)
    assert abs(e - E) <= 2e-6 * abs(E), (e, E)
    # one Dormand-Prince step through the time-step passes
    md = to_dev(m)
    acc, _, _ = B.mm_step(s.ctx, md, B.MM_RKDP, 0.0, 1e-13, tol=1.0)
    ref = llg.rkdp_stages(p, _unit64(m), 1e-13)[0]
    err = float(np.max(np.abs(to_np(md) - ref)))
    print(shape, "one RKDP step max|dm|", err)
    assert acc and err <= 1e-6


CUBE = inputs.workload("cube_256x256x64")
CUBE_SHAPE = (256, 256, 33)


@pytest.fixture(scope="module")
def cube_pair():
    mat = CUBE["material"]
    axes = inputs.tilted_axes(CUBE_SHAPE, 1)
    s = solver(CUBE_SHAPE, CUBE["cell"], pbc=CUBE["pbc"], images=0, **mat)   # FFT 256 x 256 x 128
    s.axes = to_dev(axes)
    B.mm_set_anisotropy_axes(s.ctx, s.axes)
    p = oracle(CUBE_SHAPE, CUBE["cell"], pbc=CUBE["pbc"], images=0, **dict(mat, easy_axis=axes.astype(np.float64)))
    return s, p


def test_cube_pass_lengths_heff_with_thermal_field(cube_pair):
    s, p = cube_pair
    m = inputs.random_unit(CUBE_SHAPE, 17)
    B.mm_set_thermal_clock(s.ctx, 9, CUBE["dt"])
    h, _, _ = s.heff(to_dev(m))
    t = p.terms(m.astype(np.float64), step=9, dt=CUBE["dt"])
    H = t["d"] + t["ex"] + t["an"] + t["z"] + t["th"]
    Hg = to_np(h)
    print("256x256x33: rel L2", rel_l2(Hg, H), "rel max", rel_max(Hg, H))
    assert rel_l2(Hg, H) <= HEFF_REL_L2
    assert rel_max(Hg, H) <= HEFF_REL_MAX
    # the noise alone (the largest term) against the oracle's Philox draws
    Hth = Hg - (t["d"] + t["ex"] + t["an"] + t["z"])
    assert rel_max(Hth, t["th"]) <= 2e-5
    B.mm_set_thermal_clock(s.ctx, 9, 0.0)
    h0, _, _ = s.heff(to_dev(m))
    assert rel_l2(to_np(h0), H - t["th"]) <= HEFF_REL_L2


def test_cube_pass_lengths_thermal_heun_steps(cube_pair):
    s, p = cube_pair
    m = inputs.random_unit(CUBE_SHAPE, 18)
    md = to_dev(m)
    B.mm_load(s.ctx, md, 0.0, 3)
    B.mm_advance(s.ctx, B.MM_HEUN, 2, dt_s=CUBE["dt"])
    B.mm_store(s.ctx, md)
    st = B.mm_get_stats(s.ctx)
    assert st["accepted"] == 2 and st["step_index"] == 5 and st["status"] == 0
    ref = _unit64(m)
    for k in (3, 4):
        ref = llg.heun_step(p, ref, CUBE["dt"], step=k)
    err = float(np.max(np.abs(to_np(md) - ref)))
    print("256x256x33, 2 thermal Heun steps: max|dm|", err)
    assert err <= 1e-5
