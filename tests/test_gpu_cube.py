"""3-D periodic workload with thermal noise, checked on a 32^3 crop.

The 256 x 256 x 64 cube (3 nm cells, periodic in x and y, Ms 1.1e6 A/m,
A 2e-11 J/m, Ku 2e4 J/m^3 along per-cell easy axes tilted up to 30 deg from
z, alpha 0.05, 300 K, Heun with
dt = 50 fs) runs the 3-D pass sequence (x, y forward, z column pass, y
inverse, x inverse + epilogue) and the periodic-image kernel.  The FP64
oracle cannot build the full periodic kernel in reasonable time, so the same
material, boundary conditions and step are checked on a standalone
32 x 32 x 32 crop with 2 images per periodic side:
* H_eff including the thermal field: relative L2 error <= 1e-6;
* 20 thermal Heun steps: max |dm| <= 1e-5.
"""

import numpy as np
import pytest

from oracle import llg
from paper_1102_3069_gb300 import binding as B
from paper_1102_3069_gb300 import inputs

from gpu_util import HEFF_REL_L2, HEFF_REL_MAX, oracle, rel_l2, rel_max, solver, to_dev, to_np

pytestmark = pytest.mark.gpu

W = inputs.workload("cube_256x256x64")
SHAPE = (32, 32, 32)
IMAGES = 2


@pytest.fixture(scope="module")
def pair():
    # the cube's per-cell easy axes (tilted up to 30 deg from z), drawn for the crop
    mat = W["material"]
    axes = inputs.tilted_axes(SHAPE, 0)
    s = solver(SHAPE, W["cell"], pbc=W["pbc"], images=IMAGES, **mat)
    s.axes = to_dev(axes)
    B.mm_set_anisotropy_axes(s.ctx, s.axes)
    p = oracle(SHAPE, W["cell"], pbc=W["pbc"], images=IMAGES, **dict(mat, easy_axis=axes.astype(np.float64)))
    return s, p


def test_cube_crop_heff_with_thermal_field(pair):
    s, p = pair
    m = inputs.random_unit(SHAPE, 7)
    B.mm_set_thermal_clock(s.ctx, 5, W["dt"])
    h, _, _ = s.heff(to_dev(m))
    t = p.terms(m.astype(np.float64), step=5, dt=W["dt"])
    H = t["d"] + t["ex"] + t["an"] + t["z"] + t["th"]
    Hg = to_np(h)
    print("32^3 crop: rel L2", rel_l2(Hg, H), "rel max", rel_max(Hg, H))
    assert rel_l2(Hg, H) <= HEFF_REL_L2
    assert rel_max(Hg, H) <= HEFF_REL_MAX
    # without the noise the deterministic part alone must match as well
    Hd = H - t["th"]
    B.mm_set_thermal_clock(s.ctx, 5, 0.0)
    h0, _, _ = s.heff(to_dev(m))
    assert rel_l2(to_np(h0), Hd) <= HEFF_REL_L2


def test_cube_crop_thermal_heun_steps(pair):
    s, p = pair
    m = inputs.random_unit(SHAPE, 8)
    md = to_dev(m)
    B.mm_load(s.ctx, md, 0.0, 0)
    B.mm_advance(s.ctx, B.MM_HEUN, 20, dt_s=W["dt"])
    B.mm_store(s.ctx, md)
    st = B.mm_get_stats(s.ctx)
    assert st["accepted"] == 20 and st["step_index"] == 20 and st["status"] == 0
    ref = m.astype(np.float64)
    ref /= np.sqrt((ref * ref).sum(axis=0, keepdims=True))
    for k in range(20):
        ref = llg.heun_step(p, ref, W["dt"], step=k)
    err = float(np.max(np.abs(to_np(md) - ref)))
    print("32^3 crop, 20 thermal Heun steps: max|dm|", err)
    assert err <= 1e-5
