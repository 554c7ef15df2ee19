"""The split-BF16 tensor-core z pass (mm_set_dft_precision) against the FP64
oracle.  The z transforms run as dense DFT products with bf16 operands split
into hi + lo parts (three products, fp32 accumulation).  Measured on the
GB300: relative L2 error of H_eff 1.1e-7 on the 32^3 crop of the
256 x 256 x 64 cube (periodic x and y, per-cell axes, 64-point z transforms),
against 6.2e-8 for the FP32 pass: it meets the FP32 path's bounds (relative L2
<= 1e-6, element-wise <= 5e-6 of max |H|), which are the bounds asserted here.
The variant's field must differ from the FP32 pass's (so that it is the one
that ran)."""

import numpy as np
import pytest

from oracle import llg
from paper_1102_3069_gb300 import binding as B
from paper_1102_3069_gb300 import inputs

from gpu_util import HEFF_REL_L2, HEFF_REL_MAX, oracle, rel_l2, rel_max, solver, to_dev, to_np

pytestmark = pytest.mark.gpu

W = inputs.workload("cube_256x256x64")


def _case(shape, cell, pbc, images, mat, axes=None):
    s16 = solver(shape, cell, pbc=pbc, images=images, dft_precision=B.MM_DFT_SPLIT_BF16, **mat)
    s32 = solver(shape, cell, pbc=pbc, images=images, **mat)
    if axes is not None:
        for s in (s16, s32):
            s.axes = to_dev(axes)
            B.mm_set_anisotropy_axes(s.ctx, s.axes)
        mat = dict(mat, easy_axis=axes.astype(np.float64))
    p = oracle(shape, cell, pbc=pbc, images=images, **mat)
    return s16, s32, p


@pytest.mark.parametrize("name", ["crop32", "open_block"])
def test_split_bf16_z_pass_error(name):
    if name == "crop32":
        shape, cell, pbc, images = (32, 32, 32), W["cell"], W["pbc"], 2
        mat = dict(W["material"], temperature=0.0)
        axes = inputs.tilted_axes(shape, 0)
    else:
        shape, cell, pbc, images = (20, 14, 9), (4e-9, 3e-9, 2e-9), (0, 0, 0), 0
        mat = dict(Ms=8e5, Aex=1.3e-11, Ku=5e3, easy_axis=(1.0, 2.0, 3.0), alpha=0.1, B=(0.01, -0.02, 0.03))
        axes = None
    s16, s32, p = _case(shape, cell, pbc, images, mat, axes)
    m = inputs.random_unit(shape, 23)
    H = p.heff(m.astype(np.float64))
    h16 = to_np(s16.heff(to_dev(m))[0])
    h32 = to_np(s32.heff(to_dev(m))[0])
    e16, e32 = rel_l2(h16, H), rel_l2(h32, H)
    print(name, "split-BF16 z pass: rel L2", e16, "rel max", rel_max(h16, H), "| FP32 pass: rel L2", e32)
    assert e16 <= HEFF_REL_L2
    assert rel_max(h16, H) <= HEFF_REL_MAX
    assert rel_l2(h16, h32) > 1e-9


def test_split_bf16_heun_steps_on_crop():
    shape = (32, 32, 32)
    mat = W["material"]
    axes = inputs.tilted_axes(shape, 0)
    s16, _, p = _case(shape, W["cell"], W["pbc"], 2, mat, axes)
    m = inputs.random_unit(shape, 24)
    md = to_dev(m)
    B.mm_load(s16.ctx, md, 0.0, 0)
    B.mm_advance(s16.ctx, B.MM_HEUN, 5, dt_s=W["dt"])
    B.mm_store(s16.ctx, md)
    st = B.mm_get_stats(s16.ctx)
    assert st["accepted"] == 5 and st["status"] == 0
    ref = m.astype(np.float64)
    ref /= np.sqrt((ref * ref).sum(axis=0, keepdims=True))
    for k in range(5):
        ref = llg.heun_step(p, ref, W["dt"], step=k)
    err = float(np.max(np.abs(to_np(md) - ref)))
    print("5 thermal Heun steps with the split-BF16 z pass: max|dm|", err)
    assert err <= 1e-4


def test_split_bf16_needs_a_3d_grid_and_comes_before_the_workspace():
    ctx = B.mm_init_geometry(16, 16, 1, 4e-9, 4e-9, 4e-9)
    try:
        with pytest.raises(B.MMError):
            B.mm_set_dft_precision(ctx, B.MM_DFT_SPLIT_BF16)
    finally:
        B.mm_destroy(ctx)
    s = solver((8, 8, 4), (4e-9, 4e-9, 4e-9), Ms=8e5, Aex=1.3e-11)
    with pytest.raises(B.MMError) as e:
        B.mm_set_dft_precision(s.ctx, B.MM_DFT_SPLIT_BF16)
    assert e.value.code == B.MM_ESTATE
