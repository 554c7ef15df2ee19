"""The fused y-z pass of 3-D grids with few z cells (nz <= 8): H_eff, torque
and energy against the FP64 oracle element by element (every nz from 2 to 8,
open and periodic z, ragged y, the largest y length), time steps, batches,
and that the fused pass is what ran."""

import numpy as np
import pytest

from oracle import llg
from paper_1102_3069_gb300 import binding as B
from paper_1102_3069_gb300 import inputs

from gpu_util import HEFF_REL_L2, HEFF_REL_MAX, oracle, rel_l2, rel_max, solver, to_dev, to_np

pytestmark = pytest.mark.gpu

MAT = dict(Ms=8e5, Aex=1.3e-11, Ku=5e3, easy_axis=(1.0, 2.0, 3.0), alpha=0.1, B=(0.01, -0.02, 0.03))
CELL = (4e-9, 3e-9, 2e-9)

SHAPES = [((6, 5, 2), (0, 0, 0)), ((9, 7, 3), (0, 0, 0)), ((16, 12, 4), (0, 0, 0)), ((12, 20, 5), (0, 0, 0)),
          ((7, 33, 6), (0, 0, 0)), ((10, 9, 7), (0, 0, 0)), ((8, 16, 8), (0, 0, 0)), ((16, 8, 4), (0, 0, 1)),
          ((16, 16, 8), (1, 1, 1)), ((8, 4, 2), (0, 0, 1)), ((20, 250, 3), (0, 0, 0)), ((6, 500, 2), (0, 0, 0))]


@pytest.mark.parametrize("shape,pbc", SHAPES)
def test_fused_yz_heff_matches_oracle(shape, pbc):
    m = inputs.random_unit(shape, 21)
    s = solver(shape, CELL, pbc=pbc, images=2, **MAT)
    h, tq, e = s.heff(to_dev(m), torque=True, energy=True)
    p = oracle(shape, CELL, pbc=pbc, images=2, **MAT)
    m64 = m.astype(np.float64)
    t = p.terms(m64)
    H = t["d"] + t["ex"] + t["an"] + t["z"]
    Hg = to_np(h)
    assert rel_l2(Hg, H) <= HEFF_REL_L2, rel_l2(Hg, H)
    assert rel_max(Hg, H) <= HEFF_REL_MAX, rel_max(Hg, H)
    assert rel_l2(to_np(tq), llg.ll_rhs(m64, H, p.alpha)) <= 2 * HEFF_REL_L2
    E = p.energy(m64)
    assert abs(e - E) <= 2e-6 * abs(E), (e, E)
    t1 = B.pass_times(s.ctx, lambda: s.heff(to_dev(m)))
    assert "k_yzconv" in t1 and not {"k_yfwd", "k_colconv_z", "k_yinv"} & set(t1)


def test_general_3d_passes_beyond_eight_z_cells():
    shape = (8, 6, 9)
    s = solver(shape, CELL, images=2, **MAT)
    m = inputs.random_unit(shape, 3)
    t1 = B.pass_times(s.ctx, lambda: s.heff(to_dev(m)))
    assert "k_yzconv" not in t1 and {"k_yfwd", "k_colconv_z", "k_yinv"} <= set(t1)


def _m64(m):
    m = m.astype(np.float64)
    return m / np.sqrt((m * m).sum(axis=0, keepdims=True))


@pytest.mark.parametrize("method,dt", [(B.MM_EULER, 1e-14), (B.MM_HEUN, 5e-14), (B.MM_RKDP, 1e-13)])
def test_fused_yz_step_matches_oracle(method, dt):
    shape = (24, 20, 4)
    mat = dict(MAT, alpha=0.02)
    m = inputs.random_unit(shape, 5)
    s = solver(shape, CELL, images=2, **mat)
    p = oracle(shape, CELL, images=2, **mat)
    md = to_dev(m)
    acc, t, _ = B.mm_step(s.ctx, md, method, 0.0, dt, tol=1.0)
    assert acc
    m0 = _m64(m)
    if method == B.MM_EULER:
        ref = llg.euler_step(p, m0, dt)
    elif method == B.MM_HEUN:
        ref = llg.heun_step(p, m0, dt)
    else:
        ref = llg.rkdp_stages(p, m0, dt)[0]
    assert np.max(np.abs(to_np(md) - ref)) <= 1e-6


def test_fused_yz_in_a_batch_matches_single_contexts():
    """Thin 3-D samples of several y lengths and z counts in one batch (the
    batched fused pass groups them by y length and z cells per block): one
    fixed Dormand-Prince step each, against the single-context step."""
    import torch
    shapes = [(40, 30, 2), (33, 64, 3), (64, 100, 4), (48, 20, 6), (20, 40, 8), (50, 50, 1)]
    mat = dict(MAT, alpha=0.05)
    sol, ms, ref = [], [], []
    for i, sh in enumerate(shapes):
        m = inputs.random_unit(sh, 30 + i)
        s = B.Solver(sh, CELL, images=2, tensor=False, fft_lengths=B.MM_FFT_POW2, **mat)
        sol.append(s)
        ms.append(to_dev(m))
        one = B.Solver(sh, CELL, images=2, tensor=False, fft_lengths=B.MM_FFT_POW2, **mat)
        md = to_dev(m)
        B.mm_load(one.ctx, md)
        B.mm_advance(one.ctx, B.MM_RKDP, 1, dt_s=1e-13, tol=-1.0)
        B.mm_store(one.ctx, md)
        ref.append(md)
    bt = B.Batch(sol, torch.cuda.current_stream().cuda_stream)
    B.mm_batch_load(bt.b, ms)
    B.mm_batch_advance(bt.b, B.MM_RKDP, 1, dt_s=1e-13, tol=-1.0)
    B.mm_batch_store(bt.b, ms)
    torch.cuda.synchronize()
    for sh, a, b in zip(shapes, ms, ref):
        assert float((a - b).abs().max()) < 2e-6, sh
