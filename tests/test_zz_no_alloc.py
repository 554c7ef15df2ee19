"""mm_eval_heff_static: the allocation-free field evaluation.

It serves callers that may not allocate device memory where they evaluate the
field (a host application that owns the whole device-memory budget, or a
loop that forbids cudaMalloc after start-up).  Its scratch is one static
device array inside libmm.so.  Here it is called through the C ABI twice in
a row, each time on a different magnetisation.  It launches the same kernels
as the workspace-based mm_eval_heff with only the scratch addresses changed,
so each output must equal that call's bit for bit; one shape is also compared
with the FP64 oracle directly, at the parity bound the other tests use.
Grids too large for the static array must be refused with MM_ENOMEM.

This file is named so that pytest collects it last.
"""

import numpy as np
import pytest

from paper_1102_3069_gb300 import binding as B
from paper_1102_3069_gb300 import inputs

from gpu_util import HEFF_REL_L2, HEFF_REL_MAX, oracle, rel_l2, rel_max, solver, to_dev, to_np

pytestmark = pytest.mark.gpu

MAT = dict(Ms=8e5, Aex=1.3e-11, Ku=5e3, easy_axis=(1.0, 2.0, 3.0), alpha=0.1, B=(0.01, -0.02, 0.03))


@pytest.mark.parametrize("shape,cell,pbc", [((64, 16, 1), (4e-9, 4e-9, 4e-9), (0, 0, 0)),
                                            ((33, 20, 3), (4e-9, 3e-9, 2e-9), (0, 0, 0)),
                                            ((32, 16, 4), (3e-9, 3e-9, 3e-9), (1, 1, 0))])
def test_static_matches_workspace_evaluation_twice(shape, cell, pbc):
    import torch
    s = solver(shape, cell, pbc=pbc, images=3, **MAT)
    for seed in (1, 2):                      # two calls in a row, different inputs
        m = to_dev(inputs.random_unit(shape, seed))
        h_ref, tq_ref = torch.empty_like(m), torch.empty_like(m)
        B.mm_eval_heff(s.ctx, m, h_ref, tq_ref)
        h, tq = torch.full_like(m, float("nan")), torch.full_like(m, float("nan"))
        B.mm_eval_heff_static(s.ctx, m, h, tq)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(h.cpu().numpy(), h_ref.cpu().numpy())
        np.testing.assert_array_equal(tq.cpu().numpy(), tq_ref.cpu().numpy())


def test_static_matches_oracle():
    import torch
    from oracle import llg
    shape, cell = (40, 24, 3), (4e-9, 3e-9, 2e-9)
    s = solver(shape, cell, **MAT)
    p = oracle(shape, cell, **MAT)
    for seed in (5, 6):
        m = inputs.random_unit(shape, seed)
        md = to_dev(m)
        h, tq = torch.full_like(md, float("nan")), torch.full_like(md, float("nan"))
        B.mm_eval_heff_static(s.ctx, md, h, tq)
        torch.cuda.synchronize()
        m64 = m.astype(np.float64)
        H = p.heff(m64)
        assert rel_l2(to_np(h), H) <= HEFF_REL_L2
        assert rel_max(to_np(h), H) <= HEFF_REL_MAX
        assert rel_l2(to_np(tq), llg.ll_rhs(m64, H, p.alpha)) <= 2 * HEFF_REL_L2


def test_static_without_workspace_when_demag_is_off():
    import torch
    shape, cell = (48, 20, 2), (4e-9, 4e-9, 2e-9)
    ctx = B.mm_init_geometry(*shape, *cell)          # no workspace ever handed over
    try:
        B.mm_set_material(ctx, **MAT)
        B.mm_set_demag(ctx, False)
        ref = solver(shape, cell, demag=False, **MAT)
        for seed in (3, 4):
            m = to_dev(inputs.random_unit(shape, seed))
            h_ref, _, _ = ref.heff(m)
            h = torch.full_like(m, float("nan"))
            B.mm_eval_heff_static(ctx, m, h)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(h.cpu().numpy(), h_ref.cpu().numpy())
    finally:
        B.mm_destroy(ctx)


def test_static_refuses_grids_beyond_its_scratch():
    import torch
    shape, cell = (1024, 1024, 1), (4e-9, 4e-9, 2e-9)
    s = solver(shape, cell, **MAT)
    m = to_dev(inputs.random_unit(shape, 0))
    h = torch.empty_like(m)
    with pytest.raises(B.MMError) as e:
        B.mm_eval_heff_static(s.ctx, m, h)
    assert e.value.code == B.MM_ENOMEM
    assert "MM_STATIC_SCRATCH_BYTES" in B.mm_last_error(s.ctx)
