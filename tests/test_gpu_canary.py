"""Out-of-bounds writes (compute-sanitizer is not available on the GPU pool):
every device buffer the library writes - its workspace and the caller's
arrays - is surrounded by canary bytes, and the canaries must be intact after
field evaluations and time steps of several integrators (adaptive, fixed and
maximum-variation), on grids that take the fused and the split x passes, in
2-D and 3-D."""

import numpy as np
import pytest

from paper_1102_3069_gb300 import binding as B
from paper_1102_3069_gb300 import inputs

pytestmark = pytest.mark.gpu

GUARD = 1 << 16          # canary bytes before and after each buffer
PATTERN = 0xA5


def _guarded(nbytes):
    import torch
    buf = torch.full((nbytes + 2 * GUARD + 256,), PATTERN, dtype=torch.uint8, device="cuda")
    base = buf.data_ptr()
    start = (base + GUARD + 255) // 256 * 256
    return buf, start - base


def _intact(buf, off, nbytes):
    import torch
    head = buf[:off]
    tail = buf[off + nbytes:]
    return bool(torch.all(head == PATTERN)) and bool(torch.all(tail == PATTERN))


@pytest.mark.parametrize("shape", [(13, 7, 1), (100, 37, 1), (20, 70, 3), (9, 5, 4)])
def test_no_writes_outside_the_buffers(shape):
    import torch
    cell = (4e-9, 3e-9, 2e-9)
    mat = dict(Ms=8e5, Aex=1.3e-11, Ku=5e3, easy_axis=(1.0, 2.0, 3.0), alpha=0.3, B=(0.01, -0.02, 0.03))
    ctx = B.mm_init_geometry(*shape, *cell)
    try:
        nws = B.mm_workspace_bytes(ctx)
        wsbuf, wsoff = _guarded(nws)
        B.mm_set_workspace(ctx, wsbuf.data_ptr() + wsoff, nws)
        B.mm_set_material(ctx, **mat)
        B.mm_demag_kernel(ctx)
        n3 = 3 * int(np.prod(shape)) * 4
        mbuf, moff = _guarded(n3)
        hbuf, hoff = _guarded(n3)
        tbuf, toff = _guarded(n3)
        m = torch.from_numpy(inputs.random_unit(shape, 2)).cuda()
        mview = mbuf[moff:moff + n3].view(torch.float32)
        mview.copy_(m.reshape(-1))
        hp, tp = hbuf.data_ptr() + hoff, tbuf.data_ptr() + toff
        B.mm_eval_heff(ctx, mview.data_ptr(), hp, tp, energy=True)
        B.mm_load(ctx, mview.data_ptr())
        B.mm_advance(ctx, B.MM_RKDP, 5, dt_s=1e-13, tol=1e-5)
        B.mm_advance(ctx, B.MM_RK4, 3, dt_s=2e-14)
        B.mm_advance(ctx, B.MM_HEUN, 3, dt_s=2e-14)
        B.mm_set_max_dm(ctx, 0.01)
        B.mm_advance(ctx, B.MM_EULER, 3)
        B.mm_set_max_dm(ctx, 0.0)
        B.mm_store(ctx, mview.data_ptr())
        torch.cuda.synchronize()
        assert _intact(wsbuf, wsoff, nws)
        assert _intact(mbuf, moff, n3)
        assert _intact(hbuf, hoff, n3)
        assert _intact(tbuf, toff, n3)
        assert bool(torch.isfinite(mview).all())
    finally:
        B.mm_destroy(ctx)
