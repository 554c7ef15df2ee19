"""Batched ensembles (mm_batch_*).

A batched launch runs the block bodies of the single-context kernels on the
same block decomposition, reading each sample's parameters from device memory
instead of the launch's own parameter block.  So:

* one batched Dormand-Prince step of every sample matches the FP64 oracle
  (the same bound as the single-context step parity);
* fixed-step trajectories agree with stepping each sample alone up to float32
  rounding;
* a batched relaxation leaves every sample below the torque bound, which a
  fresh single-context evaluation of the stored state confirms, with lower
  energy than the start.
"""

import numpy as np
import pytest

from oracle import llg
from paper_1102_3069_gb300 import binding as B
from paper_1102_3069_gb300 import inputs

pytestmark = pytest.mark.gpu


def _solvers(samples, stream):
    return [B.Solver(s["shape"], s["cell"], pbc=s["pbc"], stream=stream, tensor=False, fft_lengths=B.MM_FFT_POW2,
                     **s["material"])
            for s in samples]


def _m0(samples):
    import torch
    return [torch.from_numpy(inputs.random_unit(s["shape"], s["m_seed"])).cuda() for s in samples]


def test_batch_step_matches_oracle():
    import torch
    samples = inputs.ensemble(4, seed=11, nmin=32, nmax=40, nzmax=3)
    stream = torch.cuda.Stream()
    h = 1e-13
    with torch.cuda.stream(stream):
        sol = _solvers(samples, stream.cuda_stream)
        m0 = _m0(samples)
        bt = B.Batch(sol, stream.cuda_stream)
        B.mm_batch_load(bt.b, m0)
        B.mm_batch_advance(bt.b, B.MM_RKDP, 1, dt_s=h, tol=-1.0)       # one step of fixed size h
        out = [torch.empty_like(m) for m in m0]
        B.mm_batch_store(bt.b, out)
        st = B.mm_batch_get_stats(bt.b, len(sol))
        torch.cuda.synchronize()
    for i, s in enumerate(samples):
        mat = s["material"]
        p = llg.Problem(s["shape"], s["cell"], mat["Ms"], mat["Aex"], mat["alpha"], Ku=mat["Ku"],
                        u=mat["easy_axis"], B=mat["B"])
        m = m0[i].cpu().numpy().astype(np.float64)
        m /= np.sqrt((m * m).sum(axis=0, keepdims=True))
        ref = llg.rkdp_stages(p, m, h)[0]
        d = float(np.max(np.abs(out[i].cpu().numpy() - ref)))
        assert d < 1e-6, (i, s["shape"], d)
        assert st[i]["accepted"] == 1 and st[i]["evals"] == 7 and st[i]["status"] == 0
        assert abs(st[i]["t"] - h) < 1e-25


@pytest.mark.parametrize("method,calls", [
    (B.MM_RKDP, [(1, 5e-14, -1.0), (15, 5e-14, -1.0)]),  # fixed h, first same as last
    (B.MM_RK4, [(12, 5e-14, -1.0)]),                     # k1 evaluated every step
])
def test_batch_fixed_steps_match_single(method, calls):
    import torch
    # 3-D samples (z column pass) and 2-D films (y column pass) in one batch
    samples = inputs.ensemble(6, seed=3, nmin=32, nmax=80, nzmax=4) + inputs.ensemble(3, seed=4, nmin=32, nmax=90,
                                                                                       nzmax=1)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sol = _solvers(samples, stream.cuda_stream)
        m0 = _m0(samples)
        bt = B.Batch(sol, stream.cuda_stream)
        B.mm_batch_load(bt.b, m0)
        for n, dt, tol in calls:
            B.mm_batch_advance(bt.b, method, n, dt_s=dt, tol=tol)
        out = [torch.empty_like(m) for m in m0]
        B.mm_batch_store(bt.b, out)
        stb = B.mm_batch_get_stats(bt.b, len(sol))
        torch.cuda.synchronize()
        for i, s in enumerate(samples):
            one = B.Solver(s["shape"], s["cell"], pbc=s["pbc"], stream=stream.cuda_stream, tensor=False,
                           fft_lengths=B.MM_FFT_POW2, **s["material"])
            m = m0[i].clone()
            B.mm_load(one.ctx, m)
            for n, dt, tol in calls:
                B.mm_advance(one.ctx, method, n, dt_s=dt, tol=tol)
            B.mm_store(one.ctx, m)
            st = B.mm_get_stats(one.ctx)
            torch.cuda.synchronize()
            assert stb[i]["status"] == 0 and st["status"] == 0
            d = float((m - out[i]).abs().max())
            assert d < 1e-5, (i, s["shape"], d)
            for k in ("evals", "accepted", "rejected"):
                assert st[k] == stb[i][k], (i, k, st[k], stb[i][k])
            assert abs(st["t"] - stb[i]["t"]) <= 1e-9 * st["t"]
            one.close()


def test_batch_relax_reaches_torque_bound():
    import torch
    samples = inputs.ensemble(5, seed=5, nmin=32, nmax=48, nzmax=3, alpha=0.5)
    stream = torch.cuda.Stream()
    tq_tol, err_tol, max_steps = 1e-3, 1e-5, 60000
    with torch.cuda.stream(stream):
        sol = _solvers(samples, stream.cuda_stream)
        mb = _m0(samples)
        m_start = [m.clone() for m in mb]
        bt = B.Batch(sol, stream.cuda_stream)
        rc, steps, tq, conv = B.mm_batch_relax(bt.b, mb, tq_tol, err_tol, max_steps)
        torch.cuda.synchronize()
        assert rc == B.MM_OK and conv == len(samples), (rc, conv, tq)
        assert max(tq) < tq_tol and min(steps) > 0
        for i, s in enumerate(samples):
            one = B.Solver(s["shape"], s["cell"], pbc=s["pbc"], stream=stream.cuda_stream, tensor=False,
                           fft_lengths=B.MM_FFT_POW2, **s["material"])
            h, _, e1 = one.heff(mb[i], energy=True)
            _, _, e0 = one.heff(m_start[i], energy=True)
            torch.cuda.synchronize()
            mxh = torch.cross(mb[i].double(), h.double(), dim=0)
            tq_fresh = float(mxh.norm(dim=0).max()) / s["material"]["Ms"]
            assert tq_fresh < tq_tol * 1.01, (i, tq_fresh, tq[i])
            assert abs(tq_fresh - tq[i]) <= 1e-3 * tq_tol + 1e-4 * tq[i]
            assert e1 < e0
            one.close()


def test_batch_rejects_unsupported_contexts():
    import torch
    stream = torch.cuda.Stream()
    s = B.Solver((16, 40, 1), (4e-9, 4e-9, 4e-9), stream=stream.cuda_stream, tensor=False, Ms=8e5, Aex=1.3e-11)
    with pytest.raises(B.MMError) as e:
        B.mm_batch_create([s.ctx], stream.cuda_stream)          # padded x length 32 < 64
    assert e.value.code == B.MM_EINVAL
    t = B.Solver((40, 40, 1), (4e-9, 4e-9, 4e-9), stream=stream.cuda_stream, tensor=False, Ms=8e5, Aex=1.3e-11,
                 temperature=300.0, fft_lengths=B.MM_FFT_POW2)
    bt = B.Batch([t], stream.cuda_stream)
    B.mm_batch_load(bt.b, [torch.from_numpy(inputs.random_unit((40, 40, 1), 0)).cuda()])
    with pytest.raises(B.MMError) as e:
        B.mm_batch_advance(bt.b, B.MM_RK4, 1, dt_s=1e-14, tol=-1.0)   # thermal field refused in a batch
    assert e.value.code == B.MM_EINVAL


def test_batch_autotuner_register_budgets_agree():
    """The two compiled register budgets of each batched FFT pass run the same
    block body: forcing the second everywhere changes no result beyond float32
    rounding, and the autotuner reports which groups it could tune."""
    import torch
    samples = inputs.ensemble(6, seed=8, nmin=32, nmax=70, nzmax=3)   # FFT lengths 64..256
    stream = torch.cuda.Stream()
    outs, reports = {}, {}
    with torch.cuda.stream(stream):
        for mode in (0, 2, 1):
            sol = _solvers(samples, stream.cuda_stream)
            m0 = _m0(samples)
            bt = B.Batch(sol, stream.cuda_stream)
            B.mm_batch_set_tuning(bt.b, mode)
            B.mm_batch_load(bt.b, m0)
            B.mm_batch_advance(bt.b, B.MM_RKDP, 6, dt_s=5e-14, tol=-1.0)
            out = [torch.empty_like(m) for m in m0]
            B.mm_batch_store(bt.b, out)
            torch.cuda.synchronize()
            outs[mode] = out
            reports[mode] = B.mm_batch_tuning(bt.b)
    groups, tunable, alt = reports[2]
    assert tunable > 0 and alt == tunable and groups >= tunable
    assert reports[0][2] == 0 and reports[1][1] == tunable
    for mode in (1, 2):
        for a, b in zip(outs[0], outs[mode]):
            assert float((a - b).abs().max()) <= 1e-6


def test_batch_periodic_samples_match_oracle():
    """Samples with periodic axes (image sums in the kernel, no padding along
    them) in one batch with an open one: one fixed Dormand-Prince step each
    against the FP64 oracle."""
    import torch
    mat = dict(Ms=9e5, Aex=1.5e-11, Ku=1e4, easy_axis=(0.2, 0.3, 1.0), alpha=0.1, B=(0.02, 0.0, 0.01))
    samples = [dict(shape=(64, 64, 2), cell=(3e-9, 3e-9, 3e-9), pbc=(1, 1, 0), m_seed=31),
               dict(shape=(64, 40, 1), cell=(4e-9, 4e-9, 2e-9), pbc=(1, 0, 0), m_seed=32),
               dict(shape=(48, 36, 3), cell=(4e-9, 4e-9, 4e-9), pbc=(0, 0, 0), m_seed=33)]
    images, h = 2, 1e-13
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sol = [B.Solver(s["shape"], s["cell"], pbc=s["pbc"], images=images, stream=stream.cuda_stream,
                        tensor=False, fft_lengths=B.MM_FFT_POW2, **mat) for s in samples]
        m0 = _m0(samples)
        bt = B.Batch(sol, stream.cuda_stream)
        B.mm_batch_load(bt.b, m0)
        B.mm_batch_advance(bt.b, B.MM_RKDP, 1, dt_s=h, tol=-1.0)
        out = [torch.empty_like(m) for m in m0]
        B.mm_batch_store(bt.b, out)
        torch.cuda.synchronize()
    for i, s in enumerate(samples):
        p = llg.Problem(s["shape"], s["cell"], mat["Ms"], mat["Aex"], mat["alpha"], Ku=mat["Ku"],
                        u=mat["easy_axis"], B=mat["B"], pbc=tuple(bool(v) for v in s["pbc"]), images=images)
        m = m0[i].cpu().numpy().astype(np.float64)
        m /= np.sqrt((m * m).sum(axis=0, keepdims=True))
        ref = llg.rkdp_stages(p, m, h)[0]
        d = float(np.max(np.abs(out[i].cpu().numpy() - ref)))
        assert d < 1e-6, (i, s["shape"], s["pbc"], d)


def test_batch_autotuner_tile_shapes_agree():
    """The register x passes are also compiled with half the row pairs per
    block (twice the blocks, another work list): forcing that tile everywhere
    changes no result beyond float32 rounding, the tuner reports the groups
    that run it, and the timed choice (mode 1) agrees as well."""
    import torch
    samples = inputs.ensemble(6, seed=9, nmin=32, nmax=140, nzmax=3)
    stream = torch.cuda.Stream()
    outs, reports = {}, {}
    with torch.cuda.stream(stream):
        for mode in (0, 3, 1):
            sol = _solvers(samples, stream.cuda_stream)
            m0 = _m0(samples)
            bt = B.Batch(sol, stream.cuda_stream)
            B.mm_batch_set_tuning(bt.b, mode)
            B.mm_batch_load(bt.b, m0)
            B.mm_batch_advance(bt.b, B.MM_RKDP, 6, dt_s=5e-14, tol=-1.0)
            out = [torch.empty_like(m) for m in m0]
            B.mm_batch_store(bt.b, out)
            torch.cuda.synchronize()
            outs[mode] = out
            reports[mode] = B.mm_batch_tuning(bt.b)
    assert reports[3][2] > 0 and reports[0][2] == 0
    for mode in (1, 3):
        for a, b in zip(outs[0], outs[mode]):
            assert float((a - b).abs().max()) <= 1e-6
    with pytest.raises(B.MMError):
        B.mm_batch_set_tuning(bt.b, 4)
