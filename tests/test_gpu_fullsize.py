"""Parity at the benchmark's full size: the 1024 x 1024 x 1 film (2048 x 2048
padded FFT), in the launch configuration bench.py times.  The FP64 oracle
computes the whole field (its kernel takes about a minute to build), so every
cell is compared, plus one adaptive Dormand-Prince step."""

import numpy as np
import pytest

from oracle import llg
from paper_1102_3069_gb300 import binding as B
from paper_1102_3069_gb300 import inputs

from gpu_util import HEFF_REL_L2, HEFF_REL_MAX, oracle, rel_l2, rel_max, solver, to_dev, to_np

pytestmark = pytest.mark.gpu

W = inputs.workload("film_1024x1024")


@pytest.fixture(scope="module")
def pair():
    s = solver(W["shape"], W["cell"], pbc=W["pbc"], **W["material"])
    p = oracle(W["shape"], W["cell"], pbc=W["pbc"], **W["material"])
    return s, p


def test_full_size_heff(pair):
    s, p = pair
    m = W["m"]
    h, tq, e = s.heff(to_dev(m), torque=True, energy=True)
    m64 = m.astype(np.float64)
    t = p.terms(m64)
    H = t["d"] + t["ex"] + t["an"] + t["z"]
    Hg = to_np(h)
    print("rel L2", rel_l2(Hg, H), "rel max", rel_max(Hg, H))
    assert rel_l2(Hg, H) <= HEFF_REL_L2
    assert rel_max(Hg, H) <= HEFF_REL_MAX
    assert rel_l2(to_np(tq), llg.ll_rhs(m64, H, p.alpha)) <= 2 * HEFF_REL_L2
    E = p.energy(m64)
    assert abs(e - E) <= 1e-5 * abs(E), (e, E)


def test_full_size_rkdp_step(pair):
    s, p = pair
    m = W["m"]
    md = to_dev(m)
    acc, t, _ = B.mm_step(s.ctx, md, B.MM_RKDP, 0.0, 1e-13, tol=1.0)
    assert acc
    m0 = m.astype(np.float64)
    m0 /= np.sqrt((m0 * m0).sum(axis=0, keepdims=True))
    ref = llg.rkdp_stages(p, m0, 1e-13)[0]
    err = float(np.max(np.abs(to_np(md) - ref)))
    print("max|dm| one step", err)
    assert err <= 1e-6
