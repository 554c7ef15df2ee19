"""Stored oracle records (tests/golden/oracle_records.json).

The record was written by tests/golden/make_golden.py from the FP64 oracle
only.  Three kinds of checks:

* CPU, consistency: the stored numbers obey what the mathematics fixes
  whatever the oracle does - the per-term energies add up to the total (the
  energy is a sum over terms, Eq. 2-4 and the Zeeman term), dm/dt is
  perpendicular to m (both terms of Eq. 1 and of Eq. 7 are cross products
  with m), and every stepped m is a unit vector (the step renormalises).
* CPU, regression: the oracle run again on the same inputs gives the stored
  values back to FP64 rounding, so no change to its arithmetic goes unnoticed.
* GPU: the C-ABI path (field, dm/dt, energy, one Dormand-Prince or Heun
  step) matches the stored values at the sampled cells, with the same bounds
  as the element-wise parity tests.
"""

import importlib.util
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


def _gen():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


GEN = _gen()
SPECS = {s["name"]: s for s in GEN.case_specs()}
with open(os.path.join(GOLDEN, "oracle_records.json")) as _f:
    REC = json.load(_f)
NAMES = sorted(SPECS)


def test_record_covers_every_case():
    assert sorted(k for k in REC if not k.startswith("_")) == NAMES
    for name in NAMES:
        assert [tuple(c) for c in REC[name]["cells"]] == GEN.sample_cells(SPECS[name]["shape"])


@pytest.mark.parametrize("name", NAMES)
def test_record_is_self_consistent(name):
    r, spec = REC[name], SPECS[name]
    m = GEN.initial_m(spec)
    cells = [tuple(c) for c in r["cells"]]
    m_s = np.array([[m[c, z, y, x] for c in range(3)] for (z, y, x) in cells])
    d = np.array(r["dmdt"])
    # dm/dt is perpendicular to m (cross products with m only)
    assert np.all(np.abs((m_s * d).sum(axis=1)) <= 1e-12 * r["dmdt_absmax"])
    if "energy" in r and "cubic" not in spec:       # (the cubic term has no field-energy entry of its own)
        parts = r["energy_demag"] + r["energy_exchange"] + r["energy_uniaxial"] + r["energy_zeeman"]
        assert parts == pytest.approx(r["energy"], rel=1e-12, abs=0.0)
    for key in ("rkdp_m1", "heun_m1"):
        if key in r:
            n = np.linalg.norm(np.array(r[key]), axis=1)
            assert np.all(np.abs(n - 1.0) <= 1e-14)
            # the step moved every sampled cell by at most |dm/dt|max * h (plus the
            # higher-order terms of one short step)
            h = spec.get("rkdp_h", spec.get("heun_dt"))
            assert np.max(np.abs(np.array(r[key]) - m_s / np.linalg.norm(m_s, axis=1, keepdims=True))) <= \
                1.5 * r["dmdt_absmax"] * h


@pytest.mark.parametrize("name", NAMES)
def test_oracle_reproduces_record(name):
    r, spec = REC[name], SPECS[name]
    now = GEN.record(spec)
    assert now["cells"] == r["cells"]
    for key, scale in (("H", r["H_absmax"]), ("dmdt", r["dmdt_absmax"])):
        assert np.max(np.abs(np.array(now[key]) - np.array(r[key]))) <= 1e-10 * scale, key
    for key in ("H_absmax", "dmdt_absmax", "torque_max", "energy"):
        if key in r:
            assert now[key] == pytest.approx(r[key], rel=1e-10, abs=0.0), key
    for key in ("energy_demag", "energy_exchange", "energy_uniaxial", "energy_zeeman"):
        if key in r:
            assert abs(now[key] - r[key]) <= 1e-10 * abs(r["energy"]), key
    for key in ("rkdp_m1", "heun_m1"):
        if key in r:
            assert np.max(np.abs(np.array(now[key]) - np.array(r[key]))) <= 1e-12, key
    if "rkdp_err" in r:
        assert now["rkdp_err"] == pytest.approx(r["rkdp_err"], rel=1e-7, abs=0.0)


def _gpu_solver(spec):
    from paper_1102_3069_gb300 import binding as B
    s = B.Solver(spec["shape"], spec["cell"], pbc=spec["pbc"], images=spec["images"], tensor=False,
                 **spec["material"])
    if "cubic" in spec:
        c = spec["cubic"]
        B.mm_set_cubic_anisotropy(s.ctx, c["K1"], c["K2"], c["c1"], c["c2"])
    if "stt" in spec:
        t = spec["stt"]
        B.mm_set_stt(s.ctx, t["P"], t["xi"], t["j"])
    return s


def _at(a, cells):
    return np.array([[a[c, z, y, x] for c in range(3)] for (z, y, x) in cells], dtype=np.float64)


@pytest.mark.gpu
@pytest.mark.parametrize("name", NAMES)
def test_gpu_matches_record(name):
    import torch
    from paper_1102_3069_gb300 import binding as B
    r, spec = REC[name], SPECS[name]
    cells = [tuple(c) for c in r["cells"]]
    thermal = spec["material"].get("temperature", 0.0) > 0.0
    m = GEN.initial_m(spec).astype(np.float32)
    s = _gpu_solver(spec)
    if thermal:
        B.mm_set_thermal_clock(s.ctx, 0, spec["heun_dt"])
    md = torch.from_numpy(m).cuda()
    h, tq, e = s.heff(md, torque=True, energy=not thermal)
    torch.cuda.synchronize()
    # element-wise bound on H relative to its largest value, as the parity
    # tests; with the thermal field the Gaussians differ by libm-vs-device ulps
    hb = 2e-5 if thermal else 5e-6
    dH = np.max(np.abs(_at(h.cpu().numpy(), cells) - np.array(r["H"])))
    assert dH <= hb * r["H_absmax"], (name, dH / r["H_absmax"])
    # dm/dt = -gamma0/(1+a^2) [m x H + a m x (m x H)] moves by at most
    # gamma0 (1+a)/(1+a^2) |dH| <= 1.25 gamma0 |dH| for unit m, plus float32
    # rounding of the torque itself
    alpha = spec["material"]["alpha"]
    db = 2.211e5 * (1 + alpha) / (1 + alpha * alpha) * hb * r["H_absmax"] + 1e-6 * r["dmdt_absmax"]
    dD = np.max(np.abs(_at(tq.cpu().numpy(), cells) - np.array(r["dmdt"])))
    assert dD <= db, (name, dD / r["dmdt_absmax"])
    if "energy" in r:
        assert abs(e - r["energy"]) <= 2e-6 * abs(r["energy"]), (e, r["energy"])
    s.close()
    if "rkdp_h" in spec or "heun_dt" in spec:
        s = _gpu_solver(spec)
        md = torch.from_numpy(m).cuda()
        if "rkdp_h" in spec:
            acc, t, _ = B.mm_step(s.ctx, md, B.MM_RKDP, 0.0, spec["rkdp_h"], tol=1.0)
            key, dt = "rkdp_m1", spec["rkdp_h"]
        else:
            acc, t, _ = B.mm_step(s.ctx, md, B.MM_HEUN, 0.0, spec["heun_dt"])
            key, dt = "heun_m1", spec["heun_dt"]
        st = B.mm_get_stats(s.ctx)
        torch.cuda.synchronize()
        assert acc and t == pytest.approx(dt, rel=1e-12, abs=0.0)
        d1 = np.max(np.abs(_at(md.cpu().numpy(), cells) - np.array(r[key])))
        assert d1 <= (2e-6 if thermal else 1e-6), (name, d1)
        if "rkdp_err" in r:
            # err = h |sum_j (b_j - b*_j) k_j| cancels: each float32 k_j carries
            # ~1e-7 of |dm/dt|max, so agreement is a few per cent of a small err
            assert abs(st["last_err"] - r["rkdp_err"]) <= 0.1 * r["rkdp_err"] + 1e-9, (st["last_err"], r["rkdp_err"])
        s.close()
