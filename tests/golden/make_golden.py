"""Writes tests/golden/oracle_records.json: stored oracle results for four
small problems.  Run from the repository root:

    python tests/golden/make_golden.py

It calls only the FP64 oracle (``oracle/``) and the seeded input generators
(``paper_1102_3069_gb300.inputs``, which hold none of the method's
arithmetic).  No value in the record comes from the CUDA path.

What the record is for:
* ``tests/test_golden.py`` (CPU) re-runs the oracle on the same inputs and
  requires the stored values back to FP64 rounding.  A later change to the
  oracle's arithmetic therefore shows up as a changed record, which has to be
  regenerated with this script and justified by the passage of the paper it
  follows.
* the GPU half of the same test file compares the C-ABI path with the stored
  values, so the parity check does not depend on the oracle of the day.

Cases (each lists the equations it exercises):
* ``film_64x16``: the named 64 x 16 x 1 film (Eq. 1-3, Zeeman, Sec. 3.2
  zero-padded convolution), one Dormand-Prince attempt (Sec. 2.2);
* ``prism_16x8x3_periodic_xy``: a 3-D prism periodic in x and y (the CUDA
  path takes power-of-two periodic lengths) with three images per side
  (Sec. 2.1.1 periodic boundaries), uniaxial anisotropy (Eq. 4), one
  Dormand-Prince attempt;
* ``film_33x7_cubic_stt``: cubic anisotropy (Eq. 5) and the Zhang-Li
  spin-transfer torque (Eq. 7), recorded as dm/dt;
* ``film_24x10x2_thermal_heun``: one Heun step (Sec. 2.2) with the thermal
  field of Eq. 6 at 300 K (Philox-4x32-10 counter = step 0).

Sampled cells: the eight corners of the grid, the centre and the centres of
the x and y edges, and eight cells spread by fixed strides.  H in A/m, dm/dt
in 1/s, energies in J, torque dimensionless (max |m x H| / Ms).
"""

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import fields as F          # noqa: E402
from oracle import llg                  # noqa: E402
from paper_1102_3069_gb300 import inputs  # noqa: E402

OUT = os.path.join(HERE, "oracle_records.json")


def case_specs():
    """The four problems: geometry, material (mm_set_material keywords), the
    seed of random_unit and the extra terms; shared by the generator and the
    tests so both build exactly the same problem."""
    w = inputs.workload("film_64x16")
    return [
        dict(name="film_64x16", shape=w["shape"], cell=w["cell"], pbc=w["pbc"], images=10, m_seed=0,
             material=dict(w["material"]), rkdp_h=1e-13,
             cite="Eq. 1, Eq. 2, Eq. 3, Zeeman term, Sec. 3.2, Sec. 2.2 (Dormand-Prince)"),
        dict(name="prism_16x8x3_periodic_xy", shape=(16, 8, 3), cell=(3e-9, 3e-9, 3e-9), pbc=(1, 1, 0), images=3,
             m_seed=5, material=dict(Ms=1.1e6, Aex=2e-11, Ku=2e4, easy_axis=(0.2, 0.3, 1.0), alpha=0.05,
                                     B=(0.01, 0.0, 0.02)), rkdp_h=1e-13,
             cite="Eq. 1-4, Sec. 2.1.1 (periodic images), Sec. 2.2 (Dormand-Prince)"),
        dict(name="film_33x7_cubic_stt", shape=(33, 7, 1), cell=(4e-9, 3e-9, 2e-9), pbc=(0, 0, 0), images=10,
             m_seed=4, material=dict(Ms=8e5, Aex=1.3e-11, Ku=5e3, easy_axis=(1.0, 2.0, 3.0), alpha=0.1,
                                     B=(0.01, -0.02, 0.03)),
             cubic=dict(K1=4.8e4, K2=-1.5e4, c1=(1.0, 1.0, 0.0), c2=(-1.0, 1.0, 0.5)),
             stt=dict(P=0.56, xi=0.05, j=(1e12, -4e11, 2e11)),
             cite="Eq. 1-5, Eq. 7 (Zhang-Li spin-transfer torque)"),
        dict(name="film_24x10x2_thermal_heun", shape=(24, 10, 2), cell=(3e-9, 3e-9, 3e-9), pbc=(0, 0, 0), images=10,
             m_seed=3, material=dict(Ms=1.1e6, Aex=2e-11, Ku=0.0, easy_axis=(1.0, 0.0, 0.0), alpha=0.05,
                                     B=(0.0, 0.0, 0.0), temperature=300.0, seed=123456789),
             heun_dt=20e-15, cite="Eq. 1-3, Eq. 6 (thermal field), Sec. 2.2 (Heun)"),
    ]


def sample_cells(shape):
    nx, ny, nz = shape
    cells = set()
    for z in (0, nz - 1):
        for y in (0, ny - 1):
            for x in (0, nx - 1):
                cells.add((z, y, x))
    cells.add((nz // 2, ny // 2, nx // 2))
    cells.add((0, 0, nx // 2))
    cells.add((0, ny // 2, 0))
    for i in range(8):
        cells.add(((3 * i + 1) % nz, (5 * i + 3) % ny, (11 * i + 2) % nx))
    return sorted(cells)


def problem(spec):
    mat = spec["material"]
    kw = {}
    if "cubic" in spec:
        c = spec["cubic"]
        kw.update(K1=c["K1"], K2=c["K2"], c1=c["c1"], c2=c["c2"])
    if "stt" in spec:
        s = spec["stt"]
        kw.update(stt_P=s["P"], stt_xi=s["xi"], stt_j=s["j"])
    return llg.Problem(spec["shape"], spec["cell"], mat["Ms"], mat["Aex"], mat["alpha"], Ku=mat.get("Ku", 0.0),
                       u=mat.get("easy_axis", (1.0, 0.0, 0.0)), B=mat.get("B", (0.0, 0.0, 0.0)),
                       T=mat.get("temperature", 0.0), seed=mat.get("seed", 0),
                       pbc=tuple(bool(v) for v in spec["pbc"]), images=spec["images"], **kw)


def initial_m(spec):
    """float32 unit vectors as the GPU receives them, widened to float64."""
    return inputs.random_unit(spec["shape"], spec["m_seed"]).astype(np.float64)


def at(a, cells):
    return [[float(a[c, z, y, x]) for c in range(3)] for (z, y, x) in cells]


def record(spec):
    p = problem(spec)
    m = initial_m(spec)
    cells = sample_cells(spec["shape"])
    out = dict(cite=spec["cite"], cells=[list(c) for c in cells])
    dt = spec.get("heun_dt")
    t = p.terms(m, step=0, dt=dt)
    H = t["d"] + t["ex"] + t["an"] + t["cub"] + t["z"] + t["th"]
    out["H"] = at(H, cells)
    out["H_absmax"] = float(np.abs(H).max())
    rhs = p.rhs(m, step=0, dt=dt)
    out["dmdt"] = at(rhs, cells)
    out["dmdt_absmax"] = float(np.abs(rhs).max())
    out["torque_max"] = float(F.torque_max(m, H, p.Ms))
    if p.T == 0.0:
        z = np.zeros_like(m)
        out["energy"] = float(p.energy(m))
        out["energy_demag"] = float(F.energy(m, p.Ms, p.V, t["d"], z, z, z))
        out["energy_exchange"] = float(F.energy(m, p.Ms, p.V, z, t["ex"], z, z))
        out["energy_uniaxial"] = float(F.energy(m, p.Ms, p.V, z, z, t["an"], z))
        out["energy_zeeman"] = float(F.energy(m, p.Ms, p.V, z, z, z, t["z"]))
    if "rkdp_h" in spec:
        m1, _k, err = llg.rkdp_stages(p, llg.normalize(m), spec["rkdp_h"])
        out["rkdp_m1"] = at(m1, cells)
        out["rkdp_err"] = float(err)
    if dt is not None:
        m1 = llg.heun_step(p, llg.normalize(m), dt, step=0)
        out["heun_m1"] = at(m1, cells)
    return out


def main():
    rec = {"_about": ("FP64 oracle results for four small problems, written by tests/golden/make_golden.py "
                      "from oracle/ only; the inputs are paper_1102_3069_gb300.inputs.random_unit(shape, m_seed) "
                      "as float32 widened to float64.  Units: A/m, 1/s, J.")}
    for spec in case_specs():
        rec[spec["name"]] = record(spec)
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1, sort_keys=True)
        f.write("\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
