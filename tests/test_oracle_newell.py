"""Pins for oracle.newell: the cell-averaged demagnetising tensor.

Closed forms and invariants, not the formula re-typed:
* self-term of a cube is 1/3 on the diagonal (symmetry + trace);
* self-term trace is 1 for any cuboid, off-site trace is 0 (the potential of a
  uniformly magnetised body is harmonic outside it);
* parity (diagonal even, off-diagonal odd in each of its two axes);
* far field tends to the point-dipole tensor with a gap shrinking like (d/r)^2;
* the exact closed form and the quadrature (two unrelated formulas) agree in
  the band where both are accurate;
* whole-prism identity: summing N over all cell pairs of a box of cells gives
  the self-term of the whole box (superposition), which ties every offset of
  the tensor - near and far - to one closed-form number;
* thin-film and needle limits of the self-term;
* in the near field (2 to 3.5 cells, cells not touching) the closed form
  equals a 24-node quadrature of the point-dipole kernel, which pins the
  off-diagonal entries where no box identity reaches them;
* the self-term equals Aharoni's closed-form demagnetising factors of a
  rectangular prism (J. Appl. Phys. 83, 3432, 1998), an expression derived
  independently of Newell's f and g.
"""

import itertools

import numpy as np
import pytest

from oracle import newell as nw

from closed_forms import aharoni_dz as _aharoni_dz

CELLS = [(1.0, 1.0, 1.0), (4.0, 4.0, 2.0), (3.0, 3.0, 3.0), (4.0, 4.0, 3.0), (1.0, 2.0, 5.0)]


def test_cube_self_term_is_one_third():
    t = nw.newell_tensor(0.0, 0.0, 0.0, 2.5, 2.5, 2.5)
    for c in ("xx", "yy", "zz"):
        assert abs(float(t[c]) - 1.0 / 3.0) < 1e-14
    for c in ("xy", "xz", "yz"):
        assert abs(float(t[c])) < 1e-15


@pytest.mark.parametrize("cell", CELLS)
def test_self_trace_is_one(cell):
    t = nw.newell_tensor(0.0, 0.0, 0.0, *cell)
    assert abs(float(t["xx"] + t["yy"] + t["zz"]) - 1.0) < 1e-13


@pytest.mark.parametrize("cell", CELLS)
def test_offsite_trace_is_zero(cell):
    offs = np.array([(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (2, 1, 1), (3, 2, 0),
                     (7, 3, 1), (12, 5, 0), (40, 9, 2), (300, 100, 0)])
    t = nw.demag_tensor(offs[:, 0], offs[:, 1], offs[:, 2], *cell)
    tr = t["xx"] + t["yy"] + t["zz"]
    scale = np.max(np.abs(np.stack([t["xx"], t["yy"], t["zz"]])), axis=0)
    assert np.all(np.abs(tr) <= 1e-10 * scale + 1e-16)


def test_parity():
    cell = (4.0, 4.0, 2.0)
    base = np.array([(3, 2, 1), (1, 5, 2), (9, 4, 0), (30, 11, 3)])
    t0 = nw.demag_tensor(base[:, 0], base[:, 1], base[:, 2], *cell)
    # float64 rounding of the closed form near 4 cells is ~1e-12 of the largest entry
    tol = 1e-11 * np.max(np.abs(np.stack([t0[c] for c in nw.COMPONENTS])), axis=0)
    for sx, sy, sz in itertools.product((1, -1), repeat=3):
        t = nw.demag_tensor(sx * base[:, 0], sy * base[:, 1], sz * base[:, 2], *cell)
        for c in ("xx", "yy", "zz"):
            assert np.all(np.abs(t[c] - t0[c]) <= tol)
        assert np.all(np.abs(t["xy"] - sx * sy * t0["xy"]) <= tol)
        assert np.all(np.abs(t["xz"] - sx * sz * t0["xz"]) <= tol)
        assert np.all(np.abs(t["yz"] - sy * sz * t0["yz"]) <= tol)


def test_far_field_tends_to_point_dipole():
    cell = (4.0, 4.0, 2.0)
    V = cell[0] * cell[1] * cell[2]
    gaps = []
    for k in (25, 50, 100):
        off = np.array([3 * k, 2 * k, 0])
        t = nw.demag_tensor(off[0], off[1], off[2], *cell)
        d = nw.point_dipole_tensor(off[0] * cell[0], off[1] * cell[1], off[2] * cell[2], V)
        scale = max(abs(float(d[c])) for c in d)
        gaps.append(max(abs(float(t[c]) - float(d[c])) for c in d) / scale)
    assert gaps[0] < 1e-4
    # second-order convergence: doubling the distance divides the gap by ~4
    assert 3.5 < gaps[0] / gaps[1] < 4.5
    assert 3.5 < gaps[1] / gaps[2] < 4.5


@pytest.mark.parametrize("cell", CELLS)
def test_closed_form_and_quadrature_agree(cell):
    # band where the float64 closed form is still good (~1e-11) and the
    # quadrature with 8 nodes per half-axis already is (~1e-14)
    offs = [(4, 1, 0), (3, 3, 1), (5, 2, 0), (2, 4, 2), (6, 0, 0), (4, 4, 1)]
    dmax = max(cell)
    for o in offs:
        X, Y, Z = o[0] * cell[0], o[1] * cell[1], o[2] * cell[2]
        if np.sqrt(X * X + Y * Y + Z * Z) / dmax < 3.5:
            continue
        a = nw.newell_tensor(X, Y, Z, *cell)
        b = nw.quadrature_tensor(X, Y, Z, *cell, 8)
        scale = max(abs(float(a[c])) for c in a)
        for c in a:
            assert abs(float(a[c]) - float(b[c])) <= 2e-10 * scale, (o, c)


@pytest.mark.parametrize("cell,offs,nodes", [
    ((1.0, 1.0, 1.0), [(2, 1, 0), (2, 1, 1), (2, 2, 2), (3, 2, 1)], 16),
    ((4.0, 4.0, 2.0), [(2, 1, 1), (0, 2, 1), (1, 0, 2)], 16),
    ((1.0, 2.0, 5.0), [(2, 1, 0), (2, 2, 0), (3, 1, 0)], 24)])
def test_near_field_matches_fine_quadrature(cell, offs, nodes):
    # cells 2 to 3.5 cell sizes apart that do not touch: the point-dipole
    # kernel is smooth over the tent's support, so 16-24 Gauss-Legendre nodes
    # per half-axis converge to float64 level; every component, off-diagonal
    # included, is tied to an integral that does not use f or g (the box
    # identities above cancel the off-diagonal entries exactly)
    for o in offs:
        X, Y, Z = o[0] * cell[0], o[1] * cell[1], o[2] * cell[2]
        a = nw.newell_tensor(X, Y, Z, *cell)
        b = nw.quadrature_tensor(X, Y, Z, *cell, nodes)
        scale = max(abs(float(a[c])) for c in a)
        for c in a:
            assert abs(float(a[c]) - float(b[c])) <= 2e-11 * scale, (o, c)


def _prism_identity_gap(n, cell):
    nx, ny, nz = n
    ox, oy, oz = np.meshgrid(np.arange(-nx + 1, nx), np.arange(-ny + 1, ny), np.arange(-nz + 1, nz), indexing="ij")
    count = (nx - np.abs(ox)) * (ny - np.abs(oy)) * (nz - np.abs(oz))
    t = nw.demag_tensor(ox.ravel(), oy.ravel(), oz.ravel(), *cell)
    prism = nw.newell_tensor(0.0, 0.0, 0.0, nx * cell[0], ny * cell[1], nz * cell[2])
    gaps = {}
    for c in nw.COMPONENTS:
        avg = (t[c] * count.ravel()).sum() / (nx * ny * nz)
        gaps[c] = abs(avg - float(prism[c]))
    return gaps


@pytest.mark.parametrize("n,cell", [((6, 4, 1), (4.0, 4.0, 2.0)), ((9, 7, 3), (1.0, 1.0, 1.0)),
                                    ((40, 12, 1), (4.0, 4.0, 2.0)), ((64, 16, 1), (4.0, 4.0, 4.0)),
                                    ((12, 10, 6), (3.0, 3.0, 3.0)), ((100, 3, 2), (1.0, 2.0, 5.0))])
def test_whole_prism_identity(n, cell):
    gaps = _prism_identity_gap(n, cell)
    for c, g in gaps.items():
        assert g < 1e-11, (c, g)


def test_aharoni_formula_itself():
    # the restated formula before it serves as a pin: cube 1/3, trace 1
    assert _aharoni_dz(1.0, 1.0, 1.0) == pytest.approx(1.0 / 3.0, rel=1e-14, abs=0.0)
    for A, B, C in [(1.0, 2.0, 3.0), (10.0, 1.0, 0.5), (3.0, 7.0, 2.0)]:
        assert _aharoni_dz(B, C, A) + _aharoni_dz(C, A, B) + _aharoni_dz(A, B, C) == pytest.approx(1.0, abs=1e-13)


@pytest.mark.parametrize("sides", [(1.0, 2.0, 3.0), (4.0, 4.0, 2.0), (10.0, 1.0, 0.5), (3.0, 7.0, 2.0),
                                   (100.0, 100.0, 1.0), (1.0, 1.0, 100.0)])
def test_self_term_is_the_aharoni_prism_factor(sides):
    # the cell self-term of Eq. 2 is the demagnetising factor of the cell
    # itself, so every diagonal entry must equal Aharoni's closed form
    A, B, C = sides
    t = nw.newell_tensor(0.0, 0.0, 0.0, A, B, C)
    assert abs(float(t["xx"]) - _aharoni_dz(B, C, A)) <= 1e-12
    assert abs(float(t["yy"]) - _aharoni_dz(C, A, B)) <= 1e-12
    assert abs(float(t["zz"]) - _aharoni_dz(A, B, C)) <= 1e-12


def test_thin_film_and_needle_limits():
    # square platelet a x a x t: 1 - N_zz = 2 N_xx -> 0 like (t/a) ln(a/t)
    gaps = []
    for a in (100.0, 1000.0, 10000.0):
        film = nw.newell_tensor(0.0, 0.0, 0.0, a, a, 1.0)
        assert float(film["xx"]) == pytest.approx(float(film["yy"]), rel=1e-12, abs=0.0)
        gaps.append((1.0 - float(film["zz"])) / (np.log(a) / a))
    assert 0.0 < gaps[2] < gaps[1] < gaps[0] < 1.0
    needle = nw.newell_tensor(0.0, 0.0, 0.0, 1.0, 1.0, 1000.0)
    assert 0.0 < float(needle["zz"]) < 2e-3
    assert abs(float(needle["xx"]) - 0.5) < 2e-3


def test_matches_50_digit_evaluation():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50

    def f(x, y, z):
        x, y, z = mp.mpf(x), mp.mpf(y), mp.mpf(z)
        R = mp.sqrt(x * x + y * y + z * z)
        out = (2 * x * x - y * y - z * z) * R / 6
        if y * (z * z - x * x) != 0:
            out += y / 2 * (z * z - x * x) * mp.asinh(y / mp.sqrt(x * x + z * z))
        if z * (y * y - x * x) != 0:
            out += z / 2 * (y * y - x * x) * mp.asinh(z / mp.sqrt(x * x + y * y))
        if x * y * z != 0:
            out -= x * y * z * mp.atan(y * z / (x * R))
        return out

    def g(x, y, z):
        x, y, z = mp.mpf(x), mp.mpf(y), mp.mpf(z)
        R = mp.sqrt(x * x + y * y + z * z)
        out = -x * y * R / 3
        if x * y * z != 0:
            out += x * y * z * mp.asinh(z / mp.sqrt(x * x + y * y))
        if y * (3 * z * z - y * y) != 0:
            out += y / 6 * (3 * z * z - y * y) * mp.asinh(x / mp.sqrt(y * y + z * z))
        if x * (3 * z * z - x * x) != 0:
            out += x / 6 * (3 * z * z - x * x) * mp.asinh(y / mp.sqrt(x * x + z * z))
        if z != 0:
            out -= z ** 3 / 6 * mp.atan(x * y / (z * R))
        if z * y * y != 0:
            out -= z * y * y / 2 * mp.atan(x * z / (y * R))
        if z * x * x != 0:
            out -= z * x * x / 2 * mp.atan(y * z / (x * R))
        return out

    w = {-1: -1, 0: 2, 1: -1}

    def S(fn, a, b, c, da, db, dc):
        acc = mp.mpf(0)
        for i in (-1, 0, 1):
            for j in (-1, 0, 1):
                for k in (-1, 0, 1):
                    acc += w[i] * w[j] * w[k] * fn(a + i * da, b + j * db, c + k * dc)
        return acc / (4 * mp.pi * da * db * dc)

    cell = (4.0, 4.0, 2.0)
    dx, dy, dz = cell
    for o in [(0, 0, 0), (1, 0, 0), (1, 1, 0), (3, 2, 1), (6, 3, 0), (17, 4, 1), (45, 30, 0), (150, 7, 0)]:
        X, Y, Z = o[0] * dx, o[1] * dy, o[2] * dz
        ref = {"xx": S(f, X, Y, Z, dx, dy, dz), "yy": S(f, Y, X, Z, dy, dx, dz),
               "zz": S(f, Z, Y, X, dz, dy, dx), "xy": S(g, X, Y, Z, dx, dy, dz),
               "xz": S(g, X, Z, Y, dx, dz, dy)}
        got = nw.demag_tensor(*o, *cell)
        scale = max(abs(float(v)) for v in ref.values())
        for c, v in ref.items():
            assert abs(float(got[c]) - float(v)) <= 1e-11 * scale, (o, c)
