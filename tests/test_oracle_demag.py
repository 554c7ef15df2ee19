"""Pins for oracle.demag: the zero-padded / periodic FFT convolution.

* FFT convolution == brute-force O(N^2) sum (open and periodic axes);
* the field does not depend on the padded length (any L >= 2N-1 gives the
  same linear convolution);
* the transformed kernel is real (symmetric kernel, Sec. 3.2) - also with the
  even-N periodic tie-break;
* uniform magnetisation: the mean field over the body is -N_prism . M
  (superposition of the cell tensors = tensor of the whole prism);
* a film periodic in x and y tends to the infinite-slab limit
  (N_zz -> 1, N_xx -> 0) as images are added.
"""

import numpy as np
import pytest

from oracle import demag, newell


def _rand_m(shape, seed):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    m = rng.standard_normal((3, nz, ny, nx))
    return m / np.linalg.norm(m, axis=0, keepdims=True)


@pytest.mark.parametrize("shape,cell", [((5, 3, 2), (4.0, 4.0, 2.0)), ((4, 4, 1), (3.0, 3.0, 3.0)),
                                        ((7, 1, 1), (1.0, 2.0, 3.0)), ((1, 1, 3), (2.0, 2.0, 1.0)),
                                        ((6, 5, 1), (4e-9, 4e-9, 2e-9))])
def test_fft_matches_direct_sum_open(shape, cell):
    m = _rand_m(shape, 1)
    Ms = 8e5
    d = demag.Demag(shape, cell)
    Hf = d.field(m, Ms)
    Hd = demag.demag_field_direct(m, Ms, cell)
    assert np.max(np.abs(Hf - Hd)) <= 1e-12 * Ms


@pytest.mark.parametrize("shape,pbc", [((4, 3, 1), (True, False, False)), ((3, 4, 2), (False, True, False)),
                                       ((4, 4, 1), (True, True, False)), ((5, 2, 2), (True, False, True))])
def test_fft_matches_direct_sum_periodic(shape, pbc):
    m = _rand_m(shape, 2)
    cell = (3.0, 3.0, 3.0)
    Ms = 1.1e6
    d = demag.Demag(shape, cell, pbc=pbc, images=2)
    Hf = d.field(m, Ms)
    Hd = demag.demag_field_direct(m, Ms, cell, pbc=pbc, images=2)
    assert np.max(np.abs(Hf - Hd)) <= 1e-12 * Ms


def test_independent_of_padded_length():
    shape, cell = (9, 6, 3), (4.0, 4.0, 2.0)
    m = _rand_m(shape, 3)
    ref = demag.Demag(shape, cell).field(m, 1.0)      # good sizes: 18, 12, 5
    for L in [(17, 11, 5), (32, 16, 8), (21, 14, 7)]:
        H = demag.Demag(shape, cell, L=L).field(m, 1.0)
        assert np.max(np.abs(H - ref)) < 1e-13


@pytest.mark.parametrize("shape,pbc", [((8, 6, 1), (False, False, False)), ((8, 6, 3), (True, True, False)),
                                       ((6, 4, 4), (True, False, True))])
def test_kernel_spectrum_is_real(shape, pbc):
    d = demag.Demag(shape, (3.0, 2.0, 1.0), pbc=pbc, images=3)
    scale = max(np.max(np.abs(Kh.real)) for Kh in d.Khat.values())
    for c, Kh in d.Khat.items():
        assert np.max(np.abs(Kh.imag)) <= 1e-13 * scale, c


def test_padded_length_rule():
    assert demag.padded_length(64, False) == 128
    assert demag.padded_length(33, False) == 80       # 65 -> 2^4 * 5
    assert demag.padded_length(1, False) == 1
    assert demag.padded_length(1024, False) == 2048
    assert demag.padded_length(24, True) == 24
    assert demag.padded_length(50, False) == 112      # 99 -> 2^4 * 7


@pytest.mark.parametrize("shape,cell,axis", [((16, 8, 1), (4.0, 4.0, 2.0), 0), ((10, 10, 4), (3.0, 3.0, 3.0), 2)])
def test_uniform_body_mean_field(shape, cell, axis):
    nx, ny, nz = shape
    m = np.zeros((3, nz, ny, nx))
    m[axis] = 1.0
    H = demag.Demag(shape, cell).field(m, 1.0)
    prism = newell.newell_tensor(0.0, 0.0, 0.0, nx * cell[0], ny * cell[1], nz * cell[2])
    col = [("xx", "xy", "xz"), ("xy", "yy", "yz"), ("xz", "yz", "zz")][axis]
    for comp in range(3):
        assert H[comp].mean() == pytest.approx(-float(prism[col[comp]]), abs=1e-11)


def test_periodic_film_tends_to_slab():
    shape, cell = (8, 8, 1), (4.0, 4.0, 2.0)
    mz = np.zeros((3, 1, 8, 8))
    mz[2] = 1.0
    mx = np.zeros((3, 1, 8, 8))
    mx[0] = 1.0
    gz, gx = [], []
    for P in (2, 8, 32):
        d = demag.Demag(shape, cell, pbc=(True, True, False), images=P)
        gz.append(1.0 + d.field(mz, 1.0)[2].mean())      # N_zz - 1
        gx.append(-d.field(mx, 1.0)[0].mean())           # N_xx
    for g in (gz, gx):
        assert abs(g[2]) < abs(g[1]) < abs(g[0])
        assert abs(g[2]) < 5e-3
