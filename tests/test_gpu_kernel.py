"""GPU demag-kernel setup (FP64 Newell + quadrature + images) vs the oracle tensor."""

import numpy as np
import pytest

from oracle import demag, newell

from gpu_util import solver

pytestmark = pytest.mark.gpu

MAT = dict(Ms=8e5, Aex=1.3e-11)


@pytest.mark.parametrize("shape,cell", [((1, 1, 1), (4e-9, 4e-9, 4e-9)), ((7, 5, 1), (4e-9, 4e-9, 2e-9)),
                                        ((64, 16, 1), (4e-9, 4e-9, 4e-9)), ((9, 6, 3), (3e-9, 2e-9, 5e-9)),
                                        ((120, 40, 2), (4e-9, 4e-9, 2e-9))])
def test_open_tensor_octant_matches_oracle(shape, cell):
    s = solver(shape, cell, **MAT)
    nx, ny, nz = shape
    got = s.tensor.reshape(6, nz, ny, nx)
    IZ, IY, IX = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ref = newell.demag_tensor(IX.ravel(), IY.ravel(), IZ.ravel(), *cell)
    scale = max(np.max(np.abs(ref[c])) for c in newell.COMPONENTS)
    for i, c in enumerate(newell.COMPONENTS):
        err = np.max(np.abs(got[i].ravel() - ref[c]))
        assert err <= 1e-12 * scale, (c, err / scale)


@pytest.mark.parametrize("shape,pbc,images", [((8, 8, 1), (1, 1, 0), 3), ((16, 4, 2), (1, 0, 0), 4),
                                              ((4, 4, 4), (0, 0, 1), 2)])
def test_periodic_tensor_octant_matches_oracle(shape, pbc, images):
    cell = (3e-9, 3e-9, 3e-9)
    s = solver(shape, cell, pbc=pbc, images=images, **MAT)
    K = demag.padded_kernel(shape, cell, tuple(bool(p) for p in pbc), images)
    nx, ny, nz = shape
    o = [n // 2 + 1 if p else n for n, p in zip(shape, pbc)]
    got = s.tensor.reshape(6, o[2], o[1], o[0])
    scale = max(np.max(np.abs(K[c])) for c in newell.COMPONENTS)
    for i, c in enumerate(newell.COMPONENTS):
        ref = K[c][:o[2], :o[1], :o[0]]
        err = np.max(np.abs(got[i] - ref))
        assert err <= 1e-12 * scale, (c, err / scale)
