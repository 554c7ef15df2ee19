"""Helpers shared by the GPU parity tests: one call builds the CUDA solver and
the oracle problem from the same parameters and the same seeded input."""

import numpy as np

from oracle import llg
from paper_1102_3069_gb300 import binding as B

# relative L2 error bound on H_eff (FP32 path vs FP64 oracle)
HEFF_REL_L2 = 1e-6
# element-wise bound, relative to max |H| (FFT round-off is not uniform)
HEFF_REL_MAX = 5e-6


def solver(shape, cell, pbc=(0, 0, 0), images=10, demag=True, **mat):
    return B.Solver(shape, cell, pbc=pbc, images=images, demag=demag, **mat)


def oracle(shape, cell, pbc=(0, 0, 0), images=10, demag=True, Ms=8e5, Aex=1.3e-11, Ku=0.0,
           easy_axis=(1.0, 0.0, 0.0), alpha=0.02, gamma0=0.0, temperature=0.0, seed=0, B=(0.0, 0.0, 0.0)):
    kw = {}
    if gamma0:
        kw["gamma0"] = gamma0
    return llg.Problem(shape, cell, Ms, Aex, alpha, Ku=Ku, u=easy_axis, B=B, T=temperature, seed=seed,
                       pbc=tuple(bool(p) for p in pbc), images=images, demag=demag, **kw)


def to_dev(m):
    import torch
    return torch.from_numpy(np.ascontiguousarray(m, dtype=np.float32)).cuda()


def to_np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def rel_max(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
