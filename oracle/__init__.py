"""FP64 CPU oracle for the effective-field + Landau-Lifshitz time-step path.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, deliberately
unoptimised restatement of what the paper (arXiv:1102.3069, MuMax) computes:

* ``newell``   - the cell-averaged demagnetising tensor (Sec. 2.1.1, Eq. 2),
                 exact Newell form near the origin, tent-weighted Gauss-Legendre
                 quadrature of the point-dipole kernel far away;
* ``demag``    - zero-padded / periodic-image kernel and the FFT convolution
                 (Sec. 2.1.1 and Sec. 3.2 stages i-iii), plus direct O(N^2) sums;
* ``fields``   - exchange (Eq. 3), uniaxial anisotropy (Eq. 4), Zeeman,
                 thermal field (Eq. 6), total H_eff and energy;
* ``philox``   - Philox-4x32-10 counter-based generator + Box-Muller (the
                 source of the Gaussian vector eta in Eq. 6);
* ``llg``      - Landau-Lifshitz right-hand side (Eq. 1), Euler, Heun and
                 Dormand-Prince (Sec. 2.2) steps, step control, relaxation.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU
baseline leg and ``--impl reference``) may import anything from here.  The
CUDA path in ``paper_1102_3069_gb300`` never imports, links or calls it, and
this package never imports the CUDA path: the two share no code.  Inputs are
plain numpy arrays in SI units; every floating-point result is float64.

Parity status of each function is stated in its module header.  Everything
here is pinned by ``tests/test_oracle_*.py`` against closed forms, invariants,
brute force or published values; nothing is "parity unpinned".
"""

# submodules are imported explicitly by callers (oracle.newell, oracle.demag, ...)
