"""Philox-4x32-10 counter-based generator and the Gaussian draw for Eq. 6.

The paper's thermal field (Sec. 2.1.3, Eq. 6) needs Gaussian numbers that are
uncorrelated in space and time.  We draw them from the counter-based generator
Philox-4x32 with 10 rounds (Salmon, Moraes, Dror & Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11), restated here from its published
definition:

    round:  (hi0, lo0) = mulhilo32(0xD2511F53, c0)
            (hi1, lo1) = mulhilo32(0xCD9E8D57, c2)
            c <- (hi1 ^ c1 ^ k0,  lo1,  hi0 ^ c3 ^ k1,  lo0)
    key schedule between rounds:  k0 += 0x9E3779B9,  k1 += 0xBB67AE85  (mod 2^32)

Assignment of counters (a choice of this library): key = (seed low 32 bits,
seed high 32 bits); counter = (linear cell index, step low 32, step high 32, 0).
Each 32-bit word w becomes u = ((w >> 9) + 0.5) * 2^-23, exactly representable
in binary32 and strictly inside (0, 1); Box-Muller then gives
    eta_x = sqrt(-2 ln u0) cos(2 pi u1),  eta_y = sqrt(-2 ln u0) sin(2 pi u1),
    eta_z = sqrt(-2 ln u2) cos(2 pi u3).
Pins: published known-answer vectors of Philox-4x32-10; moments of eta.
"""

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox-4x32-10; all arguments are uint32 arrays/scalars."""
    c = [np.asarray(v, dtype=np.uint64) & _MASK for v in (c0, c1, c2, c3)]
    c = list(np.broadcast_arrays(*c))
    c = [v.copy() for v in c]
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK
    for r in range(10):
        if r > 0:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c[0]           # < 2^64, exact in uint64
        p1 = _M1 * c[2]
        hi0, lo0 = p0 >> _S32, p0 & _MASK
        hi1, lo1 = p1 >> _S32, p1 & _MASK
        c = [(hi1 ^ c[1] ^ k0) & _MASK, lo1, (hi0 ^ c[3] ^ k1) & _MASK, lo0]
    return [v.astype(np.uint32) for v in c]


def uniform_open(w):
    """u = ((w >> 9) + 0.5) * 2^-23 in (0, 1); exact in binary32."""
    w = np.asarray(w, dtype=np.uint64)
    return ((w >> np.uint64(9)).astype(np.float64) + 0.5) * 2.0 ** -23


def thermal_eta(shape, seed, step):
    """Standard-normal eta of shape (3, nz, ny, nx) for one time step."""
    _, nz, ny, nx = shape
    n = nz * ny * nx
    cell = np.arange(n, dtype=np.uint64)
    seed = int(seed)
    step = int(step)
    w = philox4x32_10(cell, step & 0xFFFFFFFF, (step >> 32) & 0xFFFFFFFF, 0,
                      seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    u = [uniform_open(x) for x in w]
    r01 = np.sqrt(-2.0 * np.log(u[0]))
    r23 = np.sqrt(-2.0 * np.log(u[2]))
    eta = np.stack([r01 * np.cos(2.0 * np.pi * u[1]),
                    r01 * np.sin(2.0 * np.pi * u[1]),
                    r23 * np.cos(2.0 * np.pi * u[3])])
    return eta.reshape(3, nz, ny, nx)
