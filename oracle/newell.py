"""Cell-averaged demagnetising tensor N_ab(r) of a uniformly magnetised cuboid.

Paper: Sec. 2.1.1, Eq. (2): H_ms(r) = -(1/4pi) Int grad grad (1/|r-r'|) . M(r') dr'.
On a finite-difference grid of identical cuboid cells (Sec. 2.1.1, "regular
grid" paragraph) the field averaged over the target cell at offset r from a
uniformly magnetised source cell is H = -N(r) . M.  The paper does not name the
formula for N; we use its standard closed form (Newell, Williams & Dunlop,
J. Geophys. Res. 98:9551, 1993):

    N_xx(X,Y,Z) = 1/(4 pi dx dy dz) * sum_{i,j,k in {-1,0,1}} w_i w_j w_k
                  f(X + i dx, Y + j dy, Z + k dz),      w_0 = 2, w_{+-1} = -1,

N_xy the same sum with g instead of f; the other components permute the axes.
The 27-term sum cancels catastrophically far from the origin (the terms grow
like r^3 while N falls like 1/r^3), so beyond a few tens of cells we evaluate
the same cell-average by quadrature: for separated cells

    N_ab(r) = (1/V) Int Int D_ab(r + u - u') du du' = (1/V) Int D_ab(r + w) T(w) dw,

D_ab(s) = -(1/4pi) (3 s_a s_b - delta_ab |s|^2) / |s|^5 is the point-dipole
kernel and T(w) = prod_a (d_a - |w_a|)_+ is the overlap of two boxes (the
"tent").  Each axis is split at w_a = 0 and integrated with Gauss-Legendre
nodes on [-d_a, 0] and [0, d_a].

Pins (tests/test_oracle_newell.py): cube self-term 1/3, self trace 1, off-site
trace 0, parity, far field -> point dipole, Newell == quadrature where both are
accurate (also 2-3.5 cells apart with more nodes, which pins the off-diagonal
entries in the near field), whole-prism identity, the self-term against
Aharoni's closed-form prism factors, 50-digit mpmath evaluation; the
self-term in the dynamics by the Kittel precession of a flat cell
(tests/test_oracle_llg.py).

All lengths may be given in any unit (N is dimensionless and scale-free).
"""

import numpy as np

_FOUR_PI = 4.0 * np.pi


def _as_1d(x, y, z):
    """Broadcast to a common shape and flatten (so masked updates work on 0-d input)."""
    x, y, z = np.broadcast_arrays(np.asarray(x, float), np.asarray(y, float), np.asarray(z, float))
    return x.ravel().copy(), y.ravel().copy(), z.ravel().copy(), x.shape


def _asinh_ratio(num, den):
    """asinh(num/den) where den > 0; callers mask the den == 0 entries."""
    return np.arcsinh(num / den)


def newell_f(x, y, z):
    """Newell's f(x, y, z) (symmetric in y <-> z); terms with a zero prefactor are 0."""
    x, y, z, shape = _as_1d(x, y, z)
    x2, y2, z2 = x * x, y * y, z * z
    R = np.sqrt(x2 + y2 + z2)
    out = (2.0 * x2 - y2 - z2) * R / 6.0

    pre = 0.5 * y * (z2 - x2)
    den = np.sqrt(x2 + z2)
    m = pre != 0.0
    out[m] += pre[m] * _asinh_ratio(y[m], den[m])

    pre = 0.5 * z * (y2 - x2)
    den = np.sqrt(x2 + y2)
    m = pre != 0.0
    out[m] += pre[m] * _asinh_ratio(z[m], den[m])

    pre = x * y * z
    m = pre != 0.0
    out[m] -= pre[m] * np.arctan(y[m] * z[m] / (x[m] * R[m]))
    return out.reshape(shape)


def newell_g(x, y, z):
    """Newell's g(x, y, z) used for the off-diagonal N_xy; zero-prefactor terms are 0."""
    x, y, z, shape = _as_1d(x, y, z)
    x2, y2, z2 = x * x, y * y, z * z
    R = np.sqrt(x2 + y2 + z2)
    out = -x * y * R / 3.0

    pre = x * y * z
    m = pre != 0.0
    out[m] += pre[m] * _asinh_ratio(z[m], np.sqrt(x2[m] + y2[m]))

    pre = y * (3.0 * z2 - y2) / 6.0
    m = pre != 0.0
    out[m] += pre[m] * _asinh_ratio(x[m], np.sqrt(y2[m] + z2[m]))

    pre = x * (3.0 * z2 - x2) / 6.0
    m = pre != 0.0
    out[m] += pre[m] * _asinh_ratio(y[m], np.sqrt(x2[m] + z2[m]))

    pre = z * z2 / 6.0
    m = pre != 0.0
    out[m] -= pre[m] * np.arctan(x[m] * y[m] / (z[m] * R[m]))

    pre = 0.5 * z * y2
    m = pre != 0.0
    out[m] -= pre[m] * np.arctan(x[m] * z[m] / (y[m] * R[m]))

    pre = 0.5 * z * x2
    m = pre != 0.0
    out[m] -= pre[m] * np.arctan(y[m] * z[m] / (x[m] * R[m]))
    return out.reshape(shape)


_W = {-1: -1.0, 0: 2.0, 1: -1.0}


def _newell_sum(func, a, b, c, da, db, dc):
    """sum_{i,j,k} w_i w_j w_k func(a + i da, b + j db, c + k dc) / (4 pi da db dc)."""
    acc = 0.0
    for i in (-1, 0, 1):
        for j in (-1, 0, 1):
            for k in (-1, 0, 1):
                w = _W[i] * _W[j] * _W[k]
                acc = acc + w * func(a + i * da, b + j * db, c + k * dc)
    return acc / (_FOUR_PI * da * db * dc)


COMPONENTS = ("xx", "yy", "zz", "xy", "xz", "yz")


def newell_tensor(X, Y, Z, dx, dy, dz):
    """Exact (closed-form) cell-averaged tensor at physical offset (X, Y, Z).

    Returns a dict of the six independent components.  Accurate in float64 only
    near the origin (see module docstring); use :func:`demag_tensor` in general.
    """
    X, Y, Z = np.broadcast_arrays(np.asarray(X, float), np.asarray(Y, float), np.asarray(Z, float))
    return {
        "xx": _newell_sum(newell_f, X, Y, Z, dx, dy, dz),
        "yy": _newell_sum(newell_f, Y, X, Z, dy, dx, dz),
        "zz": _newell_sum(newell_f, Z, Y, X, dz, dy, dx),
        "xy": _newell_sum(newell_g, X, Y, Z, dx, dy, dz),
        "xz": _newell_sum(newell_g, X, Z, Y, dx, dz, dy),
        "yz": _newell_sum(newell_g, Y, Z, X, dy, dz, dx),
    }


def point_dipole_tensor(X, Y, Z, V):
    """N of a point dipole of volume V: -(V/4pi) (3 r_a r_b - delta_ab r^2) / r^5."""
    X, Y, Z = np.broadcast_arrays(np.asarray(X, float), np.asarray(Y, float), np.asarray(Z, float))
    r2 = X * X + Y * Y + Z * Z
    r5 = r2 * r2 * np.sqrt(r2)
    s = -V / (_FOUR_PI * r5)
    return {
        "xx": s * (3 * X * X - r2),
        "yy": s * (3 * Y * Y - r2),
        "zz": s * (3 * Z * Z - r2),
        "xy": s * 3 * X * Y,
        "xz": s * 3 * X * Z,
        "yz": s * 3 * Y * Z,
    }


def _tent_rule(d, n):
    """Nodes/weights integrating q(w) (d - |w|) over [-d, d]: GL-n on each half."""
    t, wt = np.polynomial.legendre.leggauss(n)
    # map [-1, 1] -> [0, d]
    w_pos = 0.5 * d * (t + 1.0)
    g_pos = 0.5 * d * wt * (d - w_pos)
    nodes = np.concatenate([-w_pos[::-1], w_pos])
    weights = np.concatenate([g_pos[::-1], g_pos])
    return nodes, weights


def quadrature_tensor(X, Y, Z, dx, dy, dz, n):
    """Cell-averaged tensor by tent-weighted Gauss-Legendre (n nodes per half-axis).

    Valid only when target and source cells do not touch (the integrand is the
    point-dipole kernel, singular at zero separation).
    """
    X, Y, Z = np.broadcast_arrays(np.asarray(X, float), np.asarray(Y, float), np.asarray(Z, float))
    V = dx * dy * dz
    nx_, wx_ = _tent_rule(dx, n)
    ny_, wy_ = _tent_rule(dy, n)
    nz_, wz_ = _tent_rule(dz, n)
    acc = {c: np.zeros(X.shape) for c in COMPONENTS}
    for a, wa in zip(nx_, wx_):
        for b, wb in zip(ny_, wy_):
            for c, wc in zip(nz_, wz_):
                w = wa * wb * wc / V          # (1/V) * tent weight; D below carries V=1
                D = point_dipole_tensor(X + a, Y + b, Z + c, 1.0)
                for k in COMPONENTS:
                    acc[k] += w * D[k]
    return acc


# Switch from the closed form to quadrature at NEAR_RADIUS (distance in units
# of the largest cell edge) and grade the node count per half-axis by distance.
# Measured against 50-digit mpmath (tests/test_oracle_newell.py): the float64
# closed form has relative error ~1e-13 at 2.4 cells and ~2e-12 at 3.6 cells
# (it grows like dist^5); the quadrature below stays under ~1e-13 everywhere
# it is used.
NEAR_RADIUS = 4.0


def _quad_order(dist):
    if dist < 10.0:
        return 8
    if dist < 25.0:
        return 6
    if dist < 80.0:
        return 4
    return 3


def demag_tensor(ix, iy, iz, dx, dy, dz):
    """Tensor at integer cell offsets (ix, iy, iz): Newell near, quadrature far.

    ix, iy, iz are integer arrays (broadcastable); dx, dy, dz the cell edges.
    Returns a dict of six float64 arrays.
    """
    ix, iy, iz = np.broadcast_arrays(np.asarray(ix), np.asarray(iy), np.asarray(iz))
    X, Y, Z = ix * float(dx), iy * float(dy), iz * float(dz)
    dmax = max(dx, dy, dz)
    dist = np.sqrt(X * X + Y * Y + Z * Z) / dmax
    out = {c: np.zeros(ix.shape) for c in COMPONENTS}
    near = dist < NEAR_RADIUS
    if near.any():
        t = newell_tensor(X[near], Y[near], Z[near], dx, dy, dz)
        for c in COMPONENTS:
            out[c][near] = t[c]
    far = ~near
    if far.any():
        orders = np.array([_quad_order(d) for d in dist[far]])
        idx_far = np.flatnonzero(far)
        for n in np.unique(orders):
            sel = idx_far[orders == n]
            t = quadrature_tensor(X.ravel()[sel], Y.ravel()[sel], Z.ravel()[sel], dx, dy, dz, int(n))
            for c in COMPONENTS:
                out[c].ravel()[sel] = t[c]
    return out
