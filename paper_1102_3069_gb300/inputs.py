"""Seeded synthetic inputs shared by the tests, the bench and the oracle runs.

This module holds no step of the method: only geometries, material constants
and initial magnetisations drawn from numpy's PCG64 with a given seed.  Arrays
are float32 with shape (3, nz, ny, nx) (component, z, y, x; x fastest), unit
vectors.  The named workloads follow the configurations the solver is
measured on:

* ``film_64x16``      64 x 16 x 1 cells of 4 nm, Ms 8.6e5 A/m, A 1.3e-11 J/m,
                      Ku 0, alpha 0.02, Bz = 10 mT, random unit vectors;
* ``film_1024x1024``  1024 x 1024 x 1 cells of 4 x 4 x 2 nm, Ms 8e5 A/m,
                      A 1.3e-11 J/m, Ku 5e3 J/m^3 along x, alpha 0.01, open
                      boundaries, vortex-plus-noise start, applied field of
                      magnitude U[0, 50] mT in a uniformly random direction;
* ``cube_256x256x64`` 256 x 256 x 64 cells of 3 nm, periodic in x and y,
                      Ms 1.1e6 A/m, A 2e-11 J/m, Ku 2e4 J/m^3 along per-cell
                      easy axes tilted by U[0, 30] deg from z (``axes``; the
                      material's easy_axis is one such draw), alpha 0.05,
                      300 K, Heun with dt = 50 fs;
* ``table1_N2`` / ``table1_N3``  square and cubic grids of the Euler-step
                      timing table, 4 nm cells with the film_1024x1024
                      material;
* ``ensemble(n)``     independent samples of the batched ensemble: nx, ny
                      uniform in 32..256, nz uniform in 1..4, 4 nm cells,
                      Ms U[4e5, 1.4e6] A/m, A U[5e-12, 2e-11] J/m, Ku
                      U[0, 5e4] J/m^3, easy axis and field direction uniform
                      on the sphere, |B| U[0, 50] mT, alpha 0.02, open
                      boundaries, random unit vectors;
* ``relax_films(n)``  128 x 128 x 1 films of 4 x 4 x 3 nm cells, Ms
                      U[6e5, 1e6] A/m, A 1.3e-11 J/m, Ku U[0, 5e4] J/m^3 along
                      a random in-plane axis, in-plane field of magnitude
                      U[0, 80] mT in a random direction, alpha 1 (relaxation),
                      random unit vectors.
"""

import numpy as np


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def random_unit(shape, seed):
    """m = normalised N(0, I3) per cell; shape = (nx, ny, nz)."""
    nx, ny, nz = shape
    g = rng(seed)
    m = g.standard_normal((3, nz, ny, nx))
    m /= np.sqrt((m * m).sum(axis=0, keepdims=True))
    return m.astype(np.float32)


def vortex_noise(shape, cell, seed, core_radius=10e-9, noise=0.05, chirality=1, polarity=1):
    """In-plane curling state with an out-of-plane core exp(-(r/r0)^2), plus
    N(0, noise^2) per component, normalised."""
    nx, ny, nz = shape
    dx, dy, _ = cell
    x = (np.arange(nx) - (nx - 1) / 2.0) * dx
    y = (np.arange(ny) - (ny - 1) / 2.0) * dy
    X, Y = np.meshgrid(x, y, indexing="xy")            # (ny, nx)
    r = np.sqrt(X * X + Y * Y)
    mz = polarity * np.exp(-(r / core_radius) ** 2)
    phi = np.arctan2(Y, X)
    s = np.sqrt(np.clip(1.0 - mz * mz, 0.0, 1.0))
    mx = -chirality * np.sin(phi) * s
    my = chirality * np.cos(phi) * s
    m = np.stack([mx, my, mz])[:, None, :, :].repeat(nz, axis=1)
    g = rng(seed)
    m = m + noise * g.standard_normal(m.shape)
    m /= np.sqrt((m * m).sum(axis=0, keepdims=True))
    return m.astype(np.float32)


def smooth_tilt(shape):
    """Smooth large-amplitude state along +x with long-wavelength tilts
    (m_y ~ 0.4 sin(2 pi x/Lx) + 0.2 cos(pi y/Ly), m_z ~ 0.3 sin(pi x/Lx) sin(pi y/Ly)),
    normalised.  Its dynamics are not chaotic: a 1e-7 perturbation of it stays at
    the 1e-7 level for 1000 Dormand-Prince steps of 100 fs on the 64 x 16 film,
    whereas from random unit vectors it grows to O(1)."""
    nx, ny, nz = shape
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)
    m = np.stack([np.ones_like(X), 0.4 * np.sin(2 * np.pi * X) + 0.2 * np.cos(np.pi * Y),
                  0.3 * np.sin(np.pi * X) * np.sin(np.pi * Y)])[:, None, :, :].repeat(nz, axis=1)
    m /= np.sqrt((m * m).sum(axis=0, keepdims=True))
    return m.astype(np.float32)


def tilted_axes(shape, seed, max_deg=30.0):
    """Per-cell unit easy axes tilted from z by theta ~ U[0, max_deg] deg with
    azimuth phi ~ U[0, 2 pi), float32 (3, nz, ny, nx)."""
    nx, ny, nz = shape
    g = rng(seed + 3000)
    th = np.deg2rad(g.uniform(0.0, max_deg, (nz, ny, nx)))
    ph = g.uniform(0.0, 2 * np.pi, (nz, ny, nx))
    u = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    u /= np.sqrt((u * u).sum(axis=0, keepdims=True))
    return u.astype(np.float32)


def random_direction(g):
    v = g.standard_normal(3)
    return v / np.linalg.norm(v)


def workload(name, seed=0):
    """Geometry, material and initial m of a named workload (dict)."""
    g = rng(seed + 1000)
    if name == "film_64x16":
        shape, cell = (64, 16, 1), (4e-9, 4e-9, 4e-9)
        mat = dict(Ms=8.6e5, Aex=1.3e-11, Ku=0.0, easy_axis=(1.0, 0.0, 0.0), alpha=0.02, B=(0.0, 0.0, 0.01))
        return dict(name=name, shape=shape, cell=cell, pbc=(0, 0, 0), material=mat, m=random_unit(shape, seed))
    if name == "film_1024x1024":
        shape, cell = (1024, 1024, 1), (4e-9, 4e-9, 2e-9)
        B = tuple(float(v) for v in g.uniform(0.0, 0.05) * random_direction(g))
        mat = dict(Ms=8e5, Aex=1.3e-11, Ku=5e3, easy_axis=(1.0, 0.0, 0.0), alpha=0.01, B=B)
        return dict(name=name, shape=shape, cell=cell, pbc=(0, 0, 0), material=mat,
                    m=vortex_noise(shape, cell, seed))
    if name == "cube_256x256x64":
        shape, cell = (256, 256, 64), (3e-9, 3e-9, 3e-9)
        th = np.deg2rad(g.uniform(0.0, 30.0))
        ph = g.uniform(0.0, 2 * np.pi)
        u = (float(np.sin(th) * np.cos(ph)), float(np.sin(th) * np.sin(ph)), float(np.cos(th)))
        mat = dict(Ms=1.1e6, Aex=2e-11, Ku=2e4, easy_axis=u, alpha=0.05, temperature=300.0, seed=seed,
                   B=(0.0, 0.0, 0.0))
        return dict(name=name, shape=shape, cell=cell, pbc=(1, 1, 0), material=mat, m=random_unit(shape, seed),
                    dt=50e-15, axes=tilted_axes(shape, seed))
    if name.startswith("table1_N2_") or name.startswith("table1_N3_"):
        n = int(name.rsplit("_", 1)[1])
        shape = (n, n, 1) if name.startswith("table1_N2_") else (n, n, n)
        cell = (4e-9, 4e-9, 4e-9)
        mat = dict(Ms=8e5, Aex=1.3e-11, Ku=5e3, easy_axis=(1.0, 0.0, 0.0), alpha=0.01, B=(0.0, 0.0, 0.01))
        return dict(name=name, shape=shape, cell=cell, pbc=(0, 0, 0), material=mat, m=random_unit(shape, seed))
    raise KeyError(name)


def ensemble(n, seed=0, nmin=32, nmax=256, nzmax=4, alpha=0.02):
    """n independent samples (dicts with shape, cell, pbc, material, m_seed);
    m = random_unit(shape, m_seed) is drawn on demand."""
    g = rng(seed + 2000)
    out = []
    for i in range(n):
        nx, ny = (int(v) for v in g.integers(nmin, nmax + 1, size=2))
        nz = int(g.integers(1, nzmax + 1))
        Ms = float(g.uniform(4e5, 1.4e6))
        A = float(g.uniform(5e-12, 2e-11))
        Ku = float(g.uniform(0.0, 5e4))
        u = tuple(float(v) for v in random_direction(g))
        B = tuple(float(v) for v in g.uniform(0.0, 0.05) * random_direction(g))
        mat = dict(Ms=Ms, Aex=A, Ku=Ku, easy_axis=u, alpha=alpha, B=B)
        out.append(dict(shape=(nx, ny, nz), cell=(4e-9, 4e-9, 4e-9), pbc=(0, 0, 0), material=mat,
                        m_seed=seed * 100003 + i))
    return out


def relax_films(n, seed=0, size=128, alpha=1.0):
    """n independent 128 x 128 x 1 films for relaxation (dicts as ``ensemble``)."""
    g = rng(seed + 4000)
    out = []
    for i in range(n):
        Ms = float(g.uniform(6e5, 1e6))
        Ku = float(g.uniform(0.0, 5e4))
        pu = g.uniform(0.0, 2 * np.pi)
        pb = g.uniform(0.0, 2 * np.pi)
        b = g.uniform(0.0, 0.08)
        mat = dict(Ms=Ms, Aex=1.3e-11, Ku=Ku, easy_axis=(float(np.cos(pu)), float(np.sin(pu)), 0.0), alpha=alpha,
                   B=(float(b * np.cos(pb)), float(b * np.sin(pb)), 0.0))
        out.append(dict(shape=(size, size, 1), cell=(4e-9, 4e-9, 3e-9), pbc=(0, 0, 0), material=mat,
                        m_seed=seed * 100003 + 50000 + i))
    return out


# ---- learned warm start (Fourier neural operator on 128 x 128 films) -------

FNO_N, FNO_WIDTH, FNO_MODES, FNO_CIN, FNO_CHID, FNO_COUT = 128, 32, 16, 16, 128, 3


def fno_features(samples):
    """Input fields (B, 16, 128, 128) float32 of the warm-start operator for
    relaxation samples (``relax_films``): channel 0 Ms/1e6, 1 Ku/5e4, 2-3 the
    in-plane easy axis, 4-5 the in-plane applied field / 0.08 T, 6 (x+1/2)/128,
    7 (y+1/2)/128; channels 8-15 zero."""
    n = FNO_N
    x = np.zeros((len(samples), FNO_CIN, n, n), dtype=np.float32)
    xs = ((np.arange(n) + 0.5) / n).astype(np.float32)
    for b, s in enumerate(samples):
        m = s["material"]
        vals = [m["Ms"] / 1e6, m["Ku"] / 5e4, m["easy_axis"][0], m["easy_axis"][1], m["B"][0] / 0.08,
                m["B"][1] / 0.08]
        for ch, v in enumerate(vals):
            x[b, ch] = v
        x[b, 6] = xs[None, :]
        x[b, 7] = xs[:, None]
    return x


def fno_init(seed=0):
    """Initial weights of the warm-start operator (float64 numpy arrays):
    uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) for the point-wise maps and their
    biases, and spectral weights (1/(32*32)) * U[0,1) for the real and the
    imaginary part (the usual FNO initialisation).  Spectral weights are
    indexed [mode, out, in], mode = kx*32 + (index of ky in 0..15, 112..127)."""
    g = rng(seed + 6000)
    W, C, H, O = FNO_WIDTH, FNO_CIN, FNO_CHID, FNO_COUT
    nm = FNO_MODES * 2 * FNO_MODES

    def lin(o, i):
        a = 1.0 / np.sqrt(i)
        return g.uniform(-a, a, (o, i)), g.uniform(-a, a, o)

    p = {}
    p["lift_w"], p["lift_b"] = lin(W, 8)
    p["lift_w"] = np.concatenate([p["lift_w"], np.zeros((W, C - 8))], axis=1)
    sc = 1.0 / (W * W)
    p["spec_w"] = [sc * (g.random((nm, W, W)) + 1j * g.random((nm, W, W))) for _ in range(4)]
    p["pw_w"], p["pw_b"] = [], []
    for _ in range(4):
        w, b = lin(W, W)
        p["pw_w"].append(w)
        p["pw_b"].append(b)
    p["proj1_w"], p["proj1_b"] = lin(H, W)
    p["proj2_w"], p["proj2_b"] = lin(O, H)
    return p
