"""Landau-Lifshitz right-hand side, time integrators, step control, relaxation.

Paper: Sec. 2 Eq. (1) (Landau-Lifshitz form), Sec. 2.2 (Runge-Kutta family:
RK1 Euler, RK2 Heun, RKDP Dormand-Prince with an adaptive step bounded by a
maximum tolerable error per step).  Dividing Eq. (1) by Ms (M = Ms m):

    dm/dt = -gamma0/(1+alpha^2) [ m x H + alpha m x (m x H) ].

Readings where the paper is silent:
* RKDP tableau: Dormand & Prince (1980), J. Comput. Appl. Math. 6:19, FSAL,
  6 new evaluations per step.
* step error  err = max_i | h sum_j (b_j - b*_j) k_j,i |  (Euclidean norm per
  cell; |m| = 1 so absolute == relative); accept iff err <= tol;
  h_new = h * clamp(0.9 (tol/err)^(1/5), 0.2, 5), factor capped at 1 on the
  step right after a rejection; h < 1e-20 s is a failure.
* only the candidate m_{n+1} is renormalised (before its FSAL evaluation);
  intermediate stage states are not.  Euler and Heun renormalise the result.
* thermal field: one eta per step, shared by both Heun stages; sigma uses the
  fixed step dt (Eq. 6).  Thermal noise with the adaptive method is refused.
* relaxation: adaptive RKDP until max_i |m_i x H_i| / Ms < torque_tol.
* fixed maximum variation of m per step (the methods without an error
  estimate): every step has h = dm_max / max_i |dm/dt(m_n)|_i (capped at h_cap
  when given), the size that moves the fastest cell by dm_max to first order;
  the step itself is the method's (max_dm_step).

Pins: tests/test_oracle_llg.py (macrospin precession and damping closed forms,
Larmor/Kittel frequencies, convergence orders 1/2/5 and of every tableau,
embedded error orders, the step controller's special cases, |m| conservation,
energy decay, the Stoner-Wohlfarth angle reached by relaxation, Langevin
statistics of the thermal macrospin, the dissipation as the energy rate).
"""

import numpy as np

from . import demag as _demag
from . import fields as F
from . import philox

# Dormand-Prince 5(4) tableau
DP_C = (0.0, 1 / 5, 3 / 10, 4 / 5, 8 / 9, 1.0, 1.0)
DP_A = (
    (),
    (1 / 5,),
    (3 / 40, 9 / 40),
    (44 / 45, -56 / 15, 32 / 9),
    (19372 / 6561, -25360 / 2187, 64448 / 6561, -212 / 729),
    (9017 / 3168, -355 / 33, 46732 / 5247, 49 / 176, -5103 / 18656),
    (35 / 384, 0.0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84),
)
DP_B = (35 / 384, 0.0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84, 0.0)
DP_BSTAR = (5179 / 57600, 0.0, 7571 / 16695, 393 / 640, -92097 / 339200, 187 / 2100, 1 / 40)

H_MIN = 1e-20


class NotConverged(RuntimeError):
    pass


def normalize(m):
    n = np.sqrt((m * m).sum(axis=0, keepdims=True))
    return m / n


def ll_rhs(m, H, alpha, gamma0=F.GAMMA0):
    """dm/dt of Eq. (1) divided by Ms; H in A/m, result in 1/s."""
    mxH = np.cross(m, H, axis=0)
    mxmxH = np.cross(m, mxH, axis=0)
    return -gamma0 / (1.0 + alpha * alpha) * (mxH + alpha * mxmxH)


class Problem:
    """One finite-difference geometry + material; evaluates H_eff and dm/dt.

    shape (nx, ny, nz); cell (dx, dy, dz) in m; Ms A/m; Aex J/m; Ku J/m^3 with
    easy axis u; alpha; B applied flux density (T); T temperature (K) with
    Philox seed; gamma0 m/(A s); pbc flags; images per periodic axis.
    """

    def __init__(self, shape, cell, Ms, Aex, alpha, Ku=0.0, u=(1.0, 0.0, 0.0),
                 B=(0.0, 0.0, 0.0), T=0.0, seed=0, gamma0=F.GAMMA0,
                 pbc=(False, False, False), images=10, demag=True, L=None,
                 K1=0.0, K2=0.0, c1=(1.0, 0.0, 0.0), c2=(0.0, 1.0, 0.0),
                 stt_P=0.0, stt_xi=0.0, stt_j=(0.0, 0.0, 0.0)):
        self.shape = tuple(int(v) for v in shape)
        self.cell = tuple(float(v) for v in cell)
        self.V = self.cell[0] * self.cell[1] * self.cell[2]
        self.Ms, self.Aex, self.alpha = float(Ms), float(Aex), float(alpha)
        self.Ku = float(Ku)
        u = np.asarray(u, float)
        self.u = u / np.sqrt((u * u).sum(axis=0, keepdims=True)) if u.ndim > 1 else u / np.linalg.norm(u)
        self.B = np.asarray(B, float)
        self.T, self.seed, self.gamma0 = float(T), int(seed), float(gamma0)
        self.pbc = tuple(bool(p) for p in pbc)
        self.demag = _demag.Demag(self.shape, self.cell, self.pbc, images, L) if demag else None
        self.K1, self.K2 = float(K1), float(K2)
        self.c1, self.c2 = np.asarray(c1, float), np.asarray(c2, float)
        self.stt_P, self.stt_xi, self.stt_j = float(stt_P), float(stt_xi), tuple(float(v) for v in stt_j)
        self.n_evals = 0

    @property
    def mshape(self):
        nx, ny, nz = self.shape
        return (3, nz, ny, nx)

    def terms(self, m, step=0, dt=None):
        """All H_eff contributions (A/m) as a dict: d, ex, an, z, th."""
        m = np.asarray(m, float)
        zero = np.zeros_like(m)
        out = {
            "d": self.demag.field(m, self.Ms) if self.demag is not None else zero,
            "ex": F.exchange_field(m, self.Ms, self.Aex, self.cell, self.pbc),
            "an": F.anisotropy_field(m, self.Ms, self.Ku, self.u) if self.Ku != 0.0 else zero,
            "cub": (F.cubic_anisotropy_field(m, self.Ms, self.K1, self.K2, self.c1, self.c2)
                    if (self.K1 != 0.0 or self.K2 != 0.0) else zero),
            "z": F.zeeman_field(m, self.B),
            "th": zero,
        }
        if self.T > 0.0:
            if dt is None:
                raise ValueError("thermal field needs the fixed step dt")
            eta = philox.thermal_eta(m.shape, self.seed, step)
            out["th"] = F.thermal_field(eta, self.alpha, self.T, self.Ms, self.V, dt, self.gamma0)
        return out

    def heff(self, m, step=0, dt=None):
        t = self.terms(m, step, dt)
        self.n_evals += 1
        return t["d"] + t["ex"] + t["an"] + t["cub"] + t["z"] + t["th"]

    def rhs(self, m, step=0, dt=None):
        d = ll_rhs(m, self.heff(m, step, dt), self.alpha, self.gamma0)
        if self.stt_P != 0.0 and any(v != 0.0 for v in self.stt_j):
            d = d + F.stt_torque(m, self.alpha, self.stt_P, self.stt_xi, self.stt_j, self.cell, self.Ms, self.pbc)
        return d

    def energy(self, m):
        t = self.terms(m)
        e = F.energy(m, self.Ms, self.V, t["d"], t["ex"], t["an"], t["z"])
        if self.K1 != 0.0 or self.K2 != 0.0:
            e += self.V * F.cubic_energy_density(np.asarray(m, float), self.K1, self.K2, self.c1, self.c2).sum()
        return e

    def torque(self, m):
        return F.torque_max(m, self.heff(m), self.Ms)


def euler_step(p, m, dt, step=0):
    """RK1: m_{n+1} = normalize(m_n + dt f(m_n))."""
    return normalize(m + dt * p.rhs(m, step, dt))


def heun_step(p, m, dt, step=0):
    """RK2 (Heun): predictor m + dt k1, corrector m + dt/2 (k1 + k2); same eta in both."""
    k1 = p.rhs(m, step, dt)
    k2 = p.rhs(m + dt * k1, step, dt)
    return normalize(m + 0.5 * dt * (k1 + k2))


def rkdp_stages(p, m, h, k1=None):
    """One Dormand-Prince attempt of size h from m.

    Returns (m_next normalised, k list [k1..k7], err) where k7 = f(m_next).
    """
    if p.T > 0.0:
        raise ValueError("thermal field with the adaptive method is not supported")
    k = [p.rhs(m) if k1 is None else k1]
    for s in range(1, 6):
        ms = m.copy()
        for j, a in enumerate(DP_A[s]):
            if a != 0.0:
                ms = ms + h * a * k[j]
        k.append(p.rhs(ms))
    mn = m.copy()
    for j in range(6):
        if DP_B[j] != 0.0:
            mn = mn + h * DP_B[j] * k[j]
    mn = normalize(mn)
    k.append(p.rhs(mn))
    e = np.zeros_like(m)
    for j in range(7):
        d = DP_B[j] - DP_BSTAR[j]
        if d != 0.0:
            e = e + h * d * k[j]
    err = float(np.sqrt((e * e).sum(axis=0)).max())
    return mn, k, err


def rkdp_fixed(p, m, h, nsteps):
    """nsteps Dormand-Prince steps of fixed size h (no rejection), FSAL reuse."""
    k1 = None
    for _ in range(nsteps):
        m, k, _err = rkdp_stages(p, m, h, k1)
        k1 = k[6]
    return m


def controller_factor(err, tol, after_reject):
    if err == 0.0:
        f = 5.0
    else:
        f = 0.9 * (tol / err) ** 0.2
    f = min(max(f, 0.2), 5.0)
    if after_reject:
        f = min(f, 1.0)
    return f


class Stepper:
    """Adaptive Dormand-Prince with the controller of the module docstring."""

    def __init__(self, p, m, h0=1e-13, tol=1e-6, t=0.0):
        self.p, self.m, self.h, self.tol, self.t = p, normalize(np.asarray(m, float)), float(h0), float(tol), float(t)
        self.k1 = None
        self.after_reject = False
        self.accepted = 0
        self.rejected = 0
        self.last_torque = None

    def step(self):
        """One attempt; returns True if accepted."""
        mn, k, err = rkdp_stages(self.p, self.m, self.h, self.k1)
        if self.k1 is None:
            self.k1 = k[0]
        if err <= self.tol:
            self.t += self.h
            self.m = mn
            self.k1 = k[6]
            self.accepted += 1
            f = controller_factor(err, self.tol, self.after_reject)
            self.after_reject = False
            self.h *= f
            ok = True
        else:
            self.rejected += 1
            self.after_reject = True
            self.h *= controller_factor(err, self.tol, True)
            ok = False
        if self.h < H_MIN:
            raise NotConverged("step size underflow")
        return ok

    def run_until(self, t_end, max_steps=10 ** 9):
        n = 0
        while self.t < t_end and n < max_steps:
            self.h = min(self.h, t_end - self.t) if t_end - self.t > 0 else self.h
            self.step()
            n += 1
        return self.m


def relax(p, m, torque_tol=1e-4, h0=1e-13, tol=1e-6, max_steps=100000):
    """Adaptive RKDP until max |m x H|/Ms < torque_tol; returns (m, accepted steps, torque)."""
    st = Stepper(p, m, h0, tol)
    tq = p.torque(st.m)
    n = 0
    while tq >= torque_tol:
        if n >= max_steps:
            raise NotConverged("relax: max steps")
        if st.step():
            tq = F.torque_max(st.m, ll_heff_from_k1(p, st.m), p.Ms)
        n += 1
    return st.m, st.accepted, tq


def ll_heff_from_k1(p, m):
    """H_eff at m (the FSAL evaluation re-done explicitly, for the torque)."""
    return p.heff(m)


# ---------------------------------------------------------------------------
# The rest of the Runge-Kutta family of Sec. 2.2, as explicit tableaus.
# Coefficients from the published schemes: Kutta's third-order method, the
# classical fourth-order method, Heun-Euler (2nd order with an embedded Euler
# step), Bogacki & Shampine (1989) 3(2) with first-same-as-last, Cash & Karp
# (1990) 5(4).  For an embedded pair the step-size factor uses the exponent
# 1/q, q = order of the error estimate's leading term in h.

class Tableau:
    def __init__(self, name, a, b, bstar=None, fsal=False, q=None):
        self.name, self.a, self.b, self.bstar, self.fsal, self.q = name, a, b, bstar, fsal, q

    @property
    def stages(self):
        return len(self.b)

    @property
    def adaptive(self):
        return self.bstar is not None


TABLEAUS = {
    "rk3": Tableau("rk3", ((), (1 / 2,), (-1.0, 2.0)), (1 / 6, 2 / 3, 1 / 6)),
    "rk4": Tableau("rk4", ((), (1 / 2,), (0.0, 1 / 2), (0.0, 0.0, 1.0)), (1 / 6, 1 / 3, 1 / 3, 1 / 6)),
    "rk12": Tableau("rk12", ((), (1.0,)), (1 / 2, 1 / 2), bstar=(1.0, 0.0), q=2),
    "rk23": Tableau("rk23", ((), (1 / 2,), (0.0, 3 / 4), (2 / 9, 1 / 3, 4 / 9)), (2 / 9, 1 / 3, 4 / 9, 0.0),
                    bstar=(7 / 24, 1 / 4, 1 / 3, 1 / 8), fsal=True, q=3),
    "rkck": Tableau("rkck", ((), (1 / 5,), (3 / 40, 9 / 40), (3 / 10, -9 / 10, 6 / 5),
                             (-11 / 54, 5 / 2, -70 / 27, 35 / 27),
                             (1631 / 55296, 175 / 512, 575 / 13824, 44275 / 110592, 253 / 4096)),
                    (37 / 378, 0.0, 250 / 621, 125 / 594, 0.0, 512 / 1771),
                    bstar=(2825 / 27648, 0.0, 18575 / 48384, 13525 / 55296, 277 / 14336, 1 / 4), q=5),
    "rkdp": Tableau("rkdp", DP_A, DP_B, bstar=DP_BSTAR, fsal=True, q=5),
}


def rk_attempt(p, m, h, tab, k1=None, step=0, dt=None):
    """One attempt of an explicit tableau.

    Stage s input: m + h sum_j a_sj k_j (not renormalised); the result
    m + h sum_j b_j k_j is renormalised.  With first-same-as-last the last
    stage is evaluated at that renormalised result.  Returns (m_next, k, err),
    err = max_i |h sum_j (b_j - b*_j) k_j,i| (0 without an embedded pair).
    One thermal draw per step is shared by all stages (dt = the step).
    """
    if p.T > 0.0 and tab.adaptive:
        raise ValueError("thermal field with an adaptive method is not supported")
    k = [p.rhs(m, step, dt) if k1 is None else k1]
    S = tab.stages
    for s in range(1, S):
        ms = m.copy()
        for j, a in enumerate(tab.a[s]):
            if a != 0.0:
                ms = ms + h * a * k[j]
        if tab.fsal and s == S - 1:
            ms = normalize(ms)
        k.append(p.rhs(ms, step, dt))
    if tab.fsal:
        mn = ms
    else:
        mn = m.copy()
        for j in range(S):
            if tab.b[j] != 0.0:
                mn = mn + h * tab.b[j] * k[j]
        mn = normalize(mn)
    err = 0.0
    if tab.adaptive:
        e = np.zeros_like(m)
        for j in range(S):
            d = tab.b[j] - tab.bstar[j]
            if d != 0.0:
                e = e + h * d * k[j]
        err = float(np.sqrt((e * e).sum(axis=0)).max())
    return mn, k, err


def rk_fixed(p, m, h, nsteps, tab):
    """nsteps fixed steps of a tableau (first-same-as-last reuse when it has it)."""
    k1 = None
    for n in range(nsteps):
        m, k, _ = rk_attempt(p, m, h, tab, k1, step=n, dt=h)
        k1 = k[-1] if tab.fsal else None
    return m


class TableauStepper(Stepper):
    """Adaptive stepping of an embedded tableau with the same controller as
    Stepper but the step-size exponent 1/q of that tableau."""

    def __init__(self, p, m, tab, h0=1e-13, tol=1e-6, t=0.0):
        super().__init__(p, m, h0, tol, t)
        self.tab = tab

    def _factor(self, err, after_reject):
        f = 5.0 if err == 0.0 else 0.9 * (self.tol / err) ** (1.0 / self.tab.q)
        f = min(max(f, 0.2), 5.0)
        return min(f, 1.0) if after_reject else f

    def step(self):
        mn, k, err = rk_attempt(self.p, self.m, self.h, self.tab, self.k1 if self.tab.fsal else None)
        if err <= self.tol:
            self.t += self.h
            self.m = mn
            self.k1 = k[-1] if self.tab.fsal else None
            self.accepted += 1
            self.h *= self._factor(err, self.after_reject)
            self.after_reject = False
            ok = True
        else:
            if self.tab.fsal and self.k1 is None:
                self.k1 = k[0]
            self.rejected += 1
            self.after_reject = True
            self.h *= self._factor(err, True)
            ok = False
        if self.h < H_MIN:
            raise NotConverged("step size underflow")
        return ok


# Fixed maximum variation of m per step (Sec. 2.2): the methods without an
# error estimate, as tableaus (Euler and Heun next to RK3 and RK4).
MAXDM_TABLEAUS = {
    "euler": Tableau("euler", ((),), (1.0,)),
    "heun": Tableau("heun", ((), (1.0,)), (1 / 2, 1 / 2)),
    "rk3": TABLEAUS["rk3"],
    "rk4": TABLEAUS["rk4"],
}


def max_dm_step(p, m, tab, dm_max, h_cap=None):
    """One step whose size moves the fastest cell by dm_max to first order:
    h = dm_max / max_i |dm/dt(m)|_i, capped at h_cap.  Returns (m_next, h)."""
    if p.T > 0.0:
        raise ValueError("thermal field with a varying step is not supported")
    k1 = p.rhs(m)
    kmax = float(np.sqrt((k1 * k1).sum(axis=0)).max())
    if kmax > 0.0:
        h = dm_max / kmax
        if h_cap:
            h = min(h, h_cap)
    else:
        h = float(h_cap or 0.0)
    mn, _, _ = rk_attempt(p, m, h, tab, k1)
    return mn, h


def max_dm_run(p, m, tab, dm_max, nsteps, h_cap=None):
    """nsteps max-variation steps; returns (m, t, list of h)."""
    t, hs = 0.0, []
    for _ in range(nsteps):
        m, h = max_dm_step(p, m, tab, dm_max, h_cap)
        t += h
        hs.append(h)
    return m, t, hs
