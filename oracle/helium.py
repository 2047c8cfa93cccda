"""Hydrogen + helium chemistry in the implicit step (oracle; test infrastructure only).

Sec. "Physical Model": with helium the species are n_HI, n_HII, n_HeI, n_HeII, n_HeIII and the
electron density is Eq. electron_density's hydrogen + helium case.  The paper writes it as
n_HII + n_HeII/4 + n_HeIII/2 for helium densities stored in hydrogen-mass units (mass density /
m_H); with true number densities, as here, it reads n_e = n_HII + n_HeII + 2 n_HeIII.  Step (v)
then solves Eqs. RT-cons_energy, RT-chemical_ionization (one equation per species) and
RT-cons_radiation for U = (e_c, n_HI, n_HeI, n_HeII, E); n_HII = n_H - n_HI and
n_HeIII = n_He - n_HeI - n_HeII by conservation, n_H = (1 - Y) rho / m_H, n_He = Y rho / (4 m_H).

Readings (the paper defers the rates and the local solutions to its references):

* Opacity and photo-ionisation by the one grey field above 13.6 eV: kappa = sum_i sigma_E,i n_i,
  Gamma_i = c sigma_G,i E, heating sum_i n_i c E (sigma_E,i - h nu_i sigma_G,i) (grey
  constants of ``spectrum.helium_grey_constants``).
* Recombination: hydrogen as before (alpha_B, times the clumping factor); helium case B from
  ``rates`` (HeII -> HeI radiative plus dielectronic, HeIII -> HeII), also times the clumping
  factor.  Cooling: ``rates.cooling_rate_he``.
* Local solutions, all with their coefficients frozen at the iterate U (as for hydrogen alone):
  - S_HI: exact solution over dt of y' = A (n_H - y)(n_H - y + n_e,He) - G y with the helium
    electrons n_e,He = n_HeII + 2 n_HeIII frozen: a Riccati equation with real roots, solved
    in Bernoulli form about its smaller root (reduces to the hydrogen-only S_n at n_e,He = 0);
  - S_HeI, S_HeII: exact solution over dt of the linear chain HeI <-> HeII <-> HeIII with n_e
    frozen, d(HeI, HeII)/dt = M (HeI, HeII) + c, here the top rows of the exponential of the
    augmented matrix [[M, c], [0, 0]] dt (scipy.linalg.expm);
  - S_e: as before with the helium terms in G - Lambda; T = (gamma-1) e_int rho / (k_B n_tot),
    n_tot = n_H + n_He + n_e.
* Residual norm (Eq. rmsnorm) over N (N_s + 2) = 5 N unknowns: helium species scaled by n_He.

Pinned in tests: the helium grey constants against the incomplete-gamma series, the chain and
the Riccati solutions against adaptive ODE integration, their equilibrium limits, helium
conservation, and the reduction to the hydrogen-only model at Y = 0.
"""
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sl

from . import constants as K
from . import model as M
from . import newton as N
from . import rates

NF = 5   # (e_c, n_HI, n_HeI, n_HeII, E)


@dataclass
class HeStep(M.Step):
    """One implicit step of hydrogen + helium gas (CGS comoving, like ``model.Step``)."""
    Y: float = 0.24                        # helium mass fraction
    nHeI_n: np.ndarray = None              # n_HeI and n_HeII at the step start
    nHeII_n: np.ndarray = None
    sigma_E_HeI: float = 0.0
    sigma_G_HeI: float = 0.0
    sigma_E_HeII: float = 0.0
    sigma_G_HeII: float = 0.0
    helium: bool = True

    @property
    def n_H(self):
        """Hydrogen number density (1 - Y) rho / m_H."""
        return (1.0 - self.Y) * self.rho_b / K.M_H

    @property
    def n_He(self):
        """Helium number density Y rho / (4 m_H)."""
        return self.Y * self.rho_b / (K.M_HE_OVER_M_H * K.M_H)


def electrons(st, nHI, nHeI, nHeII):
    """Eq. electron_density (hydrogen + helium), number densities."""
    return (st.n_H - nHI) + nHeII + 2.0 * (st.n_He - nHeI - nHeII)


def temperature(st, e_c, nHI, nHeI, nHeII):
    """T from the specific internal energy (Eqs. eos, temperature) with the particle count of
    hydrogen + helium gas, n_tot = n_H + n_He + n_e (Eq. electron_density); T_iso when
    isothermal."""
    if st.isothermal:
        return st.T_iso + 0.0 * nHI
    v2 = st.v[0] ** 2 + st.v[1] ** 2 + st.v[2] ** 2
    e_int = st.e_h + e_c - 0.5 * v2
    n_tot = st.n_H + st.n_He + electrons(st, nHI, nHeI, nHeII)
    return (K.GAMMA - 1.0) * e_int * st.rho_b / (K.K_BOLTZ * n_tot)


def riccati_SHI(y0, nH, neHe, A, G, dt):
    """Exact solution at dt of y' = A (nH - y)(nH + neHe - y) - G y, y(0) = y0.

    As a quadratic A y^2 - B y + C with B = A (2 nH + neHe) + G, C = A nH (nH + neHe); its
    discriminant is d^2 = (A neHe + G)^2 + 4 A G nH >= 0, the smaller root y_eq = 2C/(B + d);
    u = y - y_eq obeys u' = A u^2 - d u, so u(t) = u0 e^{-d t} / (1 - u0 A t phi1(d t)).
    """
    d = np.sqrt((A * neHe + G) ** 2 + 4.0 * A * G * nH)
    B = A * (2.0 * nH + neHe) + G
    den = B + d
    den0 = np.real(den) == 0
    y_eq = np.where(den0, 0.0, 2.0 * A * nH * (nH + neHe) / np.where(den0, 1.0, den))
    u0 = y0 - y_eq
    q = np.exp(-d * dt)
    return y_eq + u0 * q / (1.0 - u0 * A * dt * M.phi1(d * dt))


def he_chain(x0, nHe, G1, G2, r2, r3, dt):
    """Exact solution at dt of d(HeI, HeII)/dt = M (HeI, HeII) + c with
    M = [[-G1, r2], [G1 - r3, -(G2 + r2 + r3)]], c = (0, r3 nHe)  (HeIII = nHe - HeI - HeII):
    the top rows of expm([[M, c], [0, 0]] dt) applied to (HeI0, HeII0, 1)."""
    dt_ = np.result_type(*[np.asarray(v) for v in (*x0, nHe, G1, G2, r2, r3)], float)
    HeI0, HeII0 = (np.ravel(np.asarray(x, dtype=dt_)) for x in x0)
    n = HeI0.size
    bc = lambda v: np.broadcast_to(np.ravel(np.asarray(v, dtype=dt_)), (n,)) if np.ndim(v) else np.full(n, v, dt_)
    G1, G2, r2, r3, nHe = (bc(v) for v in (G1, G2, r2, r3, nHe))
    A = np.zeros((n, 3, 3), dt_)
    A[:, 0, 0] = -G1
    A[:, 0, 1] = r2
    A[:, 1, 0] = G1 - r3
    A[:, 1, 1] = -(G2 + r2 + r3)
    A[:, 1, 2] = r3 * nHe
    X = sl.expm(A * dt)
    HeI = X[:, 0, 0] * HeI0 + X[:, 0, 1] * HeII0 + X[:, 0, 2]
    HeII = X[:, 1, 0] * HeI0 + X[:, 1, 1] * HeII0 + X[:, 1, 2]
    return HeI, HeII


def local_solutions(st, U):
    """(S_e, (S_HI, S_HeI, S_HeII)) at the iterate U = (e_c, n_HI, n_HeI, n_HeII, E)."""
    e_c, nHI, nHeI, nHeII, E = U
    shape = np.shape(nHI)
    a3 = st.a**3
    nH, nHe = st.n_H, st.n_He
    Ebar = M.spos(st.theta * E + (1.0 - st.theta) * st.E_n, st.E_min)
    cEp = K.C_LIGHT * Ebar / a3                          # c E (proper)
    T = temperature(st, e_c, nHI, nHeI, nHeII)
    ne = electrons(st, nHI, nHeI, nHeII)
    neHe = nHeII + 2.0 * (nHe - nHeI - nHeII)
    A = rates.alpha_B(T, st.recomb) * st.clump / a3
    S_HI = riccati_SHI(st.nHI_n, nH, neHe, A, st.sigma_G * cEp, st.dt)
    r2 = (rates.alpha_HeII_B(T) + rates.alpha_di(T)) * st.clump * ne / a3
    r3 = rates.alpha_HeIII_B(T) * st.clump * ne / a3
    S_HeI, S_HeII = he_chain((st.nHeI_n, st.nHeII_n), nHe, st.sigma_G_HeI * cEp, st.sigma_G_HeII * cEp,
                             r2, r3, st.dt)
    S = (S_HI, S_HeI.reshape(shape), S_HeII.reshape(shape))
    if st.isothermal:
        return None, S
    heat = cEp * (nHI * (st.sigma_E - K.HNU0 * st.sigma_G) + nHeI * (st.sigma_E_HeI - K.HNU_HEI * st.sigma_G_HeI)
                  + nHeII * (st.sigma_E_HeII - K.HNU_HEII * st.sigma_G_HeII)) / st.rho_b
    cool = 0.0
    if st.cooling:
        nHeIII = nHe - nHeI - nHeII
        cool = a3 * rates.cooling_rate_he(T, ne / a3, nHI / a3, (nH - nHI) / a3, nHeII / a3, nHeIII / a3,
                                          st.a) / st.rho_b
    Se = (heat - cool) * st.dt * M.phi1(2.0 * (st.adot / st.a) * st.dt)
    return Se, S


def residual(st, U, bE=None, freeze=False):
    """f(U) = (f_e, f_HI, f_HeI, f_HeII, f_E) (Eqs. gas_residual, chemistry_residual per
    species, radiation_residual with the helium opacity)."""
    e_c, nHI, nHeI, nHeII, E = U
    if bE is None:
        bE = M.explicit_part(st)
    src = M.emissivity(st)
    Se, (S_HI, S_HeI, S_HeII) = local_solutions(st, U)
    f_e = e_c if st.isothermal else e_c - Se
    f_E = E - bE - st.dt * st.theta * M.radiation_rhs(st, E, nHI, src, freeze, nHe=(nHeI, nHeII))
    return np.stack([f_e, nHI - S_HI, nHeI - S_HeI, nHeII - S_HeII, f_E])


def weights(st, U):
    """Per-component scales of the residual norm: e_c as for hydrogen, n_HI by n_H, the helium
    species by n_He, E by max(|E|, E^n, E_floor)."""
    e_c, nHI, nHeI, nHeII, E = np.real(U)
    wE = 1.0 / np.maximum(np.maximum(np.abs(E), st.E_n), M.weight_floor_E(st))
    we = 1.0 / np.maximum(M.internal_energy_h(st), M.E_FLOOR_INT())
    nHe = st.n_He + 0 * E
    wHe = np.where(nHe > 0, 1.0 / np.where(nHe > 0, nHe, 1.0), 0.0)
    return np.stack([we + 0 * E, 1.0 / st.n_H + 0 * E, wHe, wHe, wE])


def _scales(st, U):
    e_c, nHI, nHeI, nHeII, E = np.real(U)
    z = 0 * E
    nHe = np.maximum(st.n_He, 1e-6 * st.n_H) + z       # a usable step scale even at Y = 0
    return np.stack([np.maximum(np.abs(e_c), M.E_FLOOR_INT()) + z, st.n_H + z, nHe, nHe,
                     np.maximum(np.abs(E), st.E_min)]).reshape(NF, -1)


def jacobian(st, U, bE=None, freeze=False):
    """Complex-step Jacobian of the 5N residual: the hydrogen oracle's routine with this
    residual and the helium scales."""
    return N.jacobian(st, U, bE, freeze, residual=residual, scales=_scales)


def _clamp(st, u, iso):
    """Keep 0 < n_HI <= n_H, 0 <= n_HeI, n_HeII with n_HeI + n_HeII <= n_He and e_int > 0."""
    out = list(u)
    k = 0 if iso else 1
    if not iso:
        out[0] = np.maximum(out[0], -0.999 * M.internal_energy_h(st))
    out[k] = np.clip(out[k], 1e-300, st.n_H)
    out[k + 1] = np.clip(out[k + 1], 0.0, st.n_He)
    out[k + 2] = np.clip(out[k + 2], 0.0, st.n_He - out[k + 1])
    return out


def local_solve(st, U, tol=1e-14, maxit=60, h=1e-30):
    """Cell-local equations at fixed E by a per-cell damped Newton iteration (complex-step
    derivatives): unknowns (n_HI, n_HeI, n_HeII) isothermal, with e_c otherwise; each step is
    halved until the scaled local residual (max over the components) decreases."""
    U = np.array(np.real(U), float)
    iso = st.isothermal
    idx = [1, 2, 3] if iso else [0, 1, 2, 3]
    E = U[4]
    scl = _scales(st, U).reshape((NF,) + st.shape)
    w = weights(st, U)

    def local_f(u):             # the local equations at u, with E fixed
        Ut = U.astype(complex) if np.iscomplexobj(u[0]) else U.copy()
        for j, i in enumerate(idx):
            Ut[i] = u[j]
        Ut[4] = E
        Se, S = local_solutions(st, Ut)
        f = [] if iso else [Ut[0] - Se]
        return f + [Ut[1] - S[0], Ut[2] - S[1], Ut[3] - S[2]]

    def scaled(f):              # max over the components of the weighted local residual
        return np.max(np.stack([np.abs(np.real(fi)) * w[i] for fi, i in zip(f, idx)]), axis=0)

    u = _clamp(st, [U[i] for i in idx], iso)
    f = local_f(u)
    r = scaled(f)
    k = len(idx)
    stuck = np.zeros(st.shape, bool)            # no decrease found: at the round-off floor
    for _ in range(maxit):
        active = (r > tol) & ~stuck
        if not np.any(active):
            break
        Jl = np.zeros(st.shape + (k, k))
        for j in range(k):
            up = [x.astype(complex) for x in u]
            up[j] = up[j] + 1j * h * scl[idx[j]]
            fp = local_f(up)
            for i in range(k):
                Jl[..., i, j] = np.imag(fp[i]) / (h * scl[idx[j]])
        rhs = -np.stack([np.real(fi) for fi in f], axis=-1)
        Jl[~active] = np.eye(k)
        rhs[~active] = 0.0
        du = np.linalg.solve(Jl, rhs[..., None])[..., 0]
        lam = np.ones(st.shape)
        todo = active.copy()
        for _ in range(40):
            ut = _clamp(st, [u[j] + lam * du[..., j] for j in range(k)], iso)
            ft = [np.real(x) for x in local_f(ut)]
            rt = scaled(ft)
            ok = todo & (rt < r)
            for j in range(k):
                u[j] = np.where(ok, ut[j], u[j])
            for i in range(k):
                f[i] = np.where(ok, ft[i], np.real(f[i]))
            r = np.where(ok, rt, r)
            todo &= ~ok
            if not np.any(todo):
                break
            lam = np.where(todo, 0.5 * lam, lam)
        stuck |= todo
    for j, i in enumerate(idx):
        U[i] = u[j]
    if iso:
        U[0] = 0.0
    return U


def initial_iterate(st):
    """Start of the Newton iteration: e_c = 0, the species at their start-of-step values and
    E^n + dt 4 pi eta (the local solve that follows moves the species to S(E))."""
    return np.stack([np.zeros(st.shape), st.nHI_n.copy(), st.nHeI_n.copy(), st.nHeII_n.copy(),
                     st.E_n + st.dt * M.emissivity(st)])


def solve_step(st, tol=1e-11, maxit=60, linear="auto"):
    """Globalised Newton for f(U) = 0 (full 5N Jacobian, sparse direct solves of the E-step,
    nonlinear elimination of the cell-local unknowns, Armijo backtracking), like
    ``newton.solve_step`` for hydrogen alone; returns (U, info)."""
    bE = M.explicit_part(st)
    U = local_solve(st, initial_iterate(st))
    hist = []
    for k in range(maxit + 1):
        f = np.real(residual(st, U, bE))
        w = weights(st, U)
        nrm = rms(w, f)
        hist.append(nrm)
        if not np.isfinite(nrm):
            raise FloatingPointError("oracle residual is not finite")
        if nrm <= tol:
            return U, dict(iters=k, hist=hist)
        if k == maxit:
            break
        J = jacobian(st, U, bE)
        S = N.linear_solve(J, -f.ravel(), linear).reshape(U.shape)
        lam = 1.0
        for _ in range(40):
            Ut = U.copy()
            Ut[4] = U[4] + lam * S[4]
            Ut = local_solve(st, Ut)
            nt = rms(w, residual(st, Ut, bE))
            if nt <= (1.0 - 1e-4 * lam) * nrm and nt < nrm:
                break
            lam *= 0.5
        else:
            raise RuntimeError("oracle line search failed")
        U = Ut
    raise RuntimeError(f"oracle Newton did not converge: {hist[-3:]}")


def rms(w, f):
    """Eq. rmsnorm over the N (N_s + 2) = 5 N unknowns."""
    v = (w * np.real(f)).ravel()
    return float(np.sqrt(np.dot(v, v) / v.size))


def energy_from_temperature(T, rho_b, nHI, nHeI, nHeII, Y, v):
    """Specific total energy for temperature T of hydrogen + helium gas (Eqs. eos, temperature
    with n_tot = n_H + n_He + n_e)."""
    nH = (1.0 - Y) * rho_b / K.M_H
    nHe = Y * rho_b / (K.M_HE_OVER_M_H * K.M_H)
    n_tot = nH + nHe + (nH - nHI) + nHeII + 2.0 * (nHe - nHeI - nHeII)
    return K.K_BOLTZ * T * n_tot / ((K.GAMMA - 1.0) * rho_b) + 0.5 * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2)


class Run:
    """Multi-step oracle run of a hydrogen + helium workload (``workloads.with_helium``)."""

    def __init__(self, w, theta=None):
        from . import driver
        from . import spectrum as S
        self._h = driver.Run(w, theta)              # hydrogen bookkeeping: time, grey constants
        self.w = w
        self.Y = w["Y"]
        self.helium_grey = S.helium_grey_constants(w["spectrum"], w.get("T_B", 1e5))
        self.nHeI = np.array(w["nHeI"], float)
        self.nHeII = np.array(w["nHeII"], float)
        self._h.e_h = energy_from_temperature(w["T0"], w["rho_b"], self._h.nHI, self.nHeI, self.nHeII, self.Y, w["v"])

    def make_step(self):
        """The hydrogen run's step with the helium state and grey constants added."""
        from dataclasses import fields
        base = self._h.make_step()
        kw = {f.name: getattr(base, f.name) for f in fields(base)}
        return HeStep(**kw, Y=self.Y, nHeI_n=self.nHeI, nHeII_n=self.nHeII, **self.helium_grey)

    def advance(self, tol=1e-11):
        """Solve one hydrogen + helium step and hand it over (all species, e_h += e_c)."""
        st = self.make_step()
        U, info = solve_step(st, tol=tol)
        e_c, nHI, nHeI, nHeII, E = U
        self._h.E, self._h.nHI = E, nHI
        self.nHeI, self.nHeII = nHeI, nHeII
        self._h.e_h = self._h.e_h + e_c
        self._h.t += self._h.dt
        return U, info

    @property
    def t(self):
        """Current time."""
        return self._h.t
