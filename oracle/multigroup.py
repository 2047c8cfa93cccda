"""Multigroup flux-limited diffusion for the implicit step (oracle; test infrastructure only).

Sec. "Physical Model": the grey radiation equation (Eq. cons_radiation) is obtained from the
multifrequency one (Eq. cons_radiation_multifreq) by assuming a fixed spectral shape chi_E(nu)
over the whole ionising range [nu_0, inf) (Eq. grey_definition).  The multigroup version keeps
that assumption only within each of G frequency groups, [nu_{g-1}, nu_g) with
nu_0 < nu_1 < ... < nu_G = inf:

    E_nu(x, t, nu) = E_g(x, t) chi_E(nu) / int_g chi_E dnu   on group g,

and integrates Eq. cons_radiation_multifreq over each group.  Term by term:

  * diffusion: div(D_g grad E_g), D_g from Eq. limiter with the group's own energy and
    opacity (lagged like the grey D: from the step's starting state);
  * absorption: c kappa_g E_g with kappa_g = sigma_E,g n_HI / a^3, sigma_E,g the chi_E-weighted
    mean cross section over the group (the grey sigma_E restricted to the group);
  * emission: 4 pi eta_g = f_g 4 pi eta, f_g the fraction of the source spectrum's energy in
    the group (the sources emit the same chi_E as the grey model assumes);
  * redshift: int_g nu (adot/a) dE_nu/dnu dnu = (adot/a) ([nu E_nu] at the group's edges - E_g).
    Reading: photons redshift downwards, so the value of nu E_nu at an edge is taken from the
    group above it (upwind in frequency): the edge flux (adot/a) t_{g+1} E_{g+1}, with
    t_g = nu_{g-1} chi_E(nu_{g-1}) / int_g chi_E dnu, leaves group g+1 and enters group g.  The
    flux through nu_0 (photons leaving the ionising range) is dropped, as the grey equation,
    written with -(adot/a) E alone, drops it; with G = 1 the equations are the grey ones, and
    the edge fluxes cancel in the sum over groups, so sum_g E_g obeys the grey equation's
    expansion term;
  * chemistry and heating: Gamma = sum_g c sigma_G,g Ebar_g / a^3 and the photo-heating
    sum_g n_HI c Ebar_g (sigma_E,g - h nu_0 sigma_G,g) / a^3, with Ebar_g = pos(theta E_g +
    (1 - theta) E_g^n) as in the grey model.

Unknowns per cell: (e_c, n_HI, E_1, ..., E_G).  Only hydrogen; only the blackbody spectrum
(a monochromatic source has nothing to split).

Pinned in tests/test_oracle_multigroup.py: the group constants sum to the grey ones; the edge
coefficients against a quadrature of the spectrum's derivative (the redshift term of the
continuous spectrum); G = 1 reproduces the grey residual and root; groups with identical
constants reproduce the grey root split in proportion to their emission; the complex-step
Jacobian against central differences.
"""
import dataclasses
import math
from dataclasses import dataclass

import numpy as np
from scipy import integrate

from . import constants as K
from . import model as M
from . import newton as N
from . import rates


# --------------------------------------------------------------------- group constants


def _bb(weight, x0, x1):
    """int_{x0}^{x1} weight(x) / (e^x - 1) dx (x1 may be inf)."""
    def integrand(x):
        return weight(x) * math.exp(-x) / -math.expm1(-x)
    val, _ = integrate.quad(integrand, x0, x1, epsabs=0.0, epsrel=1e-13, limit=400)
    return val


def group_constants(edges_ev, T_B=1e5):
    """Constants of the groups [e_{g-1}, e_g) (photon energies in eV, edges_ev[0] = 13.6 eV's
    hydrogen edge, the last group open to infinity) for a T_B blackbody chi_E ~ x^3/(e^x - 1),
    x = h nu / k T_B, and the hydrogen cross section sigma_0 (nu/nu_0)^-3:

      sigma_E[g] = int_g sigma chi_E / int_g chi_E,   sigma_G[g] = int_g sigma chi_E/(h nu) / int_g chi_E,
      frac[g]    = int_g chi_E / int_all chi_E (share of the emitted energy),
      t[g]       = nu_{g-1} chi_E(nu_{g-1}) / int_g chi_E (edge coefficient; t[0] is unused),

    and eps_src, the mean photon energy of the whole spectrum (as in the grey model)."""
    kT = K.K_BOLTZ * T_B
    x0 = K.HNU0 / kT
    xs = [e * K.EV / kT for e in edges_ev] + [math.inf]
    if abs(xs[0] - x0) > 1e-12 * x0 or any(b <= a for a, b in zip(xs[:-1], xs[1:])):
        raise ValueError("group edges must start at the hydrogen edge and increase")
    G = len(edges_ev)
    sE, sG, frac, t = (np.zeros(G) for _ in range(4))
    e3_all = _bb(lambda x: x**3, x0, math.inf)
    for g in range(G):
        a, b = xs[g], xs[g + 1]
        e3 = _bb(lambda x: x**3, a, b)
        sE[g] = K.SIGMA0 * x0**3 * _bb(lambda x: 1.0, a, b) / e3
        sG[g] = K.SIGMA0 * x0**3 * _bb(lambda x: 1.0 / x, a, b) / (kT * e3)
        frac[g] = e3 / e3_all
        t[g] = a * (a**3 * math.exp(-a) / -math.expm1(-a)) / e3
    e2_all = _bb(lambda x: x**2, x0, math.inf)
    return dict(sigma_E=sE, sigma_G=sG, frac=frac, t=t, eps_src=kT * e3_all / e2_all)


# ----------------------------------------------------------------------------- step


@dataclass
class MGStep:
    """One implicit step with G radiation groups: the grey Step's data (its sigma_E, sigma_G
    unused) plus the group constants and the groups' starting energies E_n[g]."""
    base: M.Step
    sigma_E: np.ndarray
    sigma_G: np.ndarray
    frac: np.ndarray
    t: np.ndarray
    E_n: np.ndarray                     # [G, z, y, x]

    def __getattr__(self, name):        # grid, gas and time data of the base step
        return getattr(self.base, name)

    @property
    def G(self):
        return len(self.sigma_E)

    def group(self, g):
        """The grey Step of group g: its cross sections, emission share and starting energy."""
        return dataclasses.replace(self.base, sigma_E=float(self.sigma_E[g]), sigma_G=float(self.sigma_G[g]),
                                   eps_src=float(self.frac[g]) * self.base.eps_src, E_n=self.E_n[g])


def make_mg_step(st, consts, E_n=None):
    """MGStep from a grey Step and ``group_constants`` output; E_n per group defaults to the
    step's grey E^n split by the emission shares (the fixed spectrum)."""
    if E_n is None:
        E_n = consts["frac"][:, None, None, None] * st.E_n[None]
    base = dataclasses.replace(st, eps_src=consts.get("eps_src", st.eps_src))
    return MGStep(base=base, sigma_E=np.asarray(consts["sigma_E"], float), sigma_G=np.asarray(consts["sigma_G"], float),
                  frac=np.asarray(consts["frac"], float), t=np.asarray(consts["t"], float), E_n=np.asarray(E_n, float))


# ---------------------------------------------------------------------- residual


def redshift_transfer(st, E):
    """(adot/a) [t_{g+1} E_{g+1} - t_g E_g (g > 0)] per group: the edge fluxes between groups
    (the -(adot/a) E_g part is in each group's grey bracket)."""
    h = st.adot / st.a
    out = np.zeros(np.shape(E), dtype=np.result_type(E, float))
    for g in range(st.G):
        if g + 1 < st.G:
            out[g] = out[g] + h * st.t[g + 1] * E[g + 1]
        if g > 0:
            out[g] = out[g] - h * st.t[g] * E[g]
    return out


def group_rhs(st, E, nHI, freeze=False):
    """The bracket of Eq. radiation_residual for every group, with the redshift transfer."""
    out = [M.radiation_rhs(st.group(g), E[g], nHI, M.emissivity(st.group(g)), freeze) for g in range(st.G)]
    return np.stack(out) + redshift_transfer(st, E)


def explicit_part(st):
    """b_E,g = E_g^n + dt (1 - theta) [bracket of group g at time n]."""
    return st.E_n + st.dt * (1.0 - st.theta) * group_rhs(st, st.E_n, st.nHI_n)


def local_solutions(st, e_c, nHI, E):
    """(S_e, S_n) with the groups' photo-ionisation and heating summed."""
    a3 = st.a**3
    nH = st.n_H
    Gam = 0.0
    heat = 0.0
    for g in range(st.G):
        Ebar = M.spos(st.theta * E[g] + (1.0 - st.theta) * st.E_n[g], st.E_min)
        Gam = Gam + K.C_LIGHT * st.sigma_G[g] * Ebar / a3
        heat = heat + nHI * K.C_LIGHT * Ebar * (st.sigma_E[g] - K.HNU0 * st.sigma_G[g]) / (a3 * st.rho_b)
    T = M.temperature(st.base, e_c, nHI)
    A = rates.alpha_B(T, st.recomb) * st.clump / a3
    Sn = M.riccati_Sn(st.nHI_n, nH, A, Gam, st.dt)
    if st.isothermal:
        return None, Sn
    cool = 0.0
    if st.cooling:
        nHII = nH - nHI
        cool = a3 * rates.cooling_rate(T, nHII / a3, nHI / a3, nHII / a3, st.a) / st.rho_b
    Se = (heat - cool) * st.dt * M.phi1(2.0 * (st.adot / st.a) * st.dt)
    return Se, Sn


def residual(st, U, bE=None, freeze=False):
    """f(U) = (f_e, f_n, f_E1, ..., f_EG) for U = (e_c, n_HI, E_1, ..., E_G)."""
    e_c, nHI, E = U[0], U[1], U[2:]
    if bE is None:
        bE = explicit_part(st)
    Se, Sn = local_solutions(st, e_c, nHI, E)
    f_e = e_c if st.isothermal else e_c - Se
    f_n = nHI - Sn
    f_E = E - bE - st.dt * st.theta * group_rhs(st, E, nHI, freeze)
    return np.concatenate([np.stack([f_e, f_n]), f_E])


def weights(st, U):
    """Norm scales: the grey model's for (e_c, n_HI), and each group's E like the grey E
    (floor from the group's own starting energy and emission)."""
    e_c, nHI = np.real(U[0]), np.real(U[1])
    E = np.real(U[2:])
    w = [1.0 / np.maximum(M.internal_energy_h(st.base), M.E_FLOOR_INT()) + 0 * e_c, 1.0 / st.n_H + 0 * e_c]
    for g in range(st.G):
        sg = st.group(g)
        w.append(1.0 / np.maximum(np.maximum(np.abs(E[g]), st.E_n[g]), M.weight_floor_E(sg)))
    return np.stack(w)


def _scales(st, U):
    e_c, nHI = np.real(U[0]), np.real(U[1])
    out = [np.maximum(np.abs(e_c), M.E_FLOOR_INT()), st.n_H + 0 * e_c]
    out += [np.maximum(np.abs(np.real(U[2 + g])), st.E_min) for g in range(st.G)]
    return np.stack(out).reshape(2 + st.G, -1)


def jacobian(st, U, bE=None, freeze=False):
    """Sparse (G+2)N x (G+2)N Jacobian by coloured complex steps (oracle.newton.jacobian)."""
    if bE is None:
        bE = explicit_part(st)
    return N.jacobian(st, U, bE, freeze, residual=residual, scales=_scales)


def initial_iterate(st):
    """(0, n_HI^n, E_g^n + dt 4 pi eta_g)."""
    E0 = np.stack([st.E_n[g] + st.dt * M.emissivity(st.group(g)) for g in range(st.G)])
    return np.concatenate([np.stack([np.zeros(st.shape), st.nHI_n.copy()]), E0])


def local_solve(st, U, tol=1e-14, maxit=60):
    """The cell-local equations solved for (e_c, n_HI) at fixed E_g (isothermal: n_HI = S_n;
    otherwise the damped 2x2 complex-step Newton iteration of oracle.newton.local_solve)."""
    U = np.array(U, float)
    E = U[2:]
    if st.isothermal:
        U[0] = 0.0
        U[1] = np.real(local_solutions(st, U[0], U[1], E)[1])
        return U
    h = 1e-30
    se = np.maximum(M.internal_energy_h(st.base), M.E_FLOOR_INT())
    sn = st.n_H
    eint_h = M.internal_energy_h(st.base)

    def lres(ec, n):
        Se, Sn = local_solutions(st, ec, n, E)
        return ec - Se, n - Sn

    e_c, nHI = U[0], np.clip(U[1], 1e-300, st.n_H)
    fe, fn = (np.real(x) for x in lres(e_c, nHI))
    r = np.maximum(np.abs(fe) / se, np.abs(fn) / sn)
    for _ in range(maxit):
        active = r > tol
        if not np.any(active):
            break
        fe1, fn1 = lres(e_c + 1j * h * se, nHI)
        fe2, fn2 = lres(e_c, nHI + 1j * h * sn)
        a11, a21 = np.imag(fe1) / (h * se), np.imag(fn1) / (h * se)
        a12, a22 = np.imag(fe2) / (h * sn), np.imag(fn2) / (h * sn)
        det = a11 * a22 - a12 * a21
        de = np.where(active, -(a22 * fe - a12 * fn) / det, 0.0)
        dn = np.where(active, -(-a21 * fe + a11 * fn) / det, 0.0)
        lam = np.ones_like(e_c)
        todo = active.copy()
        for _ in range(40):
            ec_t = np.maximum(e_c + lam * de, -0.999 * eint_h)
            n_t = np.clip(nHI + lam * dn, 1e-300, st.n_H)
            fe_t, fn_t = (np.real(x) for x in lres(ec_t, n_t))
            r_t = np.maximum(np.abs(fe_t) / se, np.abs(fn_t) / sn)
            ok = todo & (r_t < r)
            e_c, nHI = np.where(ok, ec_t, e_c), np.where(ok, n_t, nHI)
            fe, fn, r = np.where(ok, fe_t, fe), np.where(ok, fn_t, fn), np.where(ok, r_t, r)
            todo &= ~ok
            if not np.any(todo):
                break
            lam = np.where(todo, 0.5 * lam, lam)
    U[0], U[1] = e_c, nHI
    return U


def solve_step(st, tol=1e-11, maxit=60, U0=None):
    """The root of the multigroup residual by the grey oracle's method (oracle.newton.solve_step):
    full-system Newton with complex-step Jacobian and sparse direct solves, the cell-local
    unknowns re-solved exactly after each update of the group energies, halving line search on
    the RMS norm of the component-scaled residual.  Returns (U, info)."""
    bE = explicit_part(st)
    U = initial_iterate(st) if U0 is None else np.array(U0, float)
    U = local_solve(st, U)
    hist = []
    for k in range(maxit + 1):
        f = residual(st, U, bE)
        w = weights(st, U)
        nrm = M.rms_norm(w, f)
        hist.append(nrm)
        if not np.isfinite(nrm):
            raise FloatingPointError("oracle residual is not finite")
        if nrm <= tol:
            return U, dict(iters=k, hist=hist)
        if k == maxit:
            break
        J = jacobian(st, U, bE)
        S = N.linear_solve(J, -f.ravel()).reshape(U.shape)
        lam = 1.0
        for _ in range(40):
            Ut = U.copy()
            Ut[2:] = U[2:] + lam * S[2:]
            Ut = local_solve(st, Ut)
            nt = M.rms_norm(w, residual(st, Ut, bE))
            if nt <= (1.0 - 1e-4 * lam) * nrm and nt < nrm:
                break
            lam *= 0.5
        else:
            if nrm <= 1e-9:
                return U, dict(iters=k, hist=hist, floor=True)
            raise RuntimeError("oracle line search failed")
        U = Ut
    raise RuntimeError(f"oracle Newton did not converge: {hist[-5:]}")
