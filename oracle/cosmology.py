"""Expansion histories and I-front closed forms (oracle; test infrastructure only).

* a(t) and da/dt for flat LCDM: a = (Om/OL)^{1/3} sinh^{2/3}(1.5 sqrt(OL) H0 t)
  (the Friedmann equation with matter and Lambda, Sec. "Physical Model").
* a(t) for the Lambda-free models of Table 1: q0 = 0.5 (Einstein-de Sitter,
  a ~ t^{2/3}) and q0 = 0.05 (open, Omega_m = 0.1, the parametric cycloid
  solution a = Om/(2(1-Om)) (cosh eta - 1), H0 t = Om/(2(1-Om)^{3/2}) (sinh eta - eta)).
* Sec. "Verification tests": the Stromgren radius (Eq. SG-stromgren_radius) and the
  Shapiro-Giroux I-front radius (Eqs. SG-solution, SG-tau, SG-F) by quadrature.
  r_I there is the comoving radius in units of proper length at z0.
* The I-front equation these closed forms solve, for any a(t): the comoving ionised
  volume obeys n_c dV_c/dt = Ndot - alpha_B n_c^2 V_c / a^3 (ionisations at the
  front balance photons not used up by recombinations; n_c comoving density),
  integrated with an adaptive ODE solver.

Pinned in tests: LCDM a(t) against direct integration of the Friedmann equation,
the ODE against the SG closed form for q0 = 0.5 and 0.05, and the static limit
r = R_s (1 - e^{-t/t_rec})^{1/3}.
"""
import math

import numpy as np
from scipy import integrate, optimize

from . import constants as K


class FlatLCDM:
    """Flat matter + Lambda expansion (the Friedmann equation of Sec. "Physical Model" with
    Omega_m + Omega_L = 1); times in seconds since the big bang."""

    def __init__(self, Omega_m=0.3, Omega_L=0.7, h=0.7, **_):
        self.Om, self.OL, self.h = Omega_m, Omega_L, h
        self.H0 = h * K.H100

    def a(self, t):
        """Scale factor: (Om/OL)^{1/3} sinh^{2/3}(1.5 sqrt(OL) H0 t)."""
        return (self.Om / self.OL) ** (1 / 3) * np.sinh(1.5 * math.sqrt(self.OL) * self.H0 * t) ** (2 / 3)

    def adot(self, t):
        """da/dt = H0 a sqrt(Om / a^3 + OL)."""
        a = self.a(t)
        return self.H0 * a * np.sqrt(self.Om / a**3 + self.OL)

    def t_of_a(self, a):
        """Inverse of a(t)."""
        return 2.0 / (3.0 * math.sqrt(self.OL) * self.H0) * np.arcsinh(math.sqrt(self.OL / self.Om) * a**1.5)

    def t_of_z(self, z):
        """Time at redshift z (a = 1 / (1 + z))."""
        return self.t_of_a(1.0 / (1.0 + z))


class OpenNoLambda:
    """Lambda = 0 models of Table 1: q0 = Omega_m / 2."""

    def __init__(self, q0, H0):
        self.q0, self.H0 = q0, H0
        self.Om = 2.0 * q0

    def adot(self, t):
        """da/dt = H0 a sqrt(Om / a^3 + (1 - Om) / a^2) (curvature instead of Lambda)."""
        a = self.a(t)
        return self.H0 * a * math.sqrt(self.Om / a**3 + (1 - self.Om) / a**2)

    def a(self, t):
        """Scale factor: (1.5 H0 t)^{2/3} for Om = 1, else the parametric cycloid in eta."""
        if abs(self.Om - 1.0) < 1e-12:
            return (1.5 * self.H0 * t) ** (2.0 / 3.0)
        Om = self.Om
        f = lambda eta: Om / (2 * (1 - Om) ** 1.5) * (math.sinh(eta) - eta) - self.H0 * t
        eta = optimize.brentq(f, 1e-12, 50.0, xtol=1e-15, rtol=1e-15)
        return Om / (2 * (1 - Om)) * (math.cosh(eta) - 1)

    def t_of_z(self, z):
        """Time at redshift z (a = 1 / (1 + z))."""
        return self.t_of_a(1.0 / (1.0 + z))

    def t_of_a(self, a):
        """Inverse of a(t): the cycloid's eta from a, then t(eta)."""
        if abs(self.Om - 1.0) < 1e-12:
            return 2.0 / (3.0 * self.H0) * a**1.5
        Om = self.Om
        eta = math.acosh(1 + 2 * (1 - Om) * a / Om)
        return Om / (2 * (1 - Om) ** 1.5) * (math.sinh(eta) - eta) / self.H0


def stromgren_radius(ndot, alpha, nH):
    """Eq. SG-stromgren_radius: r_S = (3 Ndot / (4 pi alpha n_H^2))^{1/3} (proper)."""
    return (3.0 * ndot / (4.0 * math.pi * alpha * nH**2)) ** (1.0 / 3.0)


def static_ifront(t, ndot, alpha, nH):
    """I-front radius in a static uniform medium: R_s (1 - exp(-t/t_rec))^{1/3}."""
    return stromgren_radius(ndot, alpha, nH) * (1.0 - math.exp(-t * alpha * nH)) ** (1.0 / 3.0)


def sg_ifront(abar, q0, z0, H0, ndot, alpha, nH0):
    """Eqs. SG-solution / SG-tau / SG-F: r_I at scale factor abar = a/a(z0) >= 1.

    Returns the comoving I-front radius in units of proper length at z0 (multiply by
    abar for the proper radius).  nH0 is the proper hydrogen density at z0.
    """
    lam = alpha * nH0 / H0 / (1.0 + z0)

    def bracket(a):       # the square-root argument of Eq. SG-F
        return 1.0 - 2.0 * q0 + 2.0 * q0 * (1.0 + z0) / a

    def F(a):             # Eq. SG-F
        return (2.0 - 4.0 * q0 - 2.0 * q0 * (1.0 + z0) / a) * math.sqrt(bracket(a))

    def tau(a):           # Eq. SG-tau
        return lam / (6.0 * q0**2 * (1.0 + z0) ** 2) * (F(a) - F(1.0))

    val, _ = integrate.quad(lambda a: math.exp(tau(a)) / math.sqrt(bracket(a)), 1.0, abar,
                            epsabs=0.0, epsrel=1e-12, limit=200)
    rS0 = stromgren_radius(ndot, alpha, nH0)
    return rS0 * (lam * math.exp(-tau(abar)) * val) ** (1.0 / 3.0)


def ifront_ode(t0, t1, a_of_t, ndot, alpha, n_comoving, V0=0.0, rtol=1e-11):
    """Integrate n_c dV_c/dt = Ndot - alpha n_c^2 V_c / a^3 from t0 to t1; returns V_c(t1) [cm^3]."""
    def rhs(t, V):        # dV_c/dt
        return [ndot / n_comoving - alpha * n_comoving * V[0] / a_of_t(t) ** 3]
    sol = integrate.solve_ivp(rhs, (t0, t1), [V0], method="DOP853", rtol=rtol, atol=1e-30 * 0 + 1e-3)
    return float(sol.y[0, -1])
