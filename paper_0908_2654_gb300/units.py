"""Unit normalisation of the paper (Eqs. units, scalings, proper_vars) for the Python side.

x~ = x/u_x, t~ = t/u_t, rho~ = rho/u_d, e~ = e/u_v^2, E~ = E/u_E, n~ = n/u_n with
u_d = u_g/u_x^3, u_v = u_x/u_t, u_E = u_d u_v^2 and u_n = u_d/m_H (hydrogen-only gas,
so n~_H = rho~).  Also the equation of state used to turn a temperature into the
specific total gas energy e_h (Eqs. eos, temperature: T = (gamma-1) e_int rho /(k_B n_tot)).
"""
from dataclasses import dataclass

import numpy as np

K_B = 1.380649e-16
M_H = 1.6735575e-24
GAMMA = 5.0 / 3.0
MYR = 3.15576e13


@dataclass
class Units:
    """The three base units and the derived ones of Eqs. units and scalings."""

    u_x: float   # cm
    u_t: float   # s
    u_g: float   # g

    @property
    def u_d(self):
        """Density unit u_g / u_x^3 [g/cm^3]."""
        return self.u_g / self.u_x**3

    @property
    def u_v(self):
        """Velocity unit u_x / u_t [cm/s]."""
        return self.u_x / self.u_t

    @property
    def u_E(self):
        """Radiation energy density unit u_d u_v^2 [erg/cm^3]."""
        return self.u_d * self.u_v**2

    @property
    def u_n(self):
        """Number density unit u_d / m_H [1/cm^3]."""
        return self.u_d / M_H

    @staticmethod
    def for_grid(dx_cm, rho_mean, u_t=MYR):
        """Length unit = cell width, time unit = 1 Myr, density unit = mean baryon density."""
        return Units(u_x=dx_cm, u_t=u_t, u_g=rho_mean * dx_cm**3)


def specific_energy(T, rho_b, nHI, v, helium=None):
    """e_h [erg/g] of gas at temperature T with neutral density nHI moving with v: hydrogen
    only (X = 1), or with helium = (Y, n_HeI, n_HeII), where the particle count is
    n_H + n_He + n_e with n_H = (1 - Y) rho / m_H, n_He = Y rho / (4 m_H)."""
    if helium is None:
        n_tot = 2.0 * rho_b / M_H - nHI
    else:
        Y, nHeI, nHeII = helium
        nH, nHe = (1.0 - Y) * rho_b / M_H, 0.25 * Y * rho_b / M_H
        n_tot = nH + nHe + (nH - nHI) + nHeII + 2.0 * (nHe - nHeI - nHeII)
    e_int = K_B * T * n_tot / ((GAMMA - 1.0) * rho_b)
    return e_int + 0.5 * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2)


def temperature(e_total, rho_b, nHI, v):
    """Temperature [K] of hydrogen-only gas (X = 1, n_tot = 2 n_H - n_HI) from its specific
    total energy e_total [erg/g] and velocity v."""
    nH = rho_b / M_H
    e_int = e_total - 0.5 * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2)
    return (GAMMA - 1.0) * e_int * rho_b / (K_B * (2.0 * nH - nHI))
