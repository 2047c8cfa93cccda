"""The package's host-side unit code (paper_0908_2654_gb300/units.py) against the oracle's
independent versions and the definitions of Eqs. units and scalings.  It covers the derived
units, the specific energy of gas at a temperature (hydrogen and hydrogen + helium) and the
temperature inverse.  No GPU is needed."""
import numpy as np
import pytest

from oracle import constants as K
from oracle import driver
from oracle import helium as H
from paper_0908_2654_gb300 import units as U


def _gas(seed, n=500):
    rng = np.random.default_rng(seed)
    rho = 10 ** rng.uniform(-30, -24, n)
    xHI = 10 ** rng.uniform(-6, 0, n)
    T = 10 ** rng.uniform(1, 8, n)
    v = tuple(rng.normal(0, 3e6, n) for _ in range(3))
    return rho, xHI, T, v


def test_derived_units_follow_their_definitions():
    u = U.Units.for_grid(3.1e21, 2.4e-31)
    assert u.u_x == 3.1e21 and u.u_t == U.MYR
    assert u.u_g == pytest.approx(2.4e-31 * 3.1e21**3, rel=1e-15)
    assert u.u_d == pytest.approx(2.4e-31, rel=1e-15)            # density unit = mean density
    assert u.u_v == pytest.approx(3.1e21 / U.MYR, rel=1e-15)
    assert u.u_E == pytest.approx(u.u_d * u.u_v**2, rel=1e-15)
    assert u.u_n == pytest.approx(u.u_d / K.M_H, rel=1e-15)


def test_constants_agree_with_the_oracle():
    assert U.K_B == K.K_BOLTZ and U.M_H == K.M_H and U.GAMMA == K.GAMMA
    assert U.MYR == pytest.approx(K.MYR, rel=1e-15)


def test_specific_energy_hydrogen_matches_oracle_and_inverts():
    rho, xHI, T, v = _gas(1)
    nHI = xHI * rho / K.M_H
    e = U.specific_energy(T, rho, nHI, v)
    np.testing.assert_allclose(e, driver.energy_from_temperature(T, rho, nHI, v), rtol=1e-14)
    np.testing.assert_allclose(U.temperature(e, rho, nHI, v), T, rtol=1e-8)


def test_specific_energy_helium_matches_oracle():
    rho, xHI, T, v = _gas(2)
    Y = 0.24
    rng = np.random.default_rng(3)
    nHe = Y * rho / (4.0 * K.M_H)
    f1 = rng.uniform(0, 1, rho.size)
    nHeI, nHeII = f1 * nHe, (1 - f1) * rng.uniform(0, 1, rho.size) * nHe
    nHI = xHI * (1 - Y) * rho / K.M_H
    e = U.specific_energy(T, rho, nHI, v, helium=(Y, nHeI, nHeII))
    np.testing.assert_allclose(e, H.energy_from_temperature(T, rho, nHI, nHeI, nHeII, Y, v), rtol=1e-14)
    # Y = 0 with no helium reduces to the hydrogen-only count
    e0 = U.specific_energy(T, rho, xHI * rho / K.M_H, v, helium=(0.0, 0 * rho, 0 * rho))
    np.testing.assert_allclose(e0, U.specific_energy(T, rho, xHI * rho / K.M_H, v), rtol=1e-14)
