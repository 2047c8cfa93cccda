"""Pins of the oracle's rate coefficients and cooling functions (oracle/rates.py,
oracle/constants.py) to facts of atomic physics that hold independently of the fits.

The paper names its rate sources (Sec. "Physical Model") but prints no rate value except
the case-B coefficient at 1e4 K. The fits are checked here against:

* textbook case-B coefficients of hydrogen;
* the hydrogenic scaling of the Coulomb problem to charge Z = 2 (HeII), namely
  alpha_Z(T) = Z alpha_1(T / Z^2), its cooling Z^3 Lambda_1(T / Z^2),
  sigma_Z(nu) = sigma_1(nu / Z^2) / Z^2 and thresholds Z^2 I_H;
* the bound on the energy a recombination removes from the gas;
* the Kramers bremsstrahlung coefficient from fundamental constants;
* the excitation energies in the Boltzmann factors;
* the published Compton coefficient;
* measured ionisation energies.

A plausible slip in a fit (a prefactor, a dropped T, an exponent or a sign) fails at
least one of these checks.
"""
import math

import numpy as np
import pytest

from oracle import constants as K
from oracle import rates as R

KB_EV = 8.617333262e-5           # Boltzmann constant [eV/K] (exact SI value)
E_ESU = 1.602176634e-19 * 2.99792458e9   # elementary charge [esu] (exact SI value times c/10)
# ionisation energies [eV] (NIST Atomic Spectra Database): H, He, He+
I_H, I_HEI, I_HEII = 13.598434, 24.587389, 54.417765


def _coef(T, a=1.0):
    return R.cooling_coefficients(np.asarray(T, float), a)


def _log_slope_in_inverse_T(f, T1, T2):
    """-d ln f / d(1/T) by a secant between T1 and T2: the energy / k of a Boltzmann factor."""
    return -(math.log(f(T2)) - math.log(f(T1))) / (1.0 / T2 - 1.0 / T1)


def test_case_b_hydrogen_matches_textbook_values():
    """Case-B recombination coefficients of hydrogen at 5000, 10000 and 20000 K:
    4.54e-13, 2.59e-13 and 1.43e-13 cm^3/s. These are the values of Osterbrock,
    Astrophysics of Gaseous Nebulae (1989), Table 2.1. The Hui & Gnedin fit claims
    better than 1 % accuracy."""
    T = np.array([5000.0, 1e4, 2e4])
    np.testing.assert_allclose(R.alpha_B(T, "hg97"), [4.54e-13, 2.59e-13, 1.43e-13], rtol=1e-2)


def test_ionisation_temperatures_of_the_fits():
    """The fits' lambda = 2 T_ion / T uses T_ion = I / k for H, He and He+."""
    for T_ion, I in ((R.T_HI, I_H), (R.T_HEI, I_HEI), (R.T_HEII, I_HEII)):
        assert T_ion == pytest.approx(I / KB_EV, rel=1e-4)


def test_heiii_recombination_is_hydrogenic():
    """For a hydrogenic ion, alpha_Z(T) = Z alpha_1(T / Z^2). Energies in the Coulomb problem
    scale as Z^2, and the cross sections scale so that the rate coefficient gains one factor
    of Z. The fits' ionisation temperatures differ from Z^2 only through the reduced
    mass: T_HeII / T_HI = 4.0018."""
    T = np.logspace(1, 8, 57)
    np.testing.assert_allclose(R.alpha_HeIII_B(T), 2.0 * R.alpha_B(T / 4.0, "hg97"), rtol=1e-3)


def test_recombination_cooling_energy_per_recombination():
    """The energy a recombination removes is beta / alpha = <sigma v E> / <sigma v>. The
    capture rate sigma v falls with electron energy, so this weighted mean lies below the
    Maxwellian mean of 3/2 kT. The HeIII coefficient follows the hydrogenic scaling
    beta_Z(T) = Z^3 beta_1(T / Z^2): a factor Z^2 on the energy and Z on the rate. Equivalently,
    the energy per recombination in units of kT is the same function of T / Z^2."""
    T = np.logspace(1, 8, 57)
    c, c4 = _coef(T), _coef(T / 4.0)
    kT = K.K_BOLTZ * T
    for beta, alpha in ((c["rec_HII"], R.alpha_B(T, "hg97")), (c["rec_HeIII"], R.alpha_HeIII_B(T)),
                        (c["rec_HeII"], R.alpha_HeII_B(T))):
        ratio = beta / (kT * alpha)
        assert np.all(ratio > 0.0) and np.all(ratio < 1.5), ratio
    np.testing.assert_allclose(c["rec_HeIII"], 8.0 * c4["rec_HII"], rtol=2e-3)


def test_bremsstrahlung_from_fundamental_constants():
    """Frequency-integrated Kramers free-free emission of a Maxwellian plasma (Rybicki &
    Lightman 1979, Sec. 5.2):
    (2^5 pi e^6 / (3 h m_e c^3)) (2 pi k T / (3 m_e))^{1/2} Z^2 n_e n_i g_B.
    The thermally averaged Gaunt factor g_B lies between 1.1 and 1.5. It varies slowly, so
    the coefficient goes as T^{1/2}. Ions of charge Z weigh Z^2."""
    C = (2**5 * math.pi * E_ESU**6 / (3.0 * K.H_PLANCK * K.M_E * K.C_LIGHT**3)
         * math.sqrt(2.0 * math.pi * K.K_BOLTZ / (3.0 * K.M_E)))
    T = np.logspace(4, 9, 41)
    g = _coef(T)["ff"] / (C * np.sqrt(T))
    assert np.all(g > 1.1 * (1 - 5e-3)) and np.all(g < 1.5), g
    slope = np.diff(np.log(_coef(T)["ff"])) / np.diff(np.log(T))
    assert np.all(np.abs(slope - 0.5) < 0.07), slope
    # assembled cooling: HeIII's bremsstrahlung is Z^2 = 4 times that of HII
    one, zero = np.ones_like(T), np.zeros_like(T)
    c = _coef(T)
    he3 = R.cooling_rate_he(T, one, zero, zero, zero, one, 1.0) - c["comp"] - c["rec_HeIII"]
    np.testing.assert_allclose(he3, 4.0 * c["ff"], rtol=1e-12)


def test_collisional_excitation_costs_the_lyman_alpha_energy():
    """Collisional excitation to n = 2 is followed by a Lyman-alpha photon. Its rate carries
    the Boltzmann factor exp(-E_12 / kT), with E_12 = (3/4) Z^2 Ry: 10.2 eV for H and
    40.8 eV for He+ (reduced-mass Rydbergs). At low T the log-slope of the rate in 1/T gives
    E_12 / k. The slowly varying prefactors shift it by less than 0.3 %."""
    E_H = 0.75 * I_H / KB_EV
    E_He = 0.75 * I_HEII / KB_EV
    sH = _log_slope_in_inverse_T(lambda t: float(_coef(t)["ce_HI"]), 1000.0, 1100.0)
    sHe = _log_slope_in_inverse_T(lambda t: float(_coef(t)["ce_HeII"]), 1000.0, 1100.0)
    assert sH == pytest.approx(E_H, rel=3e-3)
    assert sHe == pytest.approx(E_He, rel=3e-3)


def test_dielectronic_recombination_goes_through_the_heii_resonance():
    """Dielectronic recombination of He+ runs through its 2p level. The Boltzmann factor's
    energy and the energy radiated per recombination are both close to the 40.8 eV
    resonance energy."""
    E_res = 0.75 * I_HEII
    slope = _log_slope_in_inverse_T(lambda t: float(R.alpha_di(t)), 1000.0, 1100.0)
    assert slope * KB_EV == pytest.approx(E_res, rel=2e-2)
    T = np.logspace(3, 8, 21)
    np.testing.assert_allclose(_coef(T)["di_HeII"] / R.alpha_di(T) / K.EV, E_res, rtol=1e-2)


def test_compton_cooling_matches_published_coefficient():
    """Compton cooling off the CMB is 5.41e-36 n_e T (1+z)^4 erg/cm^3/s for T >> T_cmb with
    T_cmb0 = 2.7 K (Cen 1992). It scales as T_cmb^4 (T - T_cmb): zero at T = T_cmb and
    heating below it."""
    for a in (1.0, 0.2, 1.0 / 11.0):
        T_cmb = K.T_CMB0 / a
        T = np.array([1e4, 1e6])
        ref = 5.41e-36 * (K.T_CMB0 / 2.7) ** 4 * a**-4 * (T - T_cmb)
        np.testing.assert_allclose(_coef(T, a)["comp"], ref, rtol=5e-3)
        assert _coef(np.array([T_cmb]), a)["comp"][0] == 0.0
        assert _coef(np.array([0.5 * T_cmb]), a)["comp"][0] < 0.0


def test_heii_photoionisation_is_hydrogenic():
    """He+ is hydrogenic with Z = 2. Its threshold is Z^2 times hydrogen's 13.6 eV. The
    threshold cross section of the nu^-3 law is sigma_0 / Z^2, since
    sigma_Z(nu) = sigma_1(nu / Z^2) / Z^2. The HeI threshold is helium's first ionisation
    energy."""
    assert K.HNU_HEII == pytest.approx(4.0 * K.HNU0, rel=1e-3)
    assert K.SIGMA_HEII == pytest.approx(K.SIGMA0 / 4.0, rel=1e-2)
    assert K.HNU_HEI / K.EV == pytest.approx(I_HEI, rel=1e-3)
    assert K.HNU_HEII / K.EV == pytest.approx(I_HEII, rel=1e-3)
