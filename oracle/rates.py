"""Rate coefficients for hydrogen and hydrogen + helium gas (oracle; test infrastructure only).

Sec. "Physical Model": G, Lambda, alpha_ij and Gamma^ph are functions of T, E and
the ionisation state, with formulas the paper cites but does not print.  Readings
used (identical in the CUDA library, written there independently):

* alpha(T): the constant alpha_B = 2.59e-13 cm^3/s quoted in the verification
  section (mode "const"), or the Hui & Gnedin (1997) case-B fit (mode "hg97").
* Photo-heating per unit volume: n_HI c E (sigma_E - h nu_0 sigma_G)   (grey
  averages from ``spectrum``).
* Cooling per unit volume: case-B recombination cooling (Hui & Gnedin 1997),
  collisional excitation of HI and bremsstrahlung (Cen 1992), Compton cooling
  off the CMB (4 k_B sigma_T a_rad T_cmb^4 (T - T_cmb) n_e / (m_e c)).
  Collisional ionisation is not included.

Pins: alpha_hg97(1e4 K) reproduces the paper's 2.59e-13 to 0.1 %.  The paper prints
no other rate value; the fits are pinned instead to facts of atomic physics that do not
depend on them (tests/test_oracle_rate_pins.py): textbook case-B coefficients, the
hydrogenic scaling of recombination and its cooling to Z = 2, the bound of 3/2 kT on the
mean energy a recombination removes, the Kramers-Gaunt bremsstrahlung coefficient from
fundamental constants, the Lyman-alpha energies in the excitation exponents, Cen's Compton
coefficient.  Parity unpinned: the shapes of the Gaunt factor, of the excitation prefactors
and of the HeI recombination fit.

All functions accept complex arguments (the oracle Jacobian uses complex steps).
"""
import numpy as np

from . import constants as K

T_HI = 157807.0   # K, hydrogen ionisation temperature used by the Hui & Gnedin fits
T_FLOOR = 1.0     # K, rates are evaluated at max(T, T_FLOOR)


def _cmax(x, c):
    """max(x, c) compared on real parts (complex-step safe)."""
    return np.where(np.real(x) >= c, x, c)


def alpha_B(T, mode):
    """Case-B recombination coefficient [cm^3/s]."""
    if mode == "const":
        return K.ALPHA_B_PAPER + 0.0 * T
    T = _cmax(T, T_FLOOR)
    lam = 2.0 * T_HI / T
    return 2.753e-14 * lam**1.5 / (1.0 + (lam / 2.740) ** 0.407) ** 2.242


# ------------------------------------------------------------------------ helium
# Readings for hydrogen + helium gas (Sec. "Physical Model", Eq. electron_density; the paper
# cites Cen (1992), Hui & Gnedin (1997) and Abel et al. (1997) for the rates):
#   case-B radiative recombination HeII -> HeI and HeIII -> HeII (Hui & Gnedin 1997), the
#   dielectronic recombination of HeII (Aldrovandi & Pequignot form used by Cen 1992), their
#   recombination cooling, collisional excitation of HeII (Cen 1992), bremsstrahlung with
#   Z^2 = 4 for HeIII.  Collisional ionisation and HeI collisional excitation are left out,
#   like hydrogen's collisional ionisation.
T_HEI = 285335.0    # K, HeI ionisation temperature of the Hui & Gnedin fits
T_HEII = 631515.0   # K, HeII


def alpha_HeII_B(T):
    """HeII -> HeI case-B radiative recombination [cm^3/s]."""
    T = _cmax(T, T_FLOOR)
    return 1.26e-14 * (2.0 * T_HEI / T) ** 0.750


def alpha_HeIII_B(T):
    """HeIII -> HeII case-B recombination [cm^3/s] (hydrogenic, Z = 2)."""
    T = _cmax(T, T_FLOOR)
    lam = 2.0 * T_HEII / T
    return 5.506e-14 * lam**1.5 / (1.0 + (lam / 2.740) ** 0.407) ** 2.242


def alpha_di(T):
    """HeII dielectronic recombination [cm^3/s]."""
    T = _cmax(T, T_FLOOR)
    return 1.90e-3 * T**-1.5 * np.exp(-470000.0 / T) * (1.0 + 0.3 * np.exp(-94000.0 / T))


def cooling_coefficients(T, a):
    """Cooling rate coefficients by process, each per product of the proper densities named
    [erg cm^3 s^-1] (Compton per n_e [erg s^-1]):

    rec_HII   case-B recombination cooling, per n_e n_HII (Hui & Gnedin 1997)
    ce_HI     collisional excitation of HI, per n_e n_HI (Cen 1992)
    ff        bremsstrahlung of a Z = 1 ion, per n_e n_i (Z^2 n_i for charge Z; Gaunt factor
              of Cen 1992)
    comp      Compton scattering off the CMB at T_cmb = T_cmb0 / a, per n_e
    rec_HeII  HeII -> HeI recombination cooling, kT alpha_HeII, per n_e n_HeII
    rec_HeIII HeIII -> HeII case-B recombination cooling, per n_e n_HeIII: the hydrogen fit
              under the hydrogenic scaling Lambda_Z(T) = Z^3 Lambda_H(T / Z^2), Z = 2, i.e.
              Z times hydrogen's coefficient at the same lambda = 2 T_ion / T (as for alpha)
    di_HeII   dielectronic recombination cooling (the HeII 2p -> 1s energy per
              recombination), per n_e n_HeII
    ce_HeII   collisional excitation of HeII, per n_e n_HeII (Cen 1992)
    """
    T = _cmax(T, T_FLOOR)
    lam = 2.0 * T_HI / T
    lam3 = 2.0 * T_HEII / T
    T_cmb = K.T_CMB0 / a
    return dict(
        rec_HII=3.435e-30 * T * lam**1.970 / (1.0 + (lam / 2.250) ** 0.376) ** 3.720,
        ce_HI=7.5e-19 * np.exp(-118348.0 / T) / (1.0 + np.sqrt(T / 1e5)),
        ff=1.42e-27 * (1.1 + 0.34 * np.exp(-((5.5 - np.log10(T)) ** 2) / 3.0)) * np.sqrt(T),
        comp=4.0 * K.K_BOLTZ * K.SIGMA_T * K.A_RAD * T_cmb**4 / (K.M_E * K.C_LIGHT) * (T - T_cmb),
        rec_HeII=K.K_BOLTZ * T * alpha_HeII_B(T),
        rec_HeIII=2.0 * 3.435e-30 * T * lam3**1.970 / (1.0 + (lam3 / 2.250) ** 0.376) ** 3.720,
        di_HeII=6.526e-11 * alpha_di(T),
        ce_HeII=5.54e-17 * T**-0.397 * np.exp(-473638.0 / T) / (1.0 + np.sqrt(T / 1e5)),
    )


def cooling_rate(T, n_e, n_HI, n_HII, a):
    """Total cooling Lambda per unit proper volume [erg cm^-3 s^-1] (proper densities)."""
    c = cooling_coefficients(T, a)
    return (c["rec_HII"] + c["ff"]) * n_e * n_HII + c["ce_HI"] * n_e * n_HI + c["comp"] * n_e


def cooling_rate_he(T, n_e, n_HI, n_HII, n_HeII, n_HeIII, a):
    """Total cooling of hydrogen + helium gas per unit proper volume [erg cm^-3 s^-1]:
    the hydrogen terms of ``cooling_rate`` (with bremsstrahlung of all ions) plus HeII and
    HeIII recombination cooling, dielectronic recombination cooling and collisional
    excitation of HeII."""
    c = cooling_coefficients(T, a)
    return (c["rec_HII"] * n_e * n_HII + c["ce_HI"] * n_e * n_HI
            + c["ff"] * n_e * (n_HII + n_HeII + 4.0 * n_HeIII) + c["comp"] * n_e
            + (c["rec_HeII"] + c["di_HeII"] + c["ce_HeII"]) * n_e * n_HeII + c["rec_HeIII"] * n_e * n_HeIII)
