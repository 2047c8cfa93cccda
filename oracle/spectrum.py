"""Grey spectral averages for the fixed radiation spectrum (oracle; test infrastructure only).

Sec. "Physical Model", Eq. grey_definition: the radiation energy density per unit
frequency is E_nu = E~(x,t) chi_E(nu) with a prescribed shape chi_E, so the grey
E is its integral from the hydrogen edge nu_0 to infinity.  The paper takes a
T_B = 1e5 K blackbody, chi_E ~ nu^3 / (exp(h nu / k T_B) - 1); its verification
problem uses a monochromatic 13.6 eV source instead.

Integrating the opacity, photo-ionisation and heating terms over that fixed
shape gives three constants per spectrum:

  sigma_E  = int sigma chi_E dnu / int chi_E dnu           (kappa = sigma_E n_HI)
  sigma_G  = int sigma chi_E/(h nu) dnu / int chi_E dnu    (Gamma = c sigma_G E)
  eps_src  = int chi_E dnu / int chi_E/(h nu) dnu          (mean photon energy,
                                                            energy per emitted photon)

with the hydrogen cross section sigma(nu) = sigma_0 (nu / nu_0)^-3.  The heat
deposited per unit absorbed energy follows as (sigma_E - h nu_0 sigma_G).

Computed here with adaptive quadrature (scipy.integrate.quad) in x = h nu / k T_B.
Pinned in tests against closed forms: the Bose-Einstein series for the moments
of x^n/(e^x - 1), -ln(1 - e^-x0) for the nu^-3-weighted moment, and the exact
monochromatic limits.  ``helium_grey_constants`` does the same for the HeI and HeII
cross sections above their own thresholds (pinned against the incomplete-gamma series).
"""
import math

from scipy import integrate

from . import constants as K


def _bb_moment(weight, x0):
    """int_{x0}^inf weight(x) / (e^x - 1) dx by adaptive quadrature."""
    def integrand(x):
        # weight / (e^x - 1) written as weight e^-x / (1 - e^-x) so large x cannot overflow
        return weight(x) * math.exp(-x) / -math.expm1(-x)
    val, _ = integrate.quad(integrand, x0, math.inf, epsabs=0.0, epsrel=1e-13, limit=400)
    return val


def grey_constants(spectrum="blackbody", T_B=1e5):
    """Return dict(sigma_E [cm^2], sigma_G [cm^2/erg], eps_src [erg]).

    spectrum: "blackbody" (T_B in K) or "mono" (all photons at h nu_0 = 13.6 eV).
    """
    if spectrum == "mono":
        return dict(sigma_E=K.SIGMA0, sigma_G=K.SIGMA0 / K.HNU0, eps_src=K.HNU0)
    if spectrum != "blackbody":
        raise ValueError(spectrum)
    kT = K.K_BOLTZ * T_B
    x0 = K.HNU0 / kT
    e3 = _bb_moment(lambda x: x**3, x0)          # ~ int chi_E dnu
    e2 = _bb_moment(lambda x: x**2, x0)          # ~ int chi_E/(h nu) dnu  (times kT)
    s0 = _bb_moment(lambda x: 1.0, x0)           # ~ int sigma chi_E dnu / (sigma_0 x0^3)
    sm1 = _bb_moment(lambda x: 1.0 / x, x0)      # ~ int sigma chi_E/(h nu) dnu
    sigma_E = K.SIGMA0 * x0**3 * s0 / e3
    sigma_G = K.SIGMA0 * x0**3 * sm1 / (kT * e3)
    eps_src = kT * e3 / e2
    return dict(sigma_E=sigma_E, sigma_G=sigma_G, eps_src=eps_src)


def _bb_or_mono_norm(spectrum, T_B):
    kT = K.K_BOLTZ * T_B
    return kT, K.HNU0 / kT, _bb_moment(lambda x: x**3, K.HNU0 / kT)


def helium_grey_constants(spectrum="blackbody", T_B=1e5):
    """Grey constants of the helium species over the same chi_E (normalised by the energy
    above the hydrogen edge, since E integrates from nu_0): dict(sigma_E_HeI, sigma_G_HeI,
    sigma_E_HeII, sigma_G_HeII).  The cross sections vanish below each threshold; a
    monochromatic 13.6 eV spectrum leaves helium un-ionised (all zero)."""
    if spectrum == "mono":
        return dict(sigma_E_HeI=0.0, sigma_G_HeI=0.0, sigma_E_HeII=0.0, sigma_G_HeII=0.0)
    if spectrum != "blackbody":
        raise ValueError(spectrum)
    kT, x0, e3 = _bb_or_mono_norm(spectrum, T_B)
    out = {}
    # HeI: a_T [beta (x1/x)^s + (1 - beta)(x1/x)^(s+1)] x^3 / (e^x - 1), x >= x1
    x1, s, b = K.HNU_HEI / kT, K.S_HEI, K.BETA_HEI
    shape1 = lambda x, p: K.SIGMA_HEI * (b * (x1 / x) ** s + (1 - b) * (x1 / x) ** (s + 1)) * x**p
    out["sigma_E_HeI"] = _bb_moment(lambda x: shape1(x, 3), x1) / e3
    out["sigma_G_HeI"] = _bb_moment(lambda x: shape1(x, 2), x1) / (kT * e3)
    # HeII: sigma_2 (x2/x)^3 x^3 / (e^x - 1), x >= x2
    x2 = K.HNU_HEII / kT
    out["sigma_E_HeII"] = K.SIGMA_HEII * x2**3 * _bb_moment(lambda x: 1.0, x2) / e3
    out["sigma_G_HeII"] = K.SIGMA_HEII * x2**3 * _bb_moment(lambda x: 1.0 / x, x2) / (kT * e3)
    return out
