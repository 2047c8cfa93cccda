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
monochromatic limits.
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
