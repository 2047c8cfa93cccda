"""Physical constants in CGS used by the oracle (test infrastructure only).

CODATA 2018 values; the hydrogen ionisation edge h*nu_0 = 13.6 eV and the case-B
coefficient alpha_B = 2.59e-13 cm^3/s are the values the paper states in its
verification section.
"""

C_LIGHT = 2.99792458e10          # cm / s
H_PLANCK = 6.62607015e-27        # erg s
K_BOLTZ = 1.380649e-16           # erg / K
EV = 1.602176634e-12             # erg
M_H = 1.6735575e-24              # g, hydrogen atom mass (X = 1 gas: rho_b = m_H n_H)
M_E = 9.1093837015e-28           # g
SIGMA_T = 6.6524587321e-25       # cm^2, Thomson
A_RAD = 7.565723e-15             # erg cm^-3 K^-4
GAMMA = 5.0 / 3.0                # ratio of specific heats (paper)

HNU0 = 13.6 * EV                 # hydrogen ionisation threshold (paper: 13.6 eV)
SIGMA0 = 6.3e-18                 # cm^2, H photo-ionisation cross section at threshold
ALPHA_B_PAPER = 2.59e-13         # cm^3 / s, case-B coefficient quoted by the paper

# helium (hydrogen + helium chemistry): thresholds and threshold cross sections; HeI with the
# two-term power law a_T [beta (nu/nu_T)^-s + (1 - beta)(nu/nu_T)^(-s-1)] of Osterbrock (1989),
# HeII hydrogenic (Z = 2: sigma_0 / 4 at four times the hydrogen edge, nu^-3 like hydrogen)
HNU_HEI = 24.59 * EV
HNU_HEII = 54.42 * EV
SIGMA_HEI = 7.83e-18             # cm^2
BETA_HEI, S_HEI = 1.66, 2.05
SIGMA_HEII = 1.58e-18            # cm^2
M_HE_OVER_M_H = 4.0              # helium atom mass in hydrogen masses (n_He = Y rho / (4 m_H))

KPC = 3.0856775814913673e21      # cm
MPC = 1e3 * KPC
YEAR = 3.15576e7                 # s (Julian)
MYR = 1e6 * YEAR
KM = 1e5                         # cm
T_CMB0 = 2.725                   # K
H100 = 100.0 * KM / MPC          # 100 km/s/Mpc in 1/s
RHO_CRIT_H2 = 3.0 * H100**2 / (8.0 * 3.141592653589793 * 6.67430e-8)  # g/cm^3 per h^2
