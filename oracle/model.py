"""Nonlinear residual of the implicit radiation / ionisation / heating step (oracle).

Test infrastructure only.  Follows Sec. "Algorithm", subsection "Operator-Split
Hydrodynamics with Radiative Feedback": step (v) solves Eqs. RT-cons_energy,
RT-chemical_ionization and RT-cons_radiation for U = (e_c, n_HI, E) through the
residual f(U) = (f_e, f_n, f_E) of Eqs. gas_residual, chemistry_residual and
radiation_residual.  Hydrogen only (N_s = 1, n_e = n_HII = n_H - n_HI,
Eq. electron_density), X = 1 so rho_b = m_H n_H.

Everything is in CGS comoving variables: E and n are comoving densities
(proper = comoving / a^3, Eq. proper_vars), dx is the comoving cell width,
v_b the proper peculiar velocity, e_h the specific total gas energy from the
hydrodynamics, a and adot = da/dt the expansion factor and its time derivative.
Arrays are indexed [z, y, x].

Readings of points the paper leaves open (listed in the design notes):
  * D in the implicit part: by default (limiter "lagged") the limiter is evaluated from
    the step's starting state (E^n, n_HI^n) at both time levels, so the radiation
    operator is linear and symmetric within a step and the reduced (Schur) system is
    symmetric positive definite, as the conjugate-gradient solver named in
    Sec. "Algorithm" requires; limiter "new" evaluates D from the iterate.
  * FLD on cell faces: R = |E_{i+1}-E_i| / (a dx pos(mean E)), kappa_T the
    mean of the two cells' proper opacities (no scattering); R = 1/(a dx) when
    kappa_T = R = 0.  Proper spacing a*dx, so the comoving operator carries 1/a^2.
  * kappa = sigma_E n_HI / a^3; Gamma = c sigma_G E / a^3; recombination
    alpha C n_e n_HII / a^3 in the comoving rate equation (C = clumping factor).
  * m = 1 in Eq. RT-cons_radiation.
  * E may be negative in the discrete solution: with theta < 1 and dt c kappa >> 1 the
    two-level scheme maps a floor value E^n to about -(1-theta)/theta E^n.  Rates use
    pos(theta E + (1-theta) E^n).  Here pos(x) = (x + sqrt(x^2 + E_min^2))/2 is a smooth
    positive part: a hard max(., E_min) puts every cell still at the floor value on a kink
    of f, where Newton directions fail.
  * S_n: exact solution over dt of the rate equation with its coefficients frozen
    (alpha at T(U), Gamma at the theta-weighted E), a Riccati equation
        y' = A (n_H - y)^2 - Gbar y,  A = alpha C / a^3,  y(0) = n_HI^n.
  * S_e: exact solution of de/dt = -2 (adot/a) e + (G - Lambda) with frozen
    G - Lambda and e_c^n = 0; isothermal runs use f_e = e_c.
  * Point sources: 4 pi eta = sum_s Ndot_s eps_src / dx^3 in the source's cell.
  * Boundaries (Sec. "Verification tests": reflecting at the lower faces, outflow at the upper
    faces), per face: "periodic" (both faces of the axis), "reflect" (zero flux through the
    face) or "outflow".  Outflow lets radiation leave the box: beyond the face lies a ghost
    cell holding no radiation (E = 0) and a copy of the boundary cell's gas (same opacity), and
    the face flux follows Eq. limiter between the two like any interior face.  (A ghost holding
    a copy of E as well would give zero diffusive flux, i.e. a reflecting face.)
"""
from dataclasses import dataclass, field
from typing import Optional, Tuple

import numpy as np

from . import constants as K
from . import rates

E_MIN_DEFAULT = 1e-35  # erg/cm^3, the paper's initial radiation floor


def cabs(x):
    """|x| on the real part, analytic continuation of the sign (complex-step safe)."""
    return np.where(np.real(x) >= 0, x, -x)


def cmax(x, c):
    """max(x, c) compared on real parts (complex-step safe)."""
    return np.where(np.real(x) >= np.real(c), x, c)


def spos(x, eps):
    """Smooth positive part (x + sqrt(x^2 + eps^2)) / 2: equals x for x >> eps, eps/2 at 0,
    tends to 0 for x << -eps, and is differentiable everywhere (Newton needs f smooth)."""
    r = np.sqrt(x * x + eps * eps)
    neg = np.real(x) < 0
    # for x < 0 the same value as eps^2 / (2 (r - x)), free of cancellation
    return np.where(neg, eps * eps / (2.0 * (r - np.where(neg, x, -1.0))), 0.5 * (x + r))


@dataclass
class Step:
    """One implicit step's data in CGS comoving units."""
    nx: int
    ny: int
    nz: int
    dx: float                                   # comoving cell width [cm]
    periodic: Tuple[bool, bool, bool]           # (x, y, z); False = see bc (default: reflect)
    rho_b: np.ndarray                           # comoving baryon density [g/cm^3]
    e_h: np.ndarray                             # specific total gas energy after hydro [erg/g]
    v: Tuple[np.ndarray, np.ndarray, np.ndarray]  # proper peculiar velocity (x, y, z) [cm/s]
    clump: np.ndarray                           # clumping factor on the recombination term
    E_n: np.ndarray                             # radiation energy density at step start
    nHI_n: np.ndarray                           # neutral hydrogen density at step start
    a: float
    adot: float                                 # da/dt [1/s]
    dt: float                                   # [s]
    src_index: np.ndarray                       # flat [z,y,x] cell index of each source
    src_ndot: np.ndarray                        # ionising photons / s of each source
    sigma_E: float
    sigma_G: float
    eps_src: float
    theta: float = 0.51
    isothermal: bool = True
    T_iso: float = 1e4
    recomb: str = "const"                       # "const" | "hg97"
    cooling: bool = True                        # non-isothermal only
    limiter: str = "lagged"                     # "lagged" | "new" | "const"
    D_const: float = 0.0                        # proper diffusion coefficient for limiter "const"
    E_min: float = E_MIN_DEFAULT
    bc: Optional[Tuple[str, ...]] = None        # per face (x-, x+, y-, y+, z-, z+); None: from periodic

    @property
    def faces(self):
        """Boundary type of the six faces (x-, x+, y-, y+, z-, z+): "periodic", "reflect" or
        "outflow"; without ``bc`` the non-periodic axes reflect at both faces."""
        if self.bc is not None:
            bc = tuple(self.bc)
            for d in range(3):
                per = (bc[2 * d] == "periodic", bc[2 * d + 1] == "periodic")
                if per != (bool(self.periodic[d]),) * 2:
                    raise ValueError(f"boundary types {bc} disagree with periodic={self.periodic}")
            return bc
        return tuple(t for p in self.periodic for t in (("periodic",) * 2 if p else ("reflect",) * 2))

    @property
    def shape(self):
        """Array shape [z][y][x]."""
        return (self.nz, self.ny, self.nx)

    @property
    def N(self):
        """Number of cells."""
        return self.nx * self.ny * self.nz

    @property
    def n_H(self):
        """Hydrogen number density rho / m_H (X = 1)."""
        return self.rho_b / K.M_H


# --------------------------------------------------------------------------- FLD


def limiter_D(kappa_T, R):
    """Eq. limiter: D = c (2 kappa_T + R) / (6 kappa_T^2 + 3 kappa_T R + R^2)."""
    return K.C_LIGHT * (2.0 * kappa_T + R) / (6.0 * kappa_T**2 + 3.0 * kappa_T * R + R**2)


_AXIS = {0: 2, 1: 1, 2: 0}   # (x, y, z) -> numpy axis of an [z, y, x] array


def _limiter_faces(st, E, Ep, kappa, kp):
    """Eq. limiter on faces between cells with energies (E, Ep) and proper opacities (kappa, kp):
    R = |Ep - E| / (a dx pos(mean E)), kappa_T the mean opacity, R = 1/(a dx) where both vanish."""
    adx = st.a * st.dx
    if st.limiter == "const":
        return np.full(np.shape(E), st.D_const, dtype=np.result_type(E, float))
    Ef = spos(0.5 * (E + Ep), st.E_min)
    R = cabs(Ep - E) / (adx * Ef)
    kT = 0.5 * (kappa + kp)
    both0 = (np.real(kT) == 0) & (np.real(R) == 0)
    R = np.where(both0, 1.0 / adx, R)
    return limiter_D(kT, R)


def _limiter_state(st, E, kappa, freeze):
    """(E, kappa) the limiter is evaluated from: the step's start for limiter "lagged"."""
    if st.limiter == "lagged":
        E, kappa = st.E_n, opacity(st, st.nHI_n)
    if freeze:
        E = np.real(E)
        kappa = np.real(kappa)
    return E, kappa


def face_D(st, E, kappa, d, freeze=False):
    """D on the +d face of every cell (face between cell i and its +d neighbour).

    Limiter "lagged" evaluates D from the step's starting state (E^n, kappa^n) at both time
    levels; "new" from the iterate (E, kappa), and with freeze=True from its real parts only
    (a linearisation that holds D fixed); "const" uses D_const.  On the last cell along a
    non-periodic axis the +d face is the boundary: D = 0 for a reflecting face; for an outflow
    face D is the limiter between the cell and its ghost (E = 0, the cell's own opacity).
    """
    ax = _AXIS[d]
    E, kappa = _limiter_state(st, E, kappa, freeze)
    D = _limiter_faces(st, E, np.roll(E, -1, axis=ax), kappa, np.roll(kappa, -1, axis=ax))
    if not st.periodic[d]:
        last = [slice(None)] * 3
        last[ax] = -1
        last = tuple(last)
        D = D.copy()
        if st.faces[2 * d + 1] == "outflow":
            D[last] = _limiter_faces(st, E[last], 0.0 * E[last], kappa[last], kappa[last])
        else:
            D[last] = 0.0
    return D


def lower_boundary_D(st, E, kappa, d, freeze=False):
    """D on the -d boundary face of the first cell along a non-periodic axis (an [..] slab of
    the array's shape with that axis of length 1): the limiter between the cell and its ghost
    for an outflow face, 0 for a reflecting one."""
    ax = _AXIS[d]
    E, kappa = _limiter_state(st, E, kappa, freeze)
    first = [slice(None)] * 3
    first[ax] = slice(0, 1)
    first = tuple(first)
    if st.faces[2 * d] == "outflow":
        return _limiter_faces(st, E[first], 0.0 * E[first], kappa[first], kappa[first])
    return np.zeros(np.shape(E[first]), dtype=np.result_type(E, float))


def diffusion(st, E, kappa, freeze=False):
    """div(D grad E) with proper spacing a*dx: sum over the cell's faces of D (E_nb - E) / (a dx)^2,
    where the neighbour beyond an outflow face is the ghost E = 0 and a reflecting face carries
    no flux."""
    adx2 = (st.a * st.dx) ** 2
    out = np.zeros(st.shape, dtype=np.result_type(E, kappa, float))
    for d in range(3):
        ax = _AXIS[d]
        D = face_D(st, E, kappa, d, freeze)
        Enb = np.roll(E, -1, axis=ax)
        if not st.periodic[d]:
            last = [slice(None)] * 3
            last[ax] = -1
            Enb = Enb.copy()
            Enb[tuple(last)] = 0.0                      # the ghost beyond the + boundary face
        flux_p = D * (Enb - E)                          # through the +d face, into the cell
        flux_m = np.roll(flux_p, 1, axis=ax)            # the -d face is the -d neighbour's +d face
        if not st.periodic[d]:
            first = [slice(None)] * 3
            first[ax] = slice(0, 1)
            first = tuple(first)
            flux_m = flux_m.copy()
            # through the - boundary face, out of the cell into its ghost (E = 0)
            flux_m[first] = lower_boundary_D(st, E, kappa, d, freeze) * (E[first] - 0.0)
        out = out + (flux_p - flux_m) / adx2
    return out


def opacity(st, nHI, nHe=None):
    """Proper opacity kappa = sigma_E n_HI / a^3 [1/cm]; with helium (``oracle.helium``) also
    sigma_E,HeI n_HeI + sigma_E,HeII n_HeII, from nHe = (n_HeI, n_HeII) or, if None, the
    step's starting values."""
    k = st.sigma_E * nHI
    if getattr(st, "helium", False):
        nHeI, nHeII = (st.nHeI_n, st.nHeII_n) if nHe is None else nHe
        k = k + st.sigma_E_HeI * nHeI + st.sigma_E_HeII * nHeII
    return k / st.a**3


def emissivity(st):
    """4 pi eta per cell: point sources inject Ndot eps_src into the comoving cell volume."""
    ndot = np.asarray(st.src_ndot)
    src = np.zeros(st.N, dtype=np.result_type(ndot, float))
    np.add.at(src, np.asarray(st.src_index, dtype=np.int64), ndot * st.eps_src / st.dx**3)
    return src.reshape(st.shape)


def radiation_rhs(st, E, nHI, src, freeze=False, nHe=None):
    """The bracket of Eq. radiation_residual: div(D grad E) - (adot/a) E + 4 pi eta - c kappa E."""
    kappa = opacity(st, nHI, nHe)
    return diffusion(st, E, kappa, freeze) - (st.adot / st.a) * E + src - K.C_LIGHT * kappa * E


def explicit_part(st):
    """b_E = E^n + dt (1 - theta) [bracket at time n] (the last line of Eq. radiation_residual)."""
    src = emissivity(st)
    return st.E_n + st.dt * (1.0 - st.theta) * radiation_rhs(st, st.E_n, st.nHI_n, src)


# ---------------------------------------------------------------- local solutions


def phi1(x):
    """(1 - e^-x) / x, with its limit 1 at x = 0."""
    x = np.asarray(x)
    small = np.abs(np.real(x)) < 1e-8
    xs = np.where(small, 1.0, x)
    return np.where(small, 1.0 - x / 2.0 + x * x / 6.0, -np.expm1(-xs) / xs)


def riccati_Sn(y0, nH, A, G, dt):
    """Exact solution at time dt of y' = A (nH - y)^2 - G y, y(0) = y0.

    The right side factors as A (y - y_eq)(y - y_2) with roots
    y_eq = 2 A nH^2 / (2 A nH + G + d) <= nH <= y_2, d = sqrt(G^2 + 4 A G nH) = A (y_2 - y_eq).
    With u = y - y_eq the equation is Bernoulli, u' = A u^2 - d u, whose solution is
    u(t) = u0 e^{-d t} / (1 - u0 A t phi1(d t)),  phi1(x) = (1 - e^-x)/x.
    """
    d = np.sqrt(G * G + 4.0 * A * G * nH)
    den = 2.0 * A * nH + G + d
    den0 = np.real(den) == 0
    y_eq = np.where(den0, 0.0, 2.0 * A * nH * nH / np.where(den0, 1.0, den))
    u0 = y0 - y_eq
    q = np.exp(-d * dt)
    return y_eq + u0 * q / (1.0 - u0 * A * dt * phi1(d * dt))


def temperature(st, e_c, nHI):
    """Eqs. eos + temperature: T = (gamma-1) e_int rho / (k_B n_tot), n_tot = n_H + n_e."""
    if st.isothermal:
        return st.T_iso + 0.0 * nHI
    v2 = st.v[0] ** 2 + st.v[1] ** 2 + st.v[2] ** 2
    e_int = st.e_h + e_c - 0.5 * v2
    nH = st.n_H
    return (K.GAMMA - 1.0) * e_int * st.rho_b / (K.K_BOLTZ * (2.0 * nH - nHI))


def local_solutions(st, U):
    """(S_e, S_n) of Eqs. gas_residual / chemistry_residual at the iterate U."""
    e_c, nHI, E = U
    a3 = st.a**3
    nH = st.n_H
    # theta-weighted E; the theta scheme can leave E slightly negative in optically thick
    # cells holding only the floor value, so rates see max(Ebar, 0)
    Ebar = spos(st.theta * E + (1.0 - st.theta) * st.E_n, st.E_min)
    G = K.C_LIGHT * st.sigma_G * Ebar / a3                   # photo-ionisation rate [1/s]
    T = temperature(st, e_c, nHI)
    A = rates.alpha_B(T, st.recomb) * st.clump / a3
    Sn = riccati_Sn(st.nHI_n, nH, A, G, st.dt)
    if st.isothermal:
        return None, Sn
    heat = nHI * K.C_LIGHT * Ebar * (st.sigma_E - K.HNU0 * st.sigma_G) / (a3 * st.rho_b)
    cool = 0.0
    if st.cooling:
        nHII = nH - nHI
        cool = a3 * rates.cooling_rate(T, nHII / a3, nHI / a3, nHII / a3, st.a) / st.rho_b
    Se = (heat - cool) * st.dt * phi1(2.0 * (st.adot / st.a) * st.dt)
    return Se, Sn


def residual(st, U, bE=None, freeze=False):
    """f(U) = (f_e, f_n, f_E), Eqs. gas_residual, chemistry_residual, radiation_residual.

    U = (e_c, n_HI, E), each an [z,y,x] array (complex allowed).  bE = explicit_part(st)
    may be passed to avoid recomputation.  freeze=True holds the FLD coefficient D at
    its real value (a linearisation used by the method's Schur system; it does not
    change f itself, only its complex-step derivative).
    """
    e_c, nHI, E = U
    if bE is None:
        bE = explicit_part(st)
    src = emissivity(st)
    Se, Sn = local_solutions(st, U)
    f_e = e_c if st.isothermal else e_c - Se
    f_n = nHI - Sn
    f_E = E - bE - st.dt * st.theta * radiation_rhs(st, E, nHI, src, freeze)
    return np.stack([f_e, f_n, f_E])


def local_residual(st, e_c, nHI, E):
    """(f_e, f_n) alone: the cell-local equations of Eqs. gas_residual, chemistry_residual."""
    Se, Sn = local_solutions(st, (e_c, nHI, E))
    f_e = e_c if st.isothermal else e_c - Se
    return f_e, nHI - Sn


def internal_energy_h(st):
    """Specific internal energy of the hydro state, e_h - |v|^2 / 2 (Eq. eos with e the total
    specific energy)."""
    v2 = st.v[0] ** 2 + st.v[1] ** 2 + st.v[2] ** 2
    return st.e_h - 0.5 * v2


def E_FLOOR_INT():
    """Specific internal energy of 1 K gas with mu = 1 [erg/g] (norm floor)."""
    return K.K_BOLTZ / ((K.GAMMA - 1.0) * K.M_H)


E_REL_FLOOR = 1e-12


def weight_floor_E(st):
    """Smallest E scale the norm resolves: max(E_min, 1e-12 max_cells(E^n + dt 4 pi eta)),
    fixed for the step.  Radiation twelve orders of magnitude below the brightest cell of
    the step does not ionise anything within dt; asking for per-cell relative accuracy
    there is below the rounding left by the bright cells."""
    return max(st.E_min, E_REL_FLOOR * float(np.max(np.abs(st.E_n + st.dt * emissivity(st)))))


def weights(st, U):
    """Per-component scales of the residual norm (w_e, w_n, w_E) at the iterate U.

    f_E / max(|E|, E^n, E_floor), f_n / n_H, f_e / max(e_int of the hydro state, 1 K).
    """
    e_c, nHI, E = np.real(U)
    wE = 1.0 / np.maximum(np.maximum(np.abs(E), st.E_n), weight_floor_E(st))
    wn = 1.0 / st.n_H
    we = 1.0 / np.maximum(internal_energy_h(st), E_FLOOR_INT())
    return np.stack([we + 0 * E, wn + 0 * E, wE])


def rms_norm(w, f):
    """Eq. rmsnorm: ||w f||_2 / sqrt(N (N_s + 2)) with N_s = 1."""
    v = (w * np.real(f)).ravel()
    return float(np.sqrt(np.dot(v, v) / v.size))
