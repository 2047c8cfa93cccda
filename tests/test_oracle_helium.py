"""Pins of the oracle's hydrogen + helium step (``oracle.helium``; Eq. electron_density's helium
case, the species equations of Eq. RT-chemical_ionization) against what fixes them from outside:
series forms of the grey helium constants, adaptive ODE integration of the frozen-coefficient
rate equations in their unreduced three-species form, equilibrium ratios, the hydrogen-only
model at Y = 0, helium conservation, and finite differences of the complex-step Jacobian."""
import math

import numpy as np
import pytest
from scipy import integrate, special

import workloads as W
from oracle import constants as K
from oracle import driver
from oracle import helium as H
from oracle import model as M
from oracle import newton as N
from oracle import spectrum as S


def _bose_series(p, x0, kmax=400):
    """int_{x0}^inf x^p / (e^x - 1) dx = sum_k Gamma(p + 1, k x0) / k^(p + 1)."""
    a = p + 1.0

    def upper_gamma(a, z):
        if a > 0:
            return special.gammaincc(a, z) * special.gamma(a)
        return (upper_gamma(a + 1.0, z) - z**a * math.exp(-z)) / a      # recurrence down to a < 0
    return sum(upper_gamma(a, k * x0) / k**a for k in range(1, kmax + 1))


def test_helium_grey_constants_match_series():
    T_B = 1e5
    kT = K.K_BOLTZ * T_B
    g = S.helium_grey_constants("blackbody", T_B)
    x0, x1, x2 = K.HNU0 / kT, K.HNU_HEI / kT, K.HNU_HEII / kT
    e3 = _bose_series(3.0, x0)
    s, b = K.S_HEI, K.BETA_HEI
    sE1 = K.SIGMA_HEI * (b * x1**s * _bose_series(3 - s, x1) + (1 - b) * x1 ** (s + 1) * _bose_series(2 - s, x1)) / e3
    sG1 = K.SIGMA_HEI * (b * x1**s * _bose_series(2 - s, x1) + (1 - b) * x1 ** (s + 1) * _bose_series(1 - s, x1))
    sG1 /= kT * e3
    sE2 = K.SIGMA_HEII * x2**3 * -math.log1p(-math.exp(-x2)) / e3
    sG2 = K.SIGMA_HEII * x2**3 * sum(special.exp1(k * x2) for k in range(1, 400)) / (kT * e3)
    assert g["sigma_E_HeI"] == pytest.approx(sE1, rel=1e-9)
    assert g["sigma_G_HeI"] == pytest.approx(sG1, rel=1e-9)
    assert g["sigma_E_HeII"] == pytest.approx(sE2, rel=1e-9)
    assert g["sigma_G_HeII"] == pytest.approx(sG2, rel=1e-9)
    # a 13.6 eV line cannot ionise helium
    assert all(v == 0.0 for v in S.helium_grey_constants("mono").values())


CHAIN_CASES = [  # (G1, G2, r2, r3) in 1/s, dt in s
    (1e-13, 5e-14, 2e-13, 4e-13, 3e13),
    (1e-10, 1e-12, 1e-15, 1e-14, 3e13),      # strongly driven: close to equilibrium
    (0.0, 0.0, 3e-14, 1e-14, 3e13),          # recombination only
    (2e-14, 1e-14, 0.0, 0.0, 3e13),          # photo-ionisation only (no electrons)
    (0.0, 0.0, 0.0, 0.0, 3e13),              # nothing happens
]


@pytest.mark.parametrize("G1,G2,r2,r3,dt", CHAIN_CASES)
def test_helium_chain_matches_ode_integration(G1, G2, r2, r3, dt):
    nHe, x0 = 1.0, (0.6, 0.3)

    def rhs(t, y):   # the three species, unreduced
        I, II, III = y
        return [-G1 * I + r2 * II, G1 * I - (G2 + r2) * II + r3 * III, G2 * II - r3 * III]
    sol = integrate.solve_ivp(rhs, (0.0, dt), [x0[0], x0[1], nHe - x0[0] - x0[1]], method="Radau",
                              rtol=1e-12, atol=1e-15)
    I, II = H.he_chain(x0, nHe, G1, G2, r2, r3, dt)
    assert float(np.real(I[0])) == pytest.approx(sol.y[0, -1], abs=1e-10)
    assert float(np.real(II[0])) == pytest.approx(sol.y[1, -1], abs=1e-10)


def test_helium_chain_equilibrium_ratios():
    G1, G2, r2, r3 = 3e-13, 1e-13, 2e-13, 5e-13
    I, II = (float(np.real(v[0])) for v in H.he_chain((1.0, 0.0), 1.0, G1, G2, r2, r3, 1e16))
    III = 1.0 - I - II
    assert II / I == pytest.approx(G1 / r2, rel=1e-10)      # ionisation balance HeI <-> HeII
    assert III / II == pytest.approx(G2 / r3, rel=1e-10)    # HeII <-> HeIII


@pytest.mark.parametrize("A,G,neHe,dt", [(1e-6, 1e-13, 0.3, 1e13), (1e-5, 1e-11, 0.05, 1e13), (2e-6, 0.0, 0.2, 1e14)])
def test_hydrogen_with_helium_electrons_matches_ode_integration(A, G, neHe, dt):
    nH, y0 = 1.0, 0.7
    sol = integrate.solve_ivp(lambda t, y: [A * (nH - y[0]) * (nH + neHe - y[0]) - G * y[0]], (0.0, dt), [y0],
                              method="Radau", rtol=1e-12, atol=1e-15)
    assert float(H.riccati_SHI(y0, nH, neHe, A, G, dt)) == pytest.approx(sol.y[0, -1], abs=1e-10)
    # without helium electrons it is the hydrogen-only solution
    assert float(H.riccati_SHI(y0, nH, 0.0, A, G, dt)) == pytest.approx(float(M.riccati_Sn(y0, nH, A, G, dt)),
                                                                        rel=1e-14)


def he_step(w):
    """The oracle's hydrogen + helium step for workload w (``workloads.with_helium``)."""
    return H.Run(w).make_step()


def _reion6():
    return W.reionization_field(n=6, nsrc=2, box_mpc=14.4 * 6 / 256, ndot_total=4e49, dt_myr=0.3)


def test_zero_helium_is_the_hydrogen_model():
    w = _reion6()
    st_h = driver.Run(w).make_step()
    st = he_step(W.with_helium(w, Y=0.0))
    # residuals at the (unsolved) initial iterate, where every component is far from zero
    U0 = N.initial_iterate(st_h)
    U0[0] = 1e-3 * M.internal_energy_h(st_h)
    f = np.real(H.residual(st, np.stack([U0[0], U0[1], 0 * U0[1], 0 * U0[1], U0[2]])))
    f_h = M.residual(st_h, U0)
    for a, b in ((0, 0), (1, 1), (4, 2)):
        assert np.max(np.abs(f[a] - f_h[b])) <= 1e-12 * np.max(np.abs(f_h[b]))
    assert np.all(f[2] == 0) and np.all(f[3] == 0)
    U_h, _ = N.solve_step(st_h, tol=1e-11)
    U2, _ = H.solve_step(st, tol=1e-11)
    assert np.max(np.abs(U2[1] - U_h[1]) / st_h.n_H) < 1e-9
    assert np.max(np.abs(U2[4] - U_h[2]) / np.maximum(np.abs(U_h[2]), st_h.E_min)) < 1e-8


@pytest.mark.parametrize("make", [_reion6, lambda: W.stromgren_static(n=8)])
def test_helium_step_converges_and_conserves(make):
    st = he_step(W.with_helium(make()))
    U, info = H.solve_step(st, tol=1e-11)
    HeI, HeII = U[2], U[3]
    assert np.all(HeI >= 0) and np.all(HeII >= 0)
    assert np.all(HeI + HeII <= st.n_He * (1 + 1e-12))
    assert info["hist"][-1] <= 1e-11
    # ionising radiation from the 1e5 K blackbody reaches helium too
    assert np.min(HeI / st.n_He) < 0.5


def test_complex_step_jacobian_matches_finite_differences():
    st = he_step(W.with_helium(W.reionization_field(n=4, nsrc=1, box_mpc=14.4 * 4 / 256, ndot_total=1e49,
                                                    dt_myr=0.3)))
    U = H.local_solve(st, H.initial_iterate(st))
    J = H.jacobian(st, U).toarray()
    Nc = st.N
    rng = np.random.default_rng(0)
    # E columns only where E is above its floor: at the floor the heating it feeds is lost to
    # rounding in (heating - cooling), so a difference quotient cannot see it
    ok = [c for c in range(5 * Nc) if c // Nc != 4 or U[4].ravel()[c % Nc] > 1e3 * st.E_min]
    cols = rng.choice(ok, size=12, replace=False)
    scl = H._scales(st, U).ravel()
    f0 = np.abs(np.real(H.residual(st, U))).ravel()
    for c in cols:
        h = 1e-6 * scl[c]
        Up, Um = U.copy().ravel(), U.copy().ravel()
        Up[c] += h
        Um[c] -= h
        fp, fm = (np.real(H.residual(st, x.reshape(U.shape))).ravel() for x in (Up, Um))
        fd = (fp - fm) / (2 * h)
        # truncation (relative 1e-5) plus the rounding of the difference quotient, eps |f| / h
        ref = np.maximum(np.abs(J[:, c]), np.abs(fd)).max() + 1e-300
        rounding = 4e-16 * np.maximum(np.maximum(np.abs(fp), np.abs(fm)), f0) / h
        assert np.all(np.abs(J[:, c] - fd) <= 1e-5 * ref + rounding)
