"""The GPU path's closed forms for helium (helium.cuh: the helium chain from the real
eigenvalues of its rate matrix, with its Taylor and large-eigenvalue-gap branches, and the
hydrogen Riccati solution with helium electrons), compiled for the host, against the oracle's
independent routes (expm of the augmented matrix; the oracle's Riccati form) across stiff,
slow, degenerate and strongly driven regimes, values and derivatives."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import helium as H

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def host_lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("host") / "he_chain_host.so")
    subprocess.run([nvcc, "-x", "cu", "-std=c++17", "--expt-relaxed-constexpr", "-O2", "-shared", "-Xcompiler",
                    "-fPIC", "-gencode", "arch=compute_103a,code=sm_103a", os.path.join(HERE, "host", "he_chain_host.cu"),
                    "-o", out], check=True, capture_output=True)
    return ctypes.CDLL(out)


def _arr(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _regimes(rng, n):
    """Rate sets in 1/s over 10 decades, with zero photo-ionisation, zero electrons, equal
    recombination rates (coincident eigenvalues) and strongly driven cells among them."""
    G1 = 10 ** rng.uniform(-20, -9, n)
    G2 = G1 * 10 ** rng.uniform(-3, 0, n)
    r2 = 10 ** rng.uniform(-20, -11, n)
    r3 = r2 * 10 ** rng.uniform(-1, 1.5, n)
    dt = 10 ** rng.uniform(10, 15, n)
    k = n // 8
    G1[:k] = G2[:k] = 0.0                       # recombination only
    r2[k:2 * k] = r3[k:2 * k] = 0.0             # no electrons
    r3[2 * k:3 * k] = r2[2 * k:3 * k]           # coincident eigenvalues
    G1[3 * k:4 * k] *= 1e4                      # strongly driven (large 2 delta dt)
    return G1, G2, r2, r3, dt


def test_helium_chain_matches_oracle(host_lib):
    rng = np.random.default_rng(11)
    n = 4000
    G1, G2, r2, r3, dt = _regimes(rng, n)
    nHe = np.ones(n)
    f1 = rng.uniform(0, 1, n)
    x10 = f1 * rng.uniform(0, 1, n)
    x20 = (1 - f1) * rng.uniform(0, 1, n)
    out = [np.empty(n) for _ in range(4)]
    args = [_arr(v) for v in (x10, x20, nHe, G1, G2, r2, r3, dt)]
    host_lib.he_chain_host(ctypes.c_int(n), *[_p(a) for a in args], *[_p(o) for o in out])
    x1, x2, d1, d2 = out
    # the oracle's chain takes one dt; the solution depends on the rates only through rate * dt
    ref1, ref2 = (np.real(v) for v in H.he_chain((x10, x20), nHe, G1 * dt, G2 * dt, r2 * dt, r3 * dt, 1.0))
    # scaling and squaring in the oracle's expm loses ~1e-11 at |M dt| ~ 1e7 (the closed form
    # matches a 50-digit evaluation to 1e-16 there)
    assert np.max(np.abs(x1 - ref1)) < 1e-10
    assert np.max(np.abs(x2 - ref2)) < 1e-10
    # derivatives in G1 and r3 against complex steps through the oracle's route
    h = 1e-30
    g1 = (G1 + 1j * h * np.maximum(G1, 1e-25)) * dt
    c1 = np.imag(H.he_chain((x10, x20), nHe, g1, G2 * dt, r2 * dt, r3 * dt, 1.0)[0]) / (h * np.maximum(G1, 1e-25))
    g3 = (r3 + 1j * h * np.maximum(r3, 1e-25)) * dt
    c2 = np.imag(H.he_chain((x10, x20), nHe, G1 * dt, G2 * dt, r2 * dt, g3, 1.0)[1]) / (h * np.maximum(r3, 1e-25))
    s1 = np.maximum(np.abs(c1), 1e-300) * 1e-7 + 1e-9 * dt
    s2 = np.maximum(np.abs(c2), 1e-300) * 1e-7 + 1e-9 * dt
    assert np.all(np.abs(d1 - c1) <= s1)
    assert np.all(np.abs(d2 - c2) <= s2)


def test_hydrogen_with_helium_electrons_matches_oracle(host_lib):
    rng = np.random.default_rng(12)
    n = 2000
    nH = np.ones(n)
    y0 = rng.uniform(1e-6, 1.0, n)
    neHe = rng.uniform(0.0, 0.2, n)
    A = 10 ** rng.uniform(-20, -12, n)
    G = 10 ** rng.uniform(-22, -10, n)
    G[: n // 10] = 0.0
    dt = 10 ** rng.uniform(10, 15, n)
    y = np.empty(n)
    args = [_arr(v) for v in (y0, nH, neHe, A, G, dt)]
    host_lib.riccati_ne_host(ctypes.c_int(n), *[_p(a) for a in args], _p(y))
    ref = np.real(H.riccati_SHI(y0, nH, neHe, A, G, dt))
    assert np.max(np.abs(y - ref)) < 1e-12


def test_rate_fits_match_oracle_over_temperature(host_lib):
    """Hydrogen and helium recombination coefficients and the cooling coefficients of the GPU
    path (one d/dT lane, chained) against the oracle's rate functions from 1 K to 1e9 K; the
    cooling coefficients are compared through the oracle's total cooling with one density at
    a time switched on."""
    from oracle import constants as K
    from oracle import rates as R
    n = 400
    T = np.logspace(0, 9, n)
    a = 0.1
    out, dout = np.empty(9 * n), np.empty(9 * n)
    host_lib.rates_host(ctypes.c_int(n), _p(_arr(T)), ctypes.c_double(a), _p(out), _p(dout))
    out, dout = out.reshape(9, n), dout.reshape(9, n)
    aH, a2, a3, rf, ff, ce, comp, c2, c3 = out
    np.testing.assert_allclose(aH, R.alpha_B(T, "hg97"), rtol=1e-13)
    np.testing.assert_allclose(a2, R.alpha_HeII_B(T) + R.alpha_di(T), rtol=1e-13)
    np.testing.assert_allclose(a3, R.alpha_HeIII_B(T), rtol=1e-13)
    one, zero = np.ones(n), np.zeros(n)
    # cooling_rate_he(T, n_e, n_HI, n_HII, n_HeII, n_HeIII, a) with n_e = 1 and one other density
    cool = lambda nHI, nHII, n2, n3: R.cooling_rate_he(T, one, nHI, nHII, n2, n3, a)
    comp_ref = cool(zero, zero, zero, zero)
    np.testing.assert_allclose(comp, comp_ref, rtol=1e-12, atol=1e-40)
    # each reference is (total - Compton): its rounding is of the size of the Compton term
    ac = 1e-14 * np.abs(comp_ref)
    np.testing.assert_allclose(rf, cool(zero, one, zero, zero) - comp_ref, rtol=1e-12, atol=ac.max())
    np.testing.assert_allclose(ce, cool(one, zero, zero, zero) - comp_ref, rtol=1e-11, atol=ac.max())
    np.testing.assert_allclose(ff + c2, cool(zero, zero, one, zero) - comp_ref, rtol=1e-11, atol=ac.max())
    np.testing.assert_allclose(4 * ff + c3, cool(zero, zero, zero, one) - comp_ref, rtol=1e-11, atol=ac.max())
    # d/dT of the recombination coefficients against complex steps of the oracle's fits
    h = 1e-20
    for got, f in ((dout[0], lambda t: R.alpha_B(t, "hg97")), (dout[1], lambda t: R.alpha_HeII_B(t) + R.alpha_di(t)),
                   (dout[2], R.alpha_HeIII_B)):
        ref = np.imag(f(T + 1j * h * T)) / (h * T)
        np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-300)


def test_hydrogen_riccati_matches_oracle(host_lib):
    """S_n of the hydrogen-only path (e^-x and phi1 from one expm1, with the series below
    |x| = 1e-8) against the oracle's form, from frozen chemistry (d dt ~ 1e-12) to stiff."""
    from oracle import model as M
    rng = np.random.default_rng(13)
    n = 3000
    nH = np.ones(n)
    y0 = rng.uniform(1e-6, 1.0, n)
    A = 10 ** rng.uniform(-24, -10, n)
    G = 10 ** rng.uniform(-26, -8, n)
    G[: n // 10] = 0.0
    dt = 10 ** rng.uniform(10, 15, n)
    y = np.empty(n)
    args = [_arr(v) for v in (y0, nH, A, G, dt)]
    host_lib.riccati_n_host(ctypes.c_int(n), *[_p(a) for a in args], _p(y))
    ref = np.real(M.riccati_Sn(y0, nH, A, G, dt))
    assert np.max(np.abs(y - ref)) < 1e-13


def test_hydrogen_rate_fits_match_oracle_over_temperature(host_lib):
    """The hydrogen-only kernels' rates (physics.cuh t_rates: the Hui & Gnedin alpha and the
    cooling coefficients rf = recombination + bremsstrahlung, ce, comp, each with d/dT from one
    dual lane chained into the cell's partials) against the oracle's per-process coefficients
    from 1 K to 1e9 K; the chained lane that is not T stays exactly zero."""
    from oracle import rates as R
    n = 400
    T = np.logspace(0, 9, n)
    a = 0.2
    out, dout, dz = np.empty(4 * n), np.empty(4 * n), np.empty(4 * n)
    host_lib.t_rates_host(ctypes.c_int(n), _p(_arr(T)), ctypes.c_double(a), _p(out), _p(dout), _p(dz))
    out, dout = out.reshape(4, n), dout.reshape(4, n)
    c = R.cooling_coefficients(T, a)
    refs = (lambda t: R.alpha_B(t, "hg97"), lambda t: (lambda q: q["rec_HII"] + q["ff"])(R.cooling_coefficients(t, a)),
            lambda t: R.cooling_coefficients(t, a)["ce_HI"], lambda t: R.cooling_coefficients(t, a)["comp"])
    np.testing.assert_allclose(out[0], R.alpha_B(T, "hg97"), rtol=1e-13)
    np.testing.assert_allclose(out[1], c["rec_HII"] + c["ff"], rtol=1e-13)
    np.testing.assert_allclose(out[2], c["ce_HI"], rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(out[3], c["comp"], rtol=1e-13)
    h = 1e-20
    for k, f in enumerate(refs):
        ref = np.imag(f(T + 1j * h * T)) / (h * T)
        np.testing.assert_allclose(dout[k], ref, rtol=1e-10, atol=1e-300)
    assert np.all(dz == 0.0)


def test_face_limiter_matches_oracle(host_lib):
    """Eq. limiter as the face kernels evaluate it (value form and dual form), against the
    oracle's face_D on two-cell rows. The cases cover energy ratios over 60 decades, both
    energies below E_min, optically thin faces (kappa = 0), equal energies (R = 0) and the
    case kappa = R = 0. The dual form's dD/dE_i is compared with a complex step through the
    oracle."""
    from types import SimpleNamespace
    from oracle import model as M
    rng = np.random.default_rng(17)
    n = 3000
    adx, E_min = 3.1e21, 1e-35
    Ei = 10 ** rng.uniform(-40, 20, n)
    Ej = Ei * 10 ** rng.uniform(-30, 30, n)
    ki = 10 ** rng.uniform(-30, -15, n)
    kj = ki * 10 ** rng.uniform(-5, 5, n)
    k = n // 10
    ki[:k] = kj[:k] = 0.0                            # optically thin
    Ej[k:2 * k] = Ei[k:2 * k]                        # no gradient
    Ej[2 * k:3 * k] = Ei[2 * k:3 * k]
    ki[2 * k:3 * k] = kj[2 * k:3 * k] = 0.0          # kappa = R = 0
    Ei[3 * k:4 * k] *= 1e-30                         # both far below E_min
    Ej[3 * k:4 * k] = Ei[3 * k:4 * k] * 3.0
    D, Dt, dD = np.empty(n), np.empty(n), np.empty(n)
    host_lib.limiter_host(ctypes.c_int(n), *[_p(_arr(v)) for v in (Ei, Ej, ki, kj)], ctypes.c_double(adx),
                          ctypes.c_double(M.K.C_LIGHT), ctypes.c_double(E_min), _p(D), _p(Dt), _p(dD))
    st = SimpleNamespace(limiter="new", a=1.0, dx=adx, E_min=E_min, shape=(1, n, 2),
                         periodic=(False, False, False), faces=("reflect",) * 6, D_const=0.0)

    def oracle_D(ei):
        E = np.stack([ei, Ej + 0 * ei], axis=-1)[None]
        kap = np.stack([ki, kj], axis=-1)[None]
        return M.face_D(st, E, kap, 0)[0, :, 0]

    ref = np.real(oracle_D(Ei))
    np.testing.assert_allclose(D, ref, rtol=1e-13)
    np.testing.assert_allclose(Dt, D, rtol=1e-15)         # the dual quotient rounds differently (1 ulp)
    h = 1e-20
    cs = np.imag(oracle_D(Ei + 1j * h * Ei)) / (h * Ei)
    # rounding scale of the chain rule dD/dR dR/dE_i, from the magnitudes of the quotient
    # rules' terms: those of dR/dE_i, (E_f + |dE|/2) / (adx E_f^2), cancel when E_j << E_i
    # (R saturates at 2 / adx); those of dD/dR, c / den and D (3 kappa_T + 2 R) / den with
    # den = 6 kappa_T^2 + 3 kappa_T R + R^2, cancel as R -> 0 (dD/dR vanishes at R = 0)
    Ef = np.real(M.spos(0.5 * (Ei + Ej), E_min))
    R = np.abs(Ej - Ei) / (adx * Ef)
    kT = 0.5 * (ki + kj)
    den = 6.0 * kT**2 + 3.0 * kT * R + R**2
    with np.errstate(divide="ignore", invalid="ignore"):
        D_R_terms = (M.K.C_LIGHT + ref * (3.0 * kT + 2.0 * R)) / den
    scale = D_R_terms * (Ef + 0.5 * np.abs(Ej - Ei)) / (adx * Ef**2)
    has_derivative = ~((kT == 0) & (R == 0))         # kappa = R = 0: D jumps from c / R to c adx
    err = np.abs(dD - cs)[has_derivative]
    assert np.all(err <= 1e-9 * np.abs(cs[has_derivative]) + 1e-13 * scale[has_derivative])
