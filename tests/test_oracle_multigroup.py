"""Pins of the multigroup oracle (oracle/multigroup.py; Sec. "Physical Model", Eq.
cons_radiation_multifreq integrated over frequency groups) against facts that do not come from
its own formulas: the group constants add up to the grey ones (the spectrum split into groups
covers it exactly), the edge coefficients reproduce the redshift term of the continuous
spectrum computed by quadrature of its derivative, one group is the grey model, identical groups
split the grey root in proportion to their emission, the edge fluxes telescope so that the
total energy follows the grey expansion term, and the complex-step Jacobian agrees with central
differences."""
import math

import numpy as np
import pytest
from scipy import integrate

import workloads as W
from oracle import constants as K
from oracle import driver
from oracle import model as M
from oracle import multigroup as MG
from oracle import newton as N
from oracle import spectrum as S

EDGES = [13.6, 24.59, 54.42]          # eV: the H, HeI and HeII ionisation edges as group edges


def _state(shape, seed, isothermal, adot=0.0):
    w = W.random_state(shape, seed=seed, isothermal=isothermal)
    w["spectrum"] = "blackbody"
    st = driver.Run(w).make_step()
    z, y, x = np.indices(shape)
    st.E_n = 1e-18 * (1.5 + np.sin(x) * np.cos(0.7 * y + 0.3 * z))
    st.adot = adot
    return st


def test_group_constants_add_up_to_the_grey_ones():
    c = MG.group_constants(EDGES)
    g = S.grey_constants("blackbody", 1e5)
    assert np.all(c["frac"] > 0) and c["frac"].sum() == pytest.approx(1.0, rel=1e-12)
    assert np.dot(c["frac"], c["sigma_E"]) == pytest.approx(g["sigma_E"], rel=1e-11)
    assert np.dot(c["frac"], c["sigma_G"]) == pytest.approx(g["sigma_G"], rel=1e-11)
    assert c["eps_src"] == pytest.approx(g["eps_src"], rel=1e-12)
    # harder groups see smaller cross sections (sigma ~ nu^-3)
    assert np.all(np.diff(c["sigma_E"]) < 0)


def test_edge_coefficients_reproduce_the_continuum_redshift_term():
    """For the fixed spectrum split into groups (E_g = frac_g E), the model's redshift terms
    (adot/a)(t_{g+1} E_{g+1} - t_g E_g - E_g) equal (adot/a) int_g nu dE_nu/dnu dnu of the
    continuous spectrum, by quadrature of the derivative of x^3/(e^x - 1); the first group
    differs by the flux through nu_0, which the grey equation and the model drop."""
    c = MG.group_constants(EDGES)
    kT = K.K_BOLTZ * 1e5
    xs = [e * K.EV / kT for e in EDGES] + [math.inf]
    chi = lambda x: x**3 * math.exp(-x) / -math.expm1(-x)
    dchi = lambda x: (3 * x**2 * (1 - math.exp(-x)) - x**3) * math.exp(-x) / (1 - math.exp(-x)) ** 2
    total = integrate.quad(chi, xs[0], math.inf, epsrel=1e-13, limit=400)[0]
    E = 1.0
    Eg = c["frac"] * E
    G = len(EDGES)
    for g in range(G):
        model = (c["t"][g + 1] * Eg[g + 1] if g + 1 < G else 0.0) - (c["t"][g] * Eg[g] if g > 0 else 0.0) - Eg[g]
        cont = integrate.quad(lambda x: x * dchi(x), xs[g], xs[g + 1], epsrel=1e-12, limit=400)[0] * E / total
        if g == 0:
            cont += xs[0] * chi(xs[0]) * E / total          # the flux through nu_0, dropped
        assert model == pytest.approx(cont, rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("iso", [True, False])
def test_one_group_is_the_grey_model(iso):
    st = _state((4, 3, 3), 3, iso, adot=1e-17)
    c = MG.group_constants([13.6])
    mg = MG.make_mg_step(st, c)
    rng = np.random.default_rng(1)
    U = N.initial_iterate(st)
    U[2] = st.E_n * (1 + 0.3 * rng.random(st.shape))
    if not iso:
        U[0] = 1e9
    f_grey = M.residual(st, U)
    f_mg = MG.residual(mg, U)
    for k in range(3):
        np.testing.assert_allclose(f_mg[k], f_grey[k], rtol=1e-13, atol=1e-13 * np.abs(f_grey[k]).max())
    Ug, _ = N.solve_step(st, tol=1e-11)
    Um, _ = MG.solve_step(mg, tol=1e-11)
    np.testing.assert_allclose(Um, Ug, rtol=1e-10, atol=0)


@pytest.mark.parametrize("iso", [True, False])
def test_identical_groups_split_the_grey_root(iso):
    """Two groups with the grey cross sections and emission shares 0.3 / 0.7 (static universe):
    the equations are those of the grey field scaled by the shares (the limiter depends on E
    only through grad E / E), so the root is the grey root split 0.3 / 0.7 with the same n_HI
    and e_c."""
    st = _state((5, 4, 3), 12, iso)
    g = S.grey_constants("blackbody", 1e5)
    f = np.array([0.3, 0.7])
    c = dict(sigma_E=np.full(2, g["sigma_E"]), sigma_G=np.full(2, g["sigma_G"]), frac=f, t=np.zeros(2),
             eps_src=g["eps_src"])
    mg = MG.make_mg_step(st, c)
    Ug, _ = N.solve_step(st, tol=1e-11)
    Um, _ = MG.solve_step(mg, tol=1e-11)
    np.testing.assert_allclose(Um[1], Ug[1], rtol=1e-9)
    if not iso:
        np.testing.assert_allclose(Um[0], Ug[0], rtol=1e-8, atol=1e-8 * np.abs(Ug[0]).max())
    for k in range(2):
        np.testing.assert_allclose(Um[2 + k], f[k] * Ug[2], rtol=1e-9)


def test_edge_fluxes_telescope_to_the_grey_expansion_term():
    """No opacity, no sources, a uniform field, adot > 0: the sum of the group energies after the
    step equals the grey step's energy (the edge fluxes cancel in the sum), and the spectrum
    shifts towards the lowest group (redshift)."""
    shape = (3, 3, 3)
    st = _state(shape, 2, True, adot=3e-17)
    st.E_n = np.full(shape, 1e-18)
    st.src_index = np.array([], np.int64)
    st.src_ndot = np.array([])
    st.sigma_E = 0.0
    st.sigma_G = 0.0
    c = MG.group_constants(EDGES)
    c0 = dict(c, sigma_E=np.zeros(3), sigma_G=np.zeros(3))
    mg = MG.make_mg_step(st, c0)
    Ug, _ = N.solve_step(st, tol=1e-13)
    Um, _ = MG.solve_step(mg, tol=1e-13)
    np.testing.assert_allclose(Um[2:].sum(axis=0), Ug[2], rtol=1e-12)
    share = Um[2:, 0, 0, 0] / Um[2:, 0, 0, 0].sum()
    assert share[0] > c["frac"][0] and share[-1] < c["frac"][-1]


@pytest.mark.parametrize("iso", [True, False])
def test_complex_step_jacobian_matches_central_differences(iso):
    st = _state((3, 3, 3), 5, iso, adot=2e-17)
    mg = MG.make_mg_step(st, MG.group_constants(EDGES))
    U = MG.initial_iterate(mg)
    U[2:] = mg.E_n * 1.6
    if not iso:
        U[0] = 3e9
    J = MG.jacobian(mg, U).toarray()
    bE = MG.explicit_part(mg)
    flat = U.ravel()
    scale = MG._scales(mg, U).ravel()
    Jfd = np.zeros_like(J)
    for j in range(flat.size):
        h = 1e-6 * scale[j]
        up, dn = flat.copy(), flat.copy()
        up[j] += h
        dn[j] -= h
        Jfd[:, j] = (MG.residual(mg, up.reshape(U.shape), bE).ravel() - MG.residual(mg, dn.reshape(U.shape), bE).ravel()) / (2 * h)
    rows = np.abs(Jfd).max(axis=1, keepdims=True) + 1e-300
    assert np.max(np.abs(J - Jfd) / rows) < 1e-5

