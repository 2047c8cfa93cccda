"""The seeded synthetic inputs (workloads/) follow the recipe they state: the reionization-like
field's density, velocity and source statistics, its ionised blocks, and determinism under a
seed.  No GPU is needed."""
import numpy as np
import pytest

import workloads as W
from oracle import constants as K

N, NSRC = 32, 20


@pytest.fixture(scope="module")
def field():
    return W.reionization_field(n=N, nsrc=NSRC, box_mpc=14.4 * N / 256, ndot_total=1e52 * (N / 256) ** 3)


def test_seeded_and_deterministic(field):
    again = W.reionization_field(n=N, nsrc=NSRC, box_mpc=14.4 * N / 256, ndot_total=1e52 * (N / 256) ** 3)
    for key in ("rho_b", "nHI", "T0", "src_index", "src_ndot"):
        np.testing.assert_array_equal(field[key], again[key])
    for a, b in zip(field["v"], again["v"]):
        np.testing.assert_array_equal(a, b)
    other = W.reionization_field(n=N, nsrc=NSRC, seed=1234, box_mpc=14.4 * N / 256)
    assert not np.array_equal(field["rho_b"], other["rho_b"])


def test_density_is_lognormal_about_the_cosmic_mean(field):
    """ln rho Gaussian with sigma_ln = 1 and the mean-preserving shift -sigma^2/2 about
    n_H = Omega_b rho_crit / m_H = 2.20e-7 cm^-3 (Omega_b = 0.04, h = 0.7, X = 1)."""
    nH_mean = W.LCDM["Omega_b"] * W.RHO_CRIT_H2 * W.LCDM["h"] ** 2 / W.M_H
    assert nH_mean == pytest.approx(2.20e-7, rel=1e-2)
    # the generator's critical density agrees with 3 H^2 / (8 pi G) from the constants
    assert W.RHO_CRIT_H2 == pytest.approx(K.RHO_CRIT_H2, rel=1e-4)
    g = np.log(field["rho_b"] / (nH_mean * W.M_H))
    assert g.std() == pytest.approx(1.0, rel=1e-12)
    assert g.mean() == pytest.approx(-0.5, abs=1e-12)


def test_velocities_have_the_stated_dispersion(field):
    for v in field["v"]:
        assert v.std() == pytest.approx(30.0 * 1e5, rel=1e-12)
        assert abs(v.mean()) < 1e-9 * v.std()


def test_density_spectrum_slope():
    """Shell-averaged power of ln rho falls as k^-2.5 (fit over the resolved shells)."""
    n = 64
    w = W.reionization_field(n=n, nsrc=4, box_mpc=14.4 * n / 256)
    g = np.log(w["rho_b"])
    p = np.abs(np.fft.rfftn(g - g.mean())) ** 2
    kz = np.fft.fftfreq(n)[:, None, None]
    ky = np.fft.fftfreq(n)[None, :, None]
    kx = np.fft.rfftfreq(n)[None, None, :]
    k = np.sqrt(kx**2 + ky**2 + kz**2) * n
    shells = np.arange(2, 20)
    pk = np.array([p[(k >= s - 0.5) & (k < s + 0.5)].mean() for s in shells])
    slope = np.polyfit(np.log(shells), np.log(pk), 1)[0]
    assert slope == pytest.approx(-2.5, abs=0.25)


def test_sources_are_the_densest_peaks_with_rates_proportional_to_density(field):
    rho = field["rho_b"]
    src = np.asarray(field["src_index"])
    assert len(src) == NSRC and len(np.unique(src)) == NSRC
    flat = rho.ravel()
    zc, yc, xc = np.unravel_index(src, rho.shape)
    for z, y, x, s in zip(zc, yc, xc, src):         # strict maxima of the 27-cell neighbourhood
        nb = rho[np.ix_([(z - 1) % N, z, (z + 1) % N], [(y - 1) % N, y, (y + 1) % N], [(x - 1) % N, x, (x + 1) % N])]
        assert flat[s] == nb.max() and np.sum(nb == flat[s]) == 1
    # no peak outside the list is denser than the faintest source
    m = np.ones(rho.shape, bool)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dz or dy or dx:
                    m &= rho > np.roll(rho, (dz, dy, dx), axis=(0, 1, 2))
    others = np.setdiff1d(np.flatnonzero(m), src)
    assert len(others) == 0 or flat[others].max() <= flat[src].min()
    ndot = np.asarray(field["src_ndot"])
    assert ndot.sum() == pytest.approx(1e52 * (N / 256) ** 3, rel=1e-12)
    np.testing.assert_allclose(ndot / flat[src], ndot[0] / flat[src[0]], rtol=1e-12)


def test_ionised_blocks_around_sources(field):
    xHI = field["nHI"] / (field["rho_b"] / K.M_H)
    blocks = np.zeros(xHI.shape, bool)
    zc, yc, xc = np.unravel_index(np.asarray(field["src_index"]), xHI.shape)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                blocks[(zc + dz) % N, (yc + dy) % N, (xc + dx) % N] = True
    np.testing.assert_allclose(xHI[blocks], 1e-4, rtol=1e-12)
    np.testing.assert_allclose(xHI[~blocks], 0.9999, rtol=1e-12)
    assert np.all(field["T0"][blocks] == 1e4) and np.all(field["T0"][~blocks] == 100.0)


def _gold():
    import json
    import os
    return json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_stromgren_workloads_use_the_papers_values():
    """Static and cosmological Stromgren inputs: the paper's source rate, initial radiation
    energy, case-B coefficient and 1e4 K isothermal gas, the source in the octant corner
    emitting Ndot / 8, walls on every axis, and t_rec = 1 / (alpha_B n_H)."""
    gold = _gold()
    ndot, E0, alpha = (gold[k]["value"] for k in ("Ndot_photons_s", "E_initial_erg_cm3", "alpha_B_cm3_s"))
    for w in (W.stromgren_static(n=8), W.stromgren_cosmo(n=8)):
        assert w["ndot_total"] == ndot and np.all(w["src_ndot"] == ndot / 8.0)
        assert list(w["src_index"]) == [0] and w["octant"] and w["periodic"] == (False, False, False)
        assert np.all(w["E"] == E0) and np.all(w["T0"] == 1e4)
        assert w["isothermal"] and w["T_iso"] == 1e4 and w["recomb"] == "const"
    w = W.stromgren_static(n=8)
    assert w["t_rec"] == pytest.approx(1.0 / (alpha * 1e-3), rel=1e-15)
    assert w["dt"] == pytest.approx(0.01 * w["t_rec"], rel=1e-15)
    assert w["dx"] * w["nx"] == pytest.approx(6.6 * 3.0856775814913673e21, rel=1e-15)


@pytest.mark.parametrize("row", range(4))
def test_shapiro_giroux_inputs_follow_table1(row):
    """Table 1 row by row: the generator's table is the paper's, the box is L0 comoving at z0
    (proper L0 at z0), the gas is Omega_b rho_crit, comoving, fully neutral, and the source
    is the paper's monochromatic 13.6 eV one."""
    gold = _gold()
    q0, z0, L0, h, Om, OL, Ob = gold["table1"]["rows"][row]
    assert tuple(float(v) for v in W.SG_TABLE1[row]) == tuple(float(v) for v in (q0, z0, L0, h, Om, OL, Ob))
    w = W.shapiro_giroux(row, n=8)
    assert w["dx"] * w["nx"] / (1.0 + z0) == pytest.approx(L0 * 3.0856775814913673e21, rel=1e-15)
    nH = Ob * W.RHO_CRIT_H2 * h**2 / W.M_H
    np.testing.assert_allclose(w["rho_b"], nH * W.M_H, rtol=1e-15)
    np.testing.assert_allclose(w["nHI"], nH, rtol=1e-15)
    assert w["spectrum"] == "mono" and w["cosmology"] == dict(q0=q0, h=h) and w["z0"] == z0
