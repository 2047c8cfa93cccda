"""Pins of the oracle's dense discrete adjoint against central finite differences of the
whole forward run (gradients of the final volume-weighted ionised fraction)."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as A

CASES = [
    ("reion6_nonisothermal", lambda: W.reionization_field(n=6, nsrc=2, box_mpc=14.4 * 6 / 256, ndot_total=4e49,
                                                          dt_myr=0.3), 2),
    ("stromgren6_isothermal", lambda: W.stromgren_static(n=6, dt_over_trec=1e-3), 2),
]


@pytest.mark.parametrize("name,make,nsteps", CASES)
def test_adjoint_matches_finite_differences(name, make, nsteps):
    w = make()
    ndot = np.array(w["src_ndot"], float)
    clump = np.asarray(w["clump"], float)
    J, g_ndot, g_clump = A.gradient(w, ndot, clump, nsteps)
    assert 0 < J < 1
    for s in range(len(ndot)):
        h = 1e-3 * ndot[s]
        p = ndot.copy(); p[s] += h
        Jp, _ = A.forward(w, p, clump, nsteps)
        p = ndot.copy(); p[s] -= h
        Jm, _ = A.forward(w, p, clump, nsteps)
        fd = (Jp - Jm) / (2 * h)
        assert g_ndot[s] == pytest.approx(fd, rel=1e-6)
        assert g_ndot[s] > 0            # more photons, more ionisation
    v = np.random.default_rng(1).standard_normal(clump.shape)
    h = 3e-3
    Jp, _ = A.forward(w, ndot, clump + h * v, nsteps)
    Jm, _ = A.forward(w, ndot, clump - h * v, nsteps)
    fd = (Jp - Jm) / (2 * h)
    assert float(np.sum(g_clump * v)) == pytest.approx(fd, rel=1e-4)
    # clumping only adds recombinations: every cell's gradient is <= 0
    assert np.all(g_clump <= 1e-14 * np.abs(g_clump).max())


def reion6_moving():
    """The 6^3 field in a box 20 times smaller (same emission per volume), where its 30 km/s
    velocities move a sizeable fraction of a cell per step (Courant number about 0.15)."""
    return W.reionization_field(n=6, nsrc=2, box_mpc=14.4 * 6 / 256 / 20, ndot_total=4e49 / 20**3, dt_myr=0.3)


def test_adjoint_through_advection_matches_finite_differences():
    from oracle import advection as ADV
    from oracle import driver
    w = reion6_moving()
    t0, dt = driver.time_grid(w)
    a, _ = driver.expansion(w, t0 + 0.5 * dt)
    c = ADV.max_courant(w["v"], a, dt, w["dx"], w["periodic"])
    assert 0.05 < c < 1.0
    ndot = np.array(w["src_ndot"], float)
    clump = np.asarray(w["clump"], float)
    nsteps = 2
    J, g_ndot, g_clump = A.gradient(w, ndot, clump, nsteps, advect=True)
    _, g_still, _ = A.gradient(w, ndot, clump, nsteps, advect=False)
    assert np.max(np.abs(g_ndot - g_still)) > 1e-3 * np.max(np.abs(g_ndot))   # advection matters
    for s in range(len(ndot)):
        h = 1e-3 * ndot[s]
        p = ndot.copy(); p[s] += h
        Jp, _ = A.forward(w, p, clump, nsteps, advect=True)
        p = ndot.copy(); p[s] -= h
        Jm, _ = A.forward(w, p, clump, nsteps, advect=True)
        assert g_ndot[s] == pytest.approx((Jp - Jm) / (2 * h), rel=1e-6)
    v = np.random.default_rng(2).standard_normal(clump.shape)
    h = 3e-3
    Jp, _ = A.forward(w, ndot, clump + h * v, nsteps, advect=True)
    Jm, _ = A.forward(w, ndot, clump - h * v, nsteps, advect=True)
    assert float(np.sum(g_clump * v)) == pytest.approx((Jp - Jm) / (2 * h), rel=1e-4)
