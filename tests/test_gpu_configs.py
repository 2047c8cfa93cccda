"""The five workload configurations at their stated sizes, checked through properties that hold
at any size (the oracle cannot run them whole):

* static Stromgren sphere, FP64 (reflecting lower and outflow upper faces): the configuration's
  steps of 0.01 t_rec, each halved when Newton fails at it (the paper runs the problem under its
  time-step control); the I-front radius against R_s (1 - e^{-t/t_rec})^{1/3} at 128^3 to
  t_rec / 2 and at 256^3 to t_rec / 5.  Past about 0.6 t_rec the preconditioned CG needs a few
  hundred iterations per Newton step at 128^3 and Newton needs many step halvings; the runs to
  t_rec (128^3) and 2 t_rec (256^3) are opt-in (RT_LONG_TESTS=1);
* cosmological Stromgren sphere, FP64, 128^3, flat LCDM from z = 10 to z = 4 with the adaptive
  controller: the front against the oracle's integration of the expanding-universe I-front
  equation;
* reionization field at 512^3 (14.4 Mpc box), mixed precision: the first quarter Myr and one
  more step, then the oracle's residual at sampled cells of that step (evaluated on each cell's
  3^3 neighbourhood, which fixes the centre cell's residual exactly at theta = 1) and its
  cell-local equations;
* adjoint on the 128^3 field with 64 sources over 50 steps (mixed forward): gradient signs and
  directional finite differences along the emissivities and a random clumping field.
"""
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402
from oracle import constants as K  # noqa: E402
from oracle import cosmology as C  # noqa: E402
from oracle import diagnostics as D  # noqa: E402
from oracle import driver  # noqa: E402
from oracle import model as M  # noqa: E402


# the Stromgren runs to one and two recombination times take many minutes: opt in with RT_LONG_TESTS=1
LONG = pytest.mark.skipif(os.environ.get("RT_LONG_TESTS") != "1",
                          reason="long validation run; set RT_LONG_TESTS=1")


def _solver(w, **kw):
    from paper_0908_2654_gb300.solver import Solver
    return Solver(w, **kw)


def _neff(w, s):
    g = s.grey()
    return w["ndot_total"] * g["eps_src"] * g["sigma_G"] / g["sigma_E"]


def _static_stromgren_run(n, t_ends, max_newton=15, max_lin=500):
    """Steps of 0.01 t_rec (halved where Newton fails, then back), front errors at t_ends [t_rec].
    A Newton solve that cannot converge in 15 iterations with at most 500 CG iterations each is
    retried at half the step rather than pushed further."""
    w = W.stromgren_static(n=n, nsteps=200)
    s = _solver(w, precision="fp64", newton_tol=1e-8, lin_rtol=1e-6, max_newton=max_newton, max_lin=max_lin)
    neff = _neff(w, s)
    t_rec = w["t_rec"]
    errs, steps = [], []
    for t_end in t_ends:
        st = s.advance(t_end * t_rec, tau_tol=1e3, dt_max=0.01 * t_rec)
        steps.append(len(st))
        ec, nHI, E = s.state_cgs()
        rI = D.ifront_radius(nHI, w["rho_b"] / K.M_H, w["dx"], True)
        errs.append(rI / C.static_ifront(s.t, neff, K.ALPHA_B_PAPER, w["nH"]) - 1.0)
    s.close()
    return np.array(errs), steps


def test_static_stromgren_128_to_half_a_recombination_time():
    """128^3 in the configuration's 0.01 t_rec steps to t_rec / 2: the front within 8 % of the
    closed form at 0.25 and 0.5 t_rec (the diffuse FLD front lags the sharp closed-form one most
    while it is young; measured 5.7 % and 4.0 %)."""
    errs, steps = _static_stromgren_run(128, (0.25, 0.5))
    assert np.all(np.abs(errs) < 0.08), (errs, steps)
    assert steps[0] >= 25


def test_static_stromgren_256_to_a_fifth_of_a_recombination_time():
    """256^3 in 0.01 t_rec steps to t_rec / 5: the front within 8 % of the closed form."""
    errs, steps = _static_stromgren_run(256, (0.2,))
    assert np.all(np.abs(errs) < 0.08), (errs, steps)
    assert steps[0] >= 20


@LONG
def test_static_stromgren_128_to_one_recombination_time():
    errs, steps = _static_stromgren_run(128, (0.25, 0.5, 1.0), max_newton=40, max_lin=2000)
    assert np.all(np.abs(errs) < 0.08), (errs, steps)


@LONG
def test_static_stromgren_256_to_two_recombination_times():
    errs, steps = _static_stromgren_run(256, (0.25, 0.5, 1.0, 1.5, 2.0), max_newton=40, max_lin=2000)
    assert np.all(np.abs(errs) < 0.08), (errs, steps)


def test_cosmological_stromgren_128_z10_to_z4():
    """Nominally 500 steps from z = 10 to z = 4; covered with the adaptive controller."""
    w = W.stromgren_cosmo(n=128, z0=10.0, z_end=4.0, nsteps=500)
    s = _solver(w, precision="fp64", newton_tol=1e-8, lin_rtol=1e-6, max_newton=30)
    neff = _neff(w, s)
    cos = C.FlatLCDM(**w["cosmology"])
    t0 = s.t
    s.dt = 1e-3 / (K.ALPHA_B_PAPER * w["nH"] * 11.0**3)          # a thousandth of t_rec at z0
    errs = []
    for z in (9.0, 8.0, 6.0, 5.0, 4.0):
        s.advance(cos.t_of_z(z), tau_tol=0.01)
        ec, nHI, E = s.state_cgs()
        r = D.ifront_radius(nHI, w["rho_b"] / K.M_H, w["dx"], True)
        Vc = C.ifront_ode(t0, s.t, cos.a, neff, K.ALPHA_B_PAPER, w["nH"])
        errs.append(r / (3.0 * Vc / (4.0 * math.pi)) ** (1.0 / 3.0) - 1.0)
    s.close()
    assert np.all(np.abs(errs) < 0.05), errs


def _neighbourhood_step(w, run, c):
    """The oracle's step restricted to the 3^3 neighbourhood of cell c (periodic wrap), its
    centre cell at index 13."""
    shape = (w["nz"], w["ny"], w["nx"])
    z, y, x = np.unravel_index(c, shape)
    iz, iy, ix = ((np.arange(-1, 2) + q) % n for q, n in zip((z, y, x), shape))
    sl = np.ix_(iz, iy, ix)
    sub = dict(w)
    flat = np.ravel_multi_index(np.meshgrid(iz, iy, ix, indexing="ij"), shape).ravel()
    srcs = np.asarray(w["src_index"])
    inside = np.isin(srcs, flat)
    local = np.array([np.nonzero(flat == q)[0][0] for q in srcs[inside]], np.int64)
    sub.update(nx=3, ny=3, nz=3, periodic=(False, False, False), bc=None, rho_b=w["rho_b"][sl], T0=w["T0"][sl],
               v=tuple(v[sl] for v in w["v"]), clump=w["clump"][sl], E=run.E[sl], nHI=run.nHI[sl],
               src_index=local, src_ndot=np.asarray(w["src_ndot"])[inside])
    r = driver.Run(sub)
    r.e_h, r.t, r.dt = run.e_h[sl], run.t, run.dt
    return r.make_step(), sl


def test_reionization_field_512_mixed_step_sampled_residuals():
    """The 14.4 Mpc field at 512^3 (2000 sources, 1e52 photons/s): the controller covers the
    first quarter Myr, then one more step of its proposed length is checked cell by cell
    against the oracle."""
    w = W.reionization_field(n=512, nsrc=2000, box_mpc=14.4, ndot_total=1e52)
    s = _solver(w, precision="mixed", newton_tol=1e-6, lin_rtol=1e-3)
    s.dt = 0.25 * w["dt"]
    s.advance(s.t + s.dt, tau_tol=0.05)
    start = (s.E.clone(), s.nHI.clone(), s.e_h.clone(), s.t)
    stats = s.step(fold=False)
    assert stats["norm"] <= 1e-6
    u = s.units
    ec, nHI, E = s.state_cgs()
    run = driver.Run(w)
    run.E, run.nHI = start[0].cpu().numpy() * u.u_E, start[1].cpu().numpy() * u.u_n
    run.e_h, run.t, run.dt = start[2].cpu().numpy() * u.u_v**2, start[3], s.dt
    s.close()
    rng = np.random.default_rng(5)
    cells = np.concatenate([rng.choice(512**3, size=40, replace=False), np.asarray(w["src_index"][:10])])
    for c in cells:
        st, sl = _neighbourhood_step(w, run, int(c))
        U = np.stack([ec[sl], nHI[sl], E[sl]])
        f = M.residual(st, U)
        fe, fn, fE = (x.ravel()[13] for x in f)
        se = max(float(M.internal_energy_h(st).ravel()[13]), M.E_FLOOR_INT())
        assert abs(fn) / float(st.n_H.ravel()[13]) < 1e-6, c
        assert abs(fe) / se < 1e-6, c
        # f_E against the rounding scale of its terms (neighbours can be far brighter)
        Ec = U[2]
        scale = (abs(Ec.ravel()[13]) + abs(st.E_n.ravel()[13])
                 + st.dt * 3e10 * float(M.opacity(st, U[1]).ravel()[13]) * abs(Ec.ravel()[13])
                 + st.dt * float(M.emissivity(st).ravel()[13]) + np.max(np.abs(Ec)))
        assert abs(fE) / scale < 1e-5, c


def test_adjoint_128_64_sources_50_steps():
    from paper_0908_2654_gb300.adjoint import ionized_fraction
    w = W.reionization_field(n=128, nsrc=64, box_mpc=14.4 * 128 / 256, ndot_total=1e52 / 8)
    opt = dict(precision="mixed", newton_tol=1e-10, lin_rtol=1e-11, max_newton=60, max_lin=400)
    nsteps = 50
    ndot0 = np.asarray(w["src_ndot"], float)
    clump0 = np.asarray(w["clump"], np.float32)
    ndot = torch.tensor(ndot0, dtype=torch.float64, requires_grad=True)
    clump = torch.tensor(clump0, requires_grad=True)
    J = ionized_fraction(ndot, clump, w, nsteps, **opt)
    J.backward()
    g_ndot = ndot.grad.numpy()
    g_clump = clump.grad.numpy()
    assert np.all(g_ndot > 0)                            # more photons, more ionisation
    assert np.all(g_clump <= 1e-12 * np.abs(g_clump).max())   # clumping only adds recombinations
    # directional derivative along the emissivities themselves
    eps = 1e-3
    Jp = float(ionized_fraction(torch.tensor(ndot0 * (1 + eps)), torch.tensor(clump0), w, nsteps, **opt))
    Jm = float(ionized_fraction(torch.tensor(ndot0 * (1 - eps)), torch.tensor(clump0), w, nsteps, **opt))
    assert float(np.dot(g_ndot, ndot0)) == pytest.approx((Jp - Jm) / (2 * eps), rel=1e-4)
    # and along a random clumping field
    v = np.random.default_rng(7).standard_normal(clump0.shape).astype(np.float32)
    h = 1e-2
    Jp = float(ionized_fraction(torch.tensor(ndot0), torch.tensor(clump0 + h * v), w, nsteps, **opt))
    Jm = float(ionized_fraction(torch.tensor(ndot0), torch.tensor(clump0 - h * v), w, nsteps, **opt))
    assert float(np.sum(g_clump.astype(np.float64) * v)) == pytest.approx((Jp - Jm) / (2 * h), rel=1e-3)
