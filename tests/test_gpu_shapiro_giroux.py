"""The four cosmological I-front problems of the verification section (Table 1: q0 in {0.5,
0.05}, z0 in {4, 10}) run on the GPU with the adaptive time-step controller, against the
Shapiro-Giroux closed form (Eqs. SG-solution, SG-tau, SG-F, evaluated by the oracle): the
equivalent-volume I-front radius at several expansion factors, the first-order convergence of
its error in the step tolerance, agreement between meshes and (opt-in, RT_LONG_TESTS=1) the
convergence of the front under mesh refinement 16^3 -> 32^3 -> 64^3."""
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402
from oracle import constants as K  # noqa: E402
from oracle import cosmology as C  # noqa: E402


def _sg_run(row, n, tau, abars):
    """Relative error r_I / r_SG - 1 at each expansion factor abar = a / a(z0)."""
    from paper_0908_2654_gb300.solver import Solver
    w = W.shapiro_giroux(row, n=n)
    sg = w["sg"]
    s = Solver(w, precision="mixed", newton_tol=1e-8, lin_rtol=1e-6, max_newton=20, max_lin=400)
    nH0 = sg["Omega_b"] * K.RHO_CRIT_H2 * sg["h"] ** 2 * (1 + sg["z0"]) ** 3 / K.M_H
    H0 = sg["h"] * K.H100
    a0 = 1.0 / (1.0 + sg["z0"])
    s.dt = 1e-3 / (K.ALPHA_B_PAPER * nH0)           # a thousandth of the recombination time
    errs = []
    for ab in abars:
        s.advance(s.cosmo.t_of_z(1.0 / (a0 * ab) - 1.0), tau_tol=tau)
        xHII = 1.0 - s.nHI / s.rho
        V = 8.0 * float(torch.sum(xHII)) * w["dx"] ** 3           # octant: eight times the box
        r = (3.0 * V / (4.0 * math.pi)) ** (1.0 / 3.0) * a0      # comoving, in proper units at z0
        rsg = C.sg_ifront(s.cosmo.a(s.t) / a0, sg["q0"], sg["z0"], H0, 5e48, K.ALPHA_B_PAPER, nH0)
        errs.append(r / rsg - 1.0)
    s.close()
    return np.array(errs)


@pytest.mark.parametrize("row", [0, 1, 2, 3])
def test_front_follows_shapiro_giroux(row):
    err = _sg_run(row, 16, 0.005, (1.2, 1.5, 2.0))
    assert np.all(np.abs(err) < 0.06), err
    assert abs(err[-1]) < 0.03, err


def test_front_error_converges_with_the_step_tolerance():
    e1 = _sg_run(2, 16, 0.01, (1.5,))[0]
    e2 = _sg_run(2, 16, 0.005, (1.5,))[0]
    assert abs(e2) < abs(e1) / 1.4, (e1, e2)


@pytest.mark.parametrize("row", [0, 1])
def test_meshes_agree(row):
    e16 = _sg_run(row, 16, 0.005, (1.5, 2.0))
    e32 = _sg_run(row, 32, 0.005, (1.5, 2.0))
    assert np.all(np.abs(e32) < 0.03), e32
    assert np.all(np.abs(e32 - e16) < 0.01), (e16, e32)


@pytest.mark.skipif(os.environ.get("RT_LONG_TESTS") != "1", reason="long validation run; set RT_LONG_TESTS=1")
def test_front_converges_under_mesh_refinement():
    """Row 0 to abar = 2 at a step tolerance small enough (5e-4) that the time error sits below
    the mesh differences: the change from 32^3 to 64^3 is at most a third of the change from
    16^3 to 32^3, and every mesh is within 1 % of the closed form (the offset left at 64^3, about
    0.5 %, no longer changes with the mesh)."""
    e = [_sg_run(0, n, 5e-4, (2.0,))[0] for n in (16, 32, 64)]
    assert np.all(np.abs(e) < 0.01), e
    assert abs(e[2] - e[1]) <= abs(e[1] - e[0]) / 3.0, e
