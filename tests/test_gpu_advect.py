"""The advection pre-step (rt_advect, rt_advect_adjoint; step (iv), donor cell) against the
oracle's scheme and its transpose: ragged grids with walls and periodic axes, the exact shift at
Courant number 1, the Courant bound and argument errors, the 256^3 reionization field, and
multi-step gradients through advection against the oracle's dense adjoint."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402
from oracle import adjoint as OA  # noqa: E402
from oracle import advection as ADV  # noqa: E402

TOL = 1e-13     # relative to the field's largest magnitude; the two sides round c_f differently


def _solver(w, **kw):
    from paper_0908_2654_gb300.solver import Solver
    return Solver(w, precision="fp64", **kw)


def _scale_dt(s, w, courant):
    """Set the solver's dt so that the largest outflow Courant number is ``courant``."""
    a = s.inputs().a
    c1 = ADV.max_courant(w["v"], a, 1.0, w["dx"], w["periodic"])
    s.dt = courant / c1
    return a


def _advect(s, src, dst, rho=None, inp=None):
    from paper_0908_2654_gb300 import _rt
    inp = s.inputs() if inp is None else inp
    c = ctypes.c_double(-1.0)
    code = _rt.lib().rt_advect(s.handle, ctypes.byref(inp), ctypes.byref(src), ctypes.byref(dst),
                               _rt.ptr(rho[0]) if rho else None, _rt.ptr(rho[1]) if rho else None, ctypes.byref(c))
    return code, c.value


@pytest.mark.parametrize("shape,periodic", [((5, 7, 9), (False, False, False)), ((8, 6, 10), (True, True, True)),
                                            ((16, 12, 20), (True, False, True)), ((3, 1, 37), (False, True, True))])
def test_advect_matches_oracle(shape, periodic):
    from paper_0908_2654_gb300 import _rt
    w = W.random_state(shape, seed=sum(shape), periodic=periodic)
    s = _solver(w)
    a = _scale_dt(s, w, 0.9)
    u = s.units
    oE, on, orho = (torch.empty_like(s.E) for _ in range(3))
    code, cmax = _advect(s, s.state(), s.state(oE, on), rho=(s.rho, orho))
    _rt.check(code, "rt_advect")
    assert cmax == pytest.approx(0.9, rel=1e-12)
    args = (w["v"], a, s.dt, w["dx"], w["periodic"])
    for got, q, scale in ((oE, w["E"], u.u_E), (on, w["nHI"], u.u_n), (orho, w["rho_b"], u.u_d)):
        ref = ADV.advect(q, *args)
        err = np.max(np.abs(got.cpu().numpy() * scale - ref)) / np.max(np.abs(ref))
        assert err < TOL, err
    # n_HI* <= n_H*: the same fluxes move both
    assert torch.all(on <= orho * (1 + 1e-12))
    s.close()


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_courant_one_is_an_exact_shift(axis):
    from paper_0908_2654_gb300 import _rt
    w = W.random_state((6, 5, 7), seed=3)
    s = _solver(w)
    inp = s.inputs()
    inp.a, inp.dt = 1.0, s.desc.dx                  # dt / (a dx) = 1 exactly
    ones = torch.ones_like(s.E)
    inp.vx = inp.vy = inp.vz = None
    setattr(inp, "vx vy vz".split()[axis], _rt.ptr(ones))
    oE, on = torch.empty_like(s.E), torch.empty_like(s.E)
    code, cmax = _advect(s, s.state(), s.state(oE, on), inp=inp)
    _rt.check(code, "rt_advect")
    assert cmax == 1.0
    dim = 2 - axis                                   # numpy axis of x, y, z
    # q_i - (q_i - q_{i-1}) = q_{i-1} up to the two roundings of the update
    for got, q in ((oE, s.E), (on, s.nHI)):
        ref = torch.roll(q, 1, dim)
        assert torch.all(torch.abs(got - ref) <= 4.5e-16 * torch.maximum(torch.abs(q), torch.abs(ref)))
    s.close()


@pytest.mark.parametrize("periodic", [(True, True, True), (False, True, False)])
def test_adjoint_matches_oracle_transpose(periodic):
    from paper_0908_2654_gb300 import _rt
    w = W.random_state((7, 6, 9), seed=5, periodic=periodic)
    s = _solver(w)
    a = _scale_dt(s, w, 0.8)
    rng = np.random.default_rng(6)
    lE, ln = rng.normal(size=s.shape), rng.normal(size=s.shape)
    tE, tn = torch.tensor(lE, device=s.dev), torch.tensor(ln, device=s.dev)
    oE, on = torch.empty_like(tE), torch.empty_like(tn)
    inp = s.inputs()
    _rt.check(_rt.lib().rt_advect_adjoint(s.handle, ctypes.byref(inp), ctypes.byref(s.state(tE, tn)),
                                          ctypes.byref(s.state(oE, on))), "rt_advect_adjoint")
    args = (w["v"], a, s.dt, w["dx"], w["periodic"])
    for got, lam in ((oE, lE), (on, ln)):
        ref = ADV.advect_adjoint(lam, *args)
        assert np.max(np.abs(got.cpu().numpy() - ref)) < TOL * np.max(np.abs(ref))
    s.close()


def test_courant_above_one_is_rejected_and_nothing_written():
    from paper_0908_2654_gb300 import _rt
    w = W.random_state((6, 6, 6), seed=7)
    s = _solver(w)
    _scale_dt(s, w, 1.5)
    oE, on = torch.full_like(s.E, 7.0), torch.full_like(s.E, 7.0)
    code, cmax = _advect(s, s.state(), s.state(oE, on))
    assert code == _rt.RT_EINVAL
    assert cmax == pytest.approx(1.5, rel=1e-12)
    assert torch.all(oE == 7.0) and torch.all(on == 7.0)
    s.close()


def test_overlapping_arrays_are_rejected():
    from paper_0908_2654_gb300 import _rt
    s = _solver(W.random_state((4, 4, 4), seed=8))
    on = torch.empty_like(s.E)
    code, _ = _advect(s, s.state(), s.state(s.E, on))
    assert code == _rt.RT_EINVAL
    code, _ = _advect(s, s.state(), s.state(on, on))
    assert code == _rt.RT_EINVAL
    s.close()


def test_reionization_field_256():
    """The field of the throughput runs (30 km/s velocities, dt = 1 Myr at z = 9): whole-grid
    parity, conservation of every density, and n_HI <= n_H after the move."""
    import bench
    from paper_0908_2654_gb300 import _rt
    w = bench.workload(256)
    s = _solver(w)
    u = s.units
    a = s.inputs().a
    oE, on, orho = (torch.empty_like(s.E) for _ in range(3))
    code, cmax = _advect(s, s.state(), s.state(oE, on), rho=(s.rho, orho))
    _rt.check(code, "rt_advect")
    args = (w["v"], a, s.dt, w["dx"], w["periodic"])
    assert cmax == pytest.approx(ADV.max_courant(*args), rel=1e-12)
    for got, src, q, scale in ((oE, s.E, w["E"], u.u_E), (on, s.nHI, w["nHI"], u.u_n),
                               (orho, s.rho, w["rho_b"], u.u_d)):
        ref = ADV.advect(q, *args)
        assert np.max(np.abs(got.cpu().numpy() * scale - ref)) < TOL * np.max(np.abs(ref))
        assert float(torch.sum(got)) == pytest.approx(float(torch.sum(src)), rel=1e-12)
    assert torch.all(on <= orho * (1 + 1e-12))
    s.close()


def test_gradients_through_advection_match_oracle_dense_adjoint():
    from paper_0908_2654_gb300.adjoint import ionized_fraction
    w = W.reionization_field(n=6, nsrc=2, box_mpc=14.4 * 6 / 256 / 20, ndot_total=4e49 / 20**3, dt_myr=0.3)
    nsteps = 2
    ndot = torch.tensor(np.asarray(w["src_ndot"], float), dtype=torch.float64, requires_grad=True)
    clump = torch.tensor(np.asarray(w["clump"], np.float32), requires_grad=True)
    J = ionized_fraction(ndot, clump, w, nsteps, precision="fp64", newton_tol=1e-11, lin_rtol=1e-12,
                         max_newton=60, max_lin=400, advect=True)
    J.backward()
    Jo, go_ndot, go_clump = OA.gradient(w, np.asarray(w["src_ndot"], float), np.asarray(w["clump"], float), nsteps,
                                        advect=True)
    assert float(J.detach()) == pytest.approx(Jo, rel=1e-9)
    np.testing.assert_allclose(ndot.grad.cpu().numpy(), go_ndot, rtol=1e-6)
    g = clump.grad.cpu().numpy()
    assert np.max(np.abs(g - go_clump)) <= 1e-6 * np.abs(go_clump).max()


def test_helium_species_move_with_the_same_fluxes():
    """On a helium grid n_HeI and n_HeII are advected like n_HI (oracle scheme, field by field),
    and stay within n_He of the advected density."""
    from paper_0908_2654_gb300 import _rt
    w = W.with_helium(W.random_state((8, 6, 10), seed=21, periodic=(True, False, True)))
    s = _solver(w)
    a = _scale_dt(s, w, 0.9)
    u = s.units
    out = [torch.empty_like(s.E) for _ in range(5)]
    dst = s.state(out[0], out[1], None, out[3], out[4])
    code, _ = _advect(s, s.state(), dst, rho=(s.rho, out[2]))
    _rt.check(code, "rt_advect")
    args = (w["v"], a, s.dt, w["dx"], w["periodic"])
    for got, q, scale in ((out[3], w["nHeI"], u.u_n), (out[4], w["nHeII"], u.u_n), (out[1], w["nHI"], u.u_n)):
        ref = ADV.advect(q, *args)
        assert np.max(np.abs(got.cpu().numpy() * scale - ref)) < TOL * np.max(np.abs(ref))
    nHe = 0.25 * w["Y"] * out[2]
    assert torch.all(out[3] + out[4] <= nHe * (1 + 1e-12)) and torch.all(out[3] >= 0) and torch.all(out[4] >= 0)
    s.close()
