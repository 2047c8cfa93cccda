"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Element-wise comparisons on seeded inputs at sizes the oracle finishes in seconds
(several tiles, ragged shapes, periodic, reflecting and outflow faces, both precisions).
Tolerances:
  * residual and Schur system at a given iterate: 1e-11 relative to the size of the
    terms that make up each entry (both sides evaluate the same FP64 formulas; the
    difference is rounding order);
  * converged steps, both sides converged to 1e-12 in the component-scaled norm of the
    method (Eq. rmsnorm weights) so that the difference measures the implementations, not
    the stopping test:
      - 1e-10 relative on E in every cell whose E is above the norm's floor
        (max(E_min, 1e-12 of the brightest cell): below it a cell's E is round-off of the
        bright cells' arithmetic), on x_HI relative to max(x_HI, 1e-4) (the stopping test
        scales f_n by n_H, so n_HI is resolved to about the tolerance times n_H), and on e_c
        relative to the hydro state's internal energy;
      - 1e-9 in the component-scaled norm on every cell (floor cells included).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402
from oracle import driver  # noqa: E402
from oracle import model as M  # noqa: E402
from oracle import newton as N  # noqa: E402


def _solver(w, precision="fp64", **kw):
    from paper_0908_2654_gb300.solver import Solver
    return Solver(w, precision=precision, **kw)


def _perturbed_iterate(st, seed):
    rng = np.random.default_rng(seed)
    U = N.initial_iterate(st)
    U[2] = st.E_n * (1.0 + 0.3 * rng.standard_normal(st.shape)) + 1e-3 * st.E_n.mean() * rng.random(st.shape)
    U[1] = st.n_H * np.clip(st.nHI_n / st.n_H * (1 + 0.2 * rng.standard_normal(st.shape)), 1e-6, 1.0)
    if not st.isothermal:
        U[0] = 1e-3 * M.internal_energy_h(st) * rng.standard_normal(st.shape)
    return U


def _magnitude_E(st, U, bE):
    """Sum of absolute values of the terms of f_E (the scale of its rounding error)."""
    E = U[2]
    kap = M.opacity(st, U[1])
    Ld = np.abs(M.diffusion(st, np.abs(E), kap)) + 12 * np.abs(E) * 0
    # bound the diffusion term by sum_faces w (|E_nb| + |E|)
    adx2 = (st.a * st.dx) ** 2
    bound = np.zeros(st.shape)
    for d in range(3):
        ax = M._AXIS[d]
        D = M.face_D(st, E, kap, d)
        f = D * (np.abs(np.roll(E, -1, axis=ax)) + np.abs(E)) / adx2
        bound += f + np.roll(f, 1, axis=ax)
    del Ld
    return (np.abs(E) + np.abs(bE) + st.dt * st.theta * (bound + abs(st.adot / st.a) * np.abs(E)
                                                         + M.emissivity(st) + 2.998e10 * kap * np.abs(E)))


CASES = [
    ("stromgren16", lambda: W.stromgren_static(n=16)),
    ("random_outflow_faces", lambda: W.random_state((11, 9, 6), seed=6, isothermal=False,
                                                    bc=("outflow", "outflow", "reflect", "outflow",
                                                        "periodic", "periodic"))),
    ("reion_16_periodic", lambda: W.reionization_field(n=16, nsrc=4, box_mpc=14.4 * 16 / 256,
                                                       ndot_total=1e52 * (16 / 256) ** 3)),
    ("random_ragged_walls", lambda: W.random_state((12, 10, 7), seed=3, periodic=(False, True, False),
                                                   isothermal=False)),
    ("random_iso_periodic", lambda: W.random_state((9, 6, 5), seed=4, isothermal=True)),
]


@pytest.mark.parametrize("name,make", CASES)
def test_residual_matches_oracle(name, make):
    w = make()
    r = driver.Run(w)
    st = r.make_step()
    bE = M.explicit_part(st)
    U = _perturbed_iterate(st, 11)
    f_ref = M.residual(st, U, bE)
    s = _solver(w)
    f_gpu = s.residual((st.E_n, st.nHI_n), U)
    s.close()
    mag = _magnitude_E(st, U, bE)
    assert np.max(np.abs(f_gpu[2] - f_ref[2]) / mag) < 1e-11
    # local equations: scale n_H and the specific internal energy
    assert np.max(np.abs(f_gpu[1] - f_ref[1]) / st.n_H) < 1e-12
    se = np.maximum(M.internal_energy_h(st), M.E_FLOOR_INT()) + np.abs(U[0]) + np.abs(f_ref[0])
    assert np.max(np.abs(f_gpu[0] - f_ref[0]) / se) < 1e-11


@pytest.mark.parametrize("name,make", CASES)
def test_schur_system_matches_oracle(name, make):
    w = make()
    r = driver.Run(w)
    st = r.make_step()
    bE = M.explicit_part(st)
    U = _perturbed_iterate(st, 12)
    S, rhs = N.schur_system(st, U, bE)
    s = _solver(w)
    d, wx, wy, wz, rg = s.schur_system((st.E_n, st.nHI_n), U)
    s.close()
    Sd = S.diagonal().reshape(st.shape)
    scale = np.abs(Sd) + np.abs(S).sum(axis=1).A.reshape(st.shape)
    assert np.max(np.abs(d - Sd) / scale) < 1e-11
    # off-diagonal couplings: S[i, i+x] = -wx_i on interior faces
    z, y, x = np.indices(st.shape)
    flat = np.arange(st.N).reshape(st.shape)
    for wgpu, ax, n, per in ((wx, 2, st.nx, st.periodic[0]), (wy, 1, st.ny, st.periodic[1]),
                             (wz, 0, st.nz, st.periodic[2])):
        nb = np.roll(flat, -1, axis=ax)
        last = [slice(None)] * 3
        last[ax] = -1
        mask = np.ones(st.shape, bool)
        if not per:
            mask[tuple(last)] = False
        if n < 3 and per:
            continue
        ref = -np.asarray(S[flat[mask], nb[mask]]).ravel()
        assert np.allclose(wgpu[mask], ref, rtol=1e-12, atol=1e-14 * scale.max())
        if not per:
            assert np.all(wgpu[tuple(last)] == 0.0)
    mag = _magnitude_E(st, U, bE) * (1 + np.abs(Sd))
    assert np.max(np.abs(rg - rhs.reshape(st.shape)) / mag) < 1e-11


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name,make", [CASES[0], CASES[1], CASES[2],
                                       ("stromgren32_multilevel", lambda: W.stromgren_static(n=32, dt_over_trec=2e-3))])
def test_schur_solve_matches_direct_solve(name, make, precision):
    import scipy.sparse.linalg as spla
    if name not in _SOLVE_CACHE:
        w = make()
        st = driver.Run(w).make_step()
        U = N.local_solve(st, N.initial_iterate(st))
        S, _ = N.schur_system(st, U)
        b = np.random.default_rng(5).standard_normal(st.N)
        _SOLVE_CACHE[name] = (w, st, U, S, b, spla.spsolve(S.tocsc(), b))
    w, st, U, S, b, x_ref = _SOLVE_CACHE[name]
    s = _solver(w, precision=precision)
    s.schur_system((st.E_n, st.nHI_n), U)
    x_gpu, its = s.schur_solve(b.reshape(st.shape), rtol=1e-12, max_iters=300)
    s.close()
    err = np.max(np.abs(x_gpu.ravel() - x_ref)) / np.max(np.abs(x_ref))
    assert err < 1e-9, (err, its)
    assert its < 100


def test_schur_solve_is_deterministic_on_odd_periodic_axes():
    """On periodic axes of odd length two neighbouring cells share a colour; the coarse solver
    updates each colour from the old values of all cells, so repeated solves agree bit for bit
    (same iterations, same result)."""
    w = W.random_state((9, 6, 5), seed=4, isothermal=True)
    st = driver.Run(w).make_step()
    U = N.local_solve(st, N.initial_iterate(st))
    b = np.random.default_rng(9).standard_normal(st.shape)
    out = []
    for precision in ("fp64", "mixed"):
        s = _solver(w, precision=precision)
        s.schur_system((st.E_n, st.nHI_n), U)
        runs = [s.schur_solve(b, rtol=1e-12, max_iters=300) for _ in range(3)]
        s.close()
        for x, its in runs[1:]:
            assert its == runs[0][1] and np.array_equal(x, runs[0][0]), precision
        out.append(runs[0][0])
    np.testing.assert_allclose(out[0], out[1], rtol=1e-9, atol=1e-9 * np.abs(out[0]).max())


_SOLVE_CACHE = {}
_STEP_CACHE = {}


def _oracle_run(name, w, nsteps, tol):
    """Oracle trajectory (step data and converged state per step), computed once per case."""
    if name not in _STEP_CACHE:
        r = driver.Run(w)
        traj = []
        for _ in range(nsteps):
            st = r.make_step()
            U, _ = r.advance(tol=tol)
            traj.append((st, U, r.e_h.copy()))
        _STEP_CACHE[name] = traj
    return _STEP_CACHE[name]


def _floor_E(st):
    """The residual norm's E floor of a step: max(E_min, 1e-12 max(E^n + dt 4 pi eta))."""
    return M.weight_floor_E(st)


def _compare(st, U, ec, n, E, worst):
    """Fold the differences of a GPU state (ec, n, E) from the oracle's root U into worst."""
    wE = 1.0 / np.maximum(np.maximum(np.abs(U[2]), st.E_n), st.E_min)
    worst["E"] = max(worst["E"], float(np.max(np.abs(E - U[2]) * wE)))
    worst["n"] = max(worst["n"], float(np.max(np.abs(n - U[1]) / st.n_H)))
    se = np.maximum(M.internal_energy_h(st), M.E_FLOOR_INT())
    worst["e"] = max(worst["e"], float(np.max(np.abs(ec - U[0]) / se)))
    bright = np.abs(U[2]) > _floor_E(st)
    if np.any(bright):
        worst["E_rel"] = max(worst["E_rel"], float(np.max(np.abs(E - U[2])[bright] / np.abs(U[2])[bright])))
    # x_HI relative to itself down to x_HI = 1e-4: the stopping test scales f_n by n_H, so the
    # attainable relative accuracy of n_HI is about the tolerance over x_HI
    worst["x_rel"] = max(worst["x_rel"], float(np.max(np.abs(n - U[1]) / np.maximum(U[1], 1e-4 * st.n_H))))


def _step_both(name, w, nsteps, precision, tol=1e-12, reset=True):
    """GPU steps against the oracle's trajectory; with reset=True both continue from the
    oracle's state after every step (errors do not compound), otherwise the GPU runs on its own
    state for the whole trajectory."""
    traj = _oracle_run(name, w, nsteps, tol)
    s = _solver(w, precision=precision, newton_tol=tol, lin_rtol=1e-12, max_newton=60, max_lin=300)
    worst = {"E": 0.0, "n": 0.0, "e": 0.0, "E_rel": 0.0, "x_rel": 0.0}
    for st, U, e_h_next in traj:
        try:
            stats = s.step()
        except RuntimeError as e:
            raise AssertionError(f"{e}; history {getattr(e, 'stats', None)}") from e
        ec, n, E = s.state_cgs()
        _compare(st, U, ec, n, E, worst)
        if reset:
            s.E.copy_(torch.as_tensor(U[2] / s.units.u_E))
            s.nHI.copy_(torch.as_tensor(U[1] / s.units.u_n))
            if not w["isothermal"]:
                s.e_h.copy_(torch.as_tensor(e_h_next / s.units.u_v**2))
    s.close()
    return worst, stats


def _assert_parity(worst, stats):
    assert worst["E_rel"] < 1e-10 and worst["x_rel"] < 1e-10 and worst["e"] < 1e-10, (worst, stats)
    assert worst["E"] < 1e-9 and worst["n"] < 1e-9, (worst, stats)


STEP_CASES = [
    ("stromgren8", lambda: W.stromgren_static(n=8), 3),
    ("stromgren16", lambda: W.stromgren_static(n=16), 2),
    ("stromgren_ragged_24x20x12", lambda: W.stromgren_static(n=(24, 20, 12)), 2),
    ("stromgren16_walls", lambda: W.stromgren_static(n=16, bc=("reflect",) * 6), 2),
    ("cosmo16", lambda: W.stromgren_cosmo(n=16, z0=10.0, z_end=9.0, nsteps=4), 2),
    ("reion16", lambda: W.reionization_field(n=16, nsrc=4, box_mpc=14.4 * 16 / 256,
                                             ndot_total=1e52 * (16 / 256) ** 3), 2),
    ("reion16_theta051_small_dt", lambda: W.reionization_field(n=16, nsrc=4, box_mpc=14.4 * 16 / 256,
                                                               ndot_total=1e52 * (16 / 256) ** 3,
                                                               dt_myr=0.1, theta=0.51), 2),
    ("reion_ragged_20x12x16", lambda: W.reionization_field(n=(20, 12, 16), nsrc=3, box_mpc=14.4 * 20 / 256,
                                                           ndot_total=1e52 * (20 * 12 * 16 / 256**3)), 1),
    ("random_outflow_mixed_faces", lambda: W.random_state(
        (10, 9, 8), seed=8, isothermal=False, dt_myr=0.01,
        bc=("outflow", "reflect", "periodic", "periodic", "outflow", "outflow")), 1),
]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name,make,nsteps", STEP_CASES)
def test_implicit_step_matches_oracle(name, make, nsteps, precision):
    w = make()
    worst, stats = _step_both(name, w, nsteps, precision)
    _assert_parity(worst, stats)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_deep_multigrid_step_matches_oracle(precision):
    """A 40 x 40 x 24 Stromgren step: both multigrid precisions keep two global-memory levels
    (38400 and 4800 cells) above the single-CTA coarse solver, so the FP32 V-cycle's restriction,
    prolongation and smoothing run on levels of their own before the tail."""
    w = W.stromgren_static(n=(40, 40, 24), dt_over_trec=1e-3)
    worst, stats = _step_both("stromgren_deep_40x40x24", w, 1, precision)
    _assert_parity(worst, stats)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_static_stromgren_16_twenty_step_trajectory(precision):
    """The 16^3 static Stromgren configuration over its 20 steps of 0.01 t_rec, the GPU
    advancing its own state (no reset to the oracle's between steps)."""
    w = W.stromgren_static(n=16, nsteps=20)
    worst, stats = _step_both("stromgren16_trajectory20", w, 20, precision, reset=False)
    _assert_parity(worst, stats)


DEGENERATE = [((1, 1, 5), True), ((5, 1, 1), True), ((2, 2, 2), False), ((2, 2, 2), True), ((1, 4, 3), True),
              ((4, 3, 3), False)]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("shape,sources", DEGENERATE)
def test_degenerate_grid_steps_match_oracle(shape, sources, precision):
    """One-cell-thin grids, the 2^3 grid and steps without any source, two steps each, with the
    Stromgren gas (reflecting lower, outflow upper faces) in cells of the 16^3 configuration's
    width."""
    w = W.stromgren_static(n=shape, dt_over_trec=5e-3, box_kpc=6.6 * shape[0] / 16)
    if not sources:
        w["src_index"] = np.array([], np.int64)
        w["src_ndot"] = np.array([])
        w["E"] = np.full(w["E"].shape, 1e-20)        # something to lose through the outflow faces
    worst, stats = _step_both(f"degenerate_{shape}_{sources}", w, 2, precision, reset=False)
    _assert_parity(worst, stats)
