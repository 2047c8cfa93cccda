"""Full-size checks in the configuration bench.py times, and error paths of the C ABI.

* 256^3 reionization field, mixed precision, the bench's tolerances: the oracle evaluates
  its own residual f(U) at the GPU's converged state (a property that holds at any size:
  the returned state is a root to the requested tolerance) and re-solves the cell-local
  equations at sampled cells.
* 128^3 static Stromgren sphere (FP64): the I-front follows the closed form.
* Error paths: invalid shapes and sources, non-finite input, too few Newton iterations;
  the caller's state must be untouched on error.
"""

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
from oracle import newton as N  # noqa: E402


def test_bench_configuration_256_root_and_sampled_local_solutions():
    import bench
    from paper_0908_2654_gb300.solver import Solver
    w = bench.workload(256)
    s = Solver(w, precision="mixed", newton_tol=1e-6, lin_rtol=1e-3)
    stats = s.step()
    ec, n, E = s.state_cgs()
    s.close()
    run = driver.Run(w)
    st = run.make_step()
    U = np.stack([ec, n, E])
    f = M.residual(st, U)
    # the GPU's stopping test uses the same component scaling with E weights at its own iterate
    nrm = M.rms_norm(M.weights(st, U), f)
    assert nrm <= 1e-6, (nrm, stats)
    # cell-local equations at sampled cells, solved by the oracle from scratch at the GPU's E
    rng = np.random.default_rng(0)
    idx = rng.choice(st.N, size=64, replace=False)
    idx = np.concatenate([idx, np.asarray(w["src_index"][:16])])
    fe, fn = M.local_residual(st, U[0], U[1], U[2])
    scale_e = np.maximum(M.internal_energy_h(st), M.E_FLOOR_INT()).ravel()[idx]
    assert np.max(np.abs(fe.ravel()[idx]) / scale_e) < 1e-8
    assert np.max(np.abs(fn.ravel()[idx]) / st.n_H.ravel()[idx]) < 1e-8


def test_stromgren_128_front_follows_closed_form():
    from paper_0908_2654_gb300.solver import Solver
    w = W.stromgren_static(n=128, nsteps=20)
    s = Solver(w, precision="fp64", newton_tol=1e-8, lin_rtol=1e-6, max_newton=60)
    for _ in range(w["nsteps"]):
        s.step()
    ec, n, E = s.state_cgs()
    g = s.grey()
    s.close()
    neff = w["ndot_total"] * g["eps_src"] * g["sigma_G"] / g["sigma_E"]
    rI = D.ifront_radius(n, w["rho_b"] / K.M_H, w["dx"], True)
    rth = C.static_ifront(w["nsteps"] * w["dt"], neff, K.ALPHA_B_PAPER, w["nH"])
    assert rI == pytest.approx(rth, rel=0.08)


def _solver_small():
    from paper_0908_2654_gb300.solver import Solver
    return Solver(W.stromgren_static(n=8), precision="fp64", newton_tol=1e-10, lin_rtol=1e-10)


def test_empty_source_list_steps():
    from paper_0908_2654_gb300.solver import Solver
    w = W.stromgren_static(n=8)
    w["src_index"] = np.array([], np.int64)
    w["src_ndot"] = np.array([])
    s = Solver(w, precision="mixed", newton_tol=1e-10, lin_rtol=1e-10)
    E0 = s.E.clone()
    s.step()
    ec, n, E = s.state_cgs()
    s.close()
    assert np.all(np.isfinite(E)) and np.all(n > 0)
    # no emission: the radiation floor can only decay
    assert float(torch.max(s.E)) <= float(torch.max(E0)) * (1 + 1e-12)


def test_out_of_range_source_is_rejected_and_state_kept():
    from paper_0908_2654_gb300 import _rt
    s = _solver_small()
    s.src_cell[0] = 10**6
    E0, n0 = s.E.clone(), s.nHI.clone()
    with pytest.raises(_rt.RTError) as e:
        s.step()
    assert e.value.code == _rt.RT_EINVAL
    assert torch.equal(s.E, E0) and torch.equal(s.nHI, n0)
    s.close()


def test_non_finite_input_is_rejected_and_state_kept():
    from paper_0908_2654_gb300 import _rt
    s = _solver_small()
    s.E[0, 0, 1] = float("nan")
    E0, n0 = s.E.clone(), s.nHI.clone()
    with pytest.raises(_rt.RTError) as e:
        s.step()
    assert e.value.code == _rt.RT_ENONFINITE
    assert torch.equal(torch.nan_to_num(s.E), torch.nan_to_num(E0)) and torch.equal(s.nHI, n0)
    s.close()


@pytest.mark.parametrize("field,value", [("rho", 0.0), ("rho", -1.0), ("rho", float("nan")), ("e_h", float("nan")),
                                         ("e_h", -1e3)])
def test_invalid_hydro_state_is_rejected_and_state_kept(field, value):
    """The hydro state handed over by the operator split is checked on the device before any
    state is touched: density positive and finite, energy finite, internal energy of
    non-isothermal gas positive."""
    from paper_0908_2654_gb300 import _rt
    from paper_0908_2654_gb300.solver import Solver
    w = W.random_state((8, 6, 4), seed=2, isothermal=False)
    s = Solver(w, precision="fp64", newton_tol=1e-10, lin_rtol=1e-10)
    getattr(s, field)[1, 2, 3] = value if field == "rho" or value != value else value * float(s.e_h.abs().max())
    E0, n0 = s.E.clone(), s.nHI.clone()
    with pytest.raises(_rt.RTError) as e:
        s.step()
    assert e.value.code == _rt.RT_EINVAL and "hydro state" in str(e.value)
    assert torch.equal(s.E, E0) and torch.equal(s.nHI, n0)
    s.close()


def test_newton_iteration_cap_reports_no_convergence_and_keeps_state():
    from paper_0908_2654_gb300 import _rt
    from paper_0908_2654_gb300.solver import Solver
    s = Solver(W.stromgren_static(n=8), precision="fp64", newton_tol=1e-14, lin_rtol=1e-10, max_newton=1)
    E0, n0 = s.E.clone(), s.nHI.clone()
    with pytest.raises(_rt.RTError) as e:
        s.step()
    assert e.value.code == _rt.RT_ENOCONV
    assert e.value.stats["newton_iters"] == 1
    assert torch.equal(s.E, E0) and torch.equal(s.nHI, n0)
    s.close()


def test_unsupported_shape_is_rejected():
    from paper_0908_2654_gb300 import _rt
    from paper_0908_2654_gb300.solver import Solver
    w = W.random_state((65, 64, 64), seed=1)     # odd dimension on a level above the coarse bound
    with pytest.raises(_rt.RTError) as e:
        Solver(w, precision="mixed")
    assert e.value.code == _rt.RT_EINVAL
