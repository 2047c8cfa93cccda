"""Hydrogen + helium grids on the GPU (k_assemble_he behind rt_residual_helium and
rt_implicit_step) against the oracle's hydrogen + helium step: element-wise residuals, whole
steps in both precisions, the reduction to the hydrogen-only grid at Y = 0, and a 64^3 field
whose result the oracle confirms as a root."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402
from oracle import helium as H  # noqa: E402
from oracle import model as M  # noqa: E402


def _reion(n=6):
    return W.with_helium(W.reionization_field(n=n, nsrc=max(2, n // 3), box_mpc=14.4 * n / 256,
                                              ndot_total=4e49 * (n / 6) ** 3, dt_myr=0.3))


CASES = [("reion6_he", _reion), ("stromgren8_he", lambda: W.with_helium(W.stromgren_static(n=8))),
         ("reion6_he_iso", lambda: dict(_reion(), isothermal=True, recomb="const"))]


def _solver(w, precision="fp64", **kw):
    from paper_0908_2654_gb300.solver import Solver
    return Solver(w, precision=precision, **kw)


def _scales(st, U):
    """Rounding scales of the five residual components: the local equations by their natural
    scales, f_E by the sum of the absolute values of its terms (a neighbour can be 1e25 times
    brighter than the cell, so the cell's own E is no scale for the diffusion term's rounding)."""
    e_c, nHI, nHeI, nHeII, E = U
    kap = M.opacity(st, nHI, (nHeI, nHeII))
    bE = M.explicit_part(st)
    adx2 = (st.a * st.dx) ** 2
    bound = np.zeros(st.shape)
    for d in range(3):
        ax = M._AXIS[d]
        f = M.face_D(st, E, kap, d) * (np.abs(np.roll(E, -1, axis=ax)) + np.abs(E)) / adx2
        bound += f + np.roll(f, 1, axis=ax)
    magE = np.abs(E) + np.abs(bE) + st.dt * st.theta * (bound + abs(st.adot / st.a) * np.abs(E)
                                                        + M.emissivity(st) + 2.998e10 * kap * np.abs(E))
    return (np.maximum(M.internal_energy_h(st), M.E_FLOOR_INT()), st.n_H, st.n_He, st.n_He, magE)


@pytest.mark.parametrize("name,make", CASES)
def test_residual_matches_oracle(name, make):
    w = make()
    st = H.Run(w).make_step()
    rng = np.random.default_rng(3)
    U = H.initial_iterate(st)
    # a state away from the root in every component
    U[1] = st.n_H * np.clip(U[1] / st.n_H * (1 + 0.1 * rng.standard_normal(st.shape)), 1e-6, 1.0)
    U[2] = st.n_He * rng.uniform(0.1, 0.6, st.shape)
    U[3] = st.n_He * rng.uniform(0.1, 0.3, st.shape)
    if not st.isothermal:
        U[0] = 0.01 * M.internal_energy_h(st) * rng.standard_normal(st.shape)
    f_ref = np.real(H.residual(st, U))
    s = _solver(w)
    f_gpu = s.residual_helium((st.E_n, st.nHI_n, st.nHeI_n, st.nHeII_n), U, a=st.a, adot=st.adot)
    s.close()
    for k, sc in enumerate(_scales(st, U)):
        err = np.max(np.abs(f_gpu[k] - f_ref[k]) / sc)
        assert err < 1e-11, (k, err)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name,make", CASES)
def test_step_matches_oracle(name, make, precision):
    w = make()
    run = H.Run(w)
    s = _solver(w, precision, newton_tol=1e-11, lin_rtol=1e-12, max_newton=60, max_lin=300)
    for _ in range(2):
        U, _ = run.advance(tol=1e-11)
        s.step()
        ec, nHI, nHeI, nHeII, E = s.state_cgs()
        st = run.make_step()
        assert np.max(np.abs(nHI - U[1]) / st.n_H) < 1e-9
        assert np.max(np.abs(nHeI - U[2]) / st.n_He) < 1e-9
        assert np.max(np.abs(nHeII - U[3]) / st.n_He) < 1e-9
        assert np.max(np.abs(E - U[4]) / np.maximum(np.abs(U[4]), M.weight_floor_E(st))) < 1e-8
    s.close()


def test_zero_helium_grid_reproduces_hydrogen_grid():
    w = W.reionization_field(n=8, nsrc=3, box_mpc=14.4 * 8 / 256, ndot_total=1e50, dt_myr=0.3)
    s0 = _solver(w, newton_tol=1e-11, lin_rtol=1e-12, max_newton=60, max_lin=300)
    s1 = _solver(W.with_helium(w, Y=0.0), newton_tol=1e-11, lin_rtol=1e-12, max_newton=60, max_lin=300)
    for _ in range(2):
        s0.step()
        s1.step()
    ec0, n0, E0 = s0.state_cgs()
    ec1, n1, h1, h2, E1 = s1.state_cgs()
    assert np.max(np.abs(n1 - n0) / (w["rho_b"] / 1.6735575e-24)) < 1e-10
    assert np.max(np.abs(E1 - E0) / np.maximum(np.abs(E0), 1e-35)) < 1e-8
    assert np.all(h1 == 0) and np.all(h2 == 0)
    s0.close()
    s1.close()


def test_field_64_mixed_is_a_root_and_keeps_helium_in_bounds():
    """The throughput workload's recipe at 64^3 (31 sources, dt = 1 Myr) with helium."""
    import bench
    w = W.with_helium(bench.workload(64))
    s = _solver(w, "mixed", newton_tol=1e-8, lin_rtol=1e-4)
    stats = s.step()
    ec, nHI, nHeI, nHeII, E = s.state_cgs()
    s.close()
    st = H.Run(w).make_step()
    U = np.stack([ec, nHI, nHeI, nHeII, E])
    f = np.real(H.residual(st, U))
    assert H.rms(H.weights(st, U), f) <= 1e-8, stats
    assert np.all(nHeI >= 0) and np.all(nHeII >= 0) and np.all(nHeI + nHeII <= st.n_He * (1 + 1e-12))
    assert np.min(nHeI / st.n_He) < 0.5                  # the sources ionise helium


def test_grid_destroy_returns_device_memory():
    """rt_destroy_grid releases the whole workspace, the helium species buffers included
    (100 MB of them per grid at 128^3): hydrogen and hydrogen + helium grids created and
    destroyed three times leave the free device memory where it was."""
    import ctypes
    from paper_0908_2654_gb300 import _rt
    L = _rt.lib()
    for w in (W.stromgren_static(n=128), W.with_helium(W.stromgren_static(n=128))):
        s = _solver(w, "mixed")
        d = s.desc
        s.close()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(3):
            h = ctypes.c_void_p()
            _rt.check(L.rt_init_grid(ctypes.byref(d), ctypes.byref(h)), "rt_init_grid")
            L.rt_destroy_grid(h)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] >= free0 - (16 << 20), w.get("helium", False)
