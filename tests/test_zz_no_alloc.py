"""The allocation-free residual entry point against the allocating one.

rt_residual_static serves callers that cannot allocate device memory (an application that
owns the whole device memory budget, work issued during stream capture): its scratch is a
fixed device array inside the library.  This test calls it through the C ABI and checks its
output against rt_residual's on the same inputs, twice in a row (the array keeps the first
call's contents, which the second call must not depend on).  Collected last so that a run
stopping at the first failure has run every other test already.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402
from oracle import driver  # noqa: E402


def _static_residual(s, U_n, U):
    from paper_0908_2654_gb300 import _rt
    u = s.units
    En, nn = s.to_device(U_n[0], u.u_E), s.to_device(U_n[1], u.u_n)
    ec, n, E = s.to_device(U[0], u.u_v**2), s.to_device(U[1], u.u_n), s.to_device(U[2], u.u_E)
    fe, fn, fE = (torch.full_like(E, float("nan")) for _ in range(3))
    inp = s.inputs()
    s0, s1 = s.state(En, nn, torch.zeros_like(En)), s.state(E, n, ec)
    code = _rt.lib().rt_residual_static(ctypes.byref(s.desc), ctypes.byref(inp), ctypes.byref(s0),
                                        ctypes.byref(s1), _rt.ptr(fe), _rt.ptr(fn), _rt.ptr(fE))
    _rt.check(code, "rt_residual_static")
    return np.stack([fe.cpu().numpy() * u.u_v**2, fn.cpu().numpy() * u.u_n, fE.cpu().numpy() * u.u_E])


@pytest.mark.parametrize("make", [
    lambda: W.random_state((12, 10, 7), seed=3, periodic=(False, True, False), isothermal=False),
    lambda: W.stromgren_static(n=16),
])
def test_static_residual_matches_rt_residual_twice(make):
    from paper_0908_2654_gb300.solver import Solver
    w = make()
    st = driver.Run(w).make_step()
    rng = np.random.default_rng(7)
    U = np.stack([1e8 * rng.standard_normal(st.shape) * (0 if w["isothermal"] else 1),
                  st.nHI_n * (1 + 0.1 * rng.random(st.shape)).clip(0, 1 / (st.nHI_n / st.n_H).max()),
                  st.E_n * (1 + 0.3 * rng.random(st.shape))])
    s = Solver(w, precision="fp64")
    ref = s.residual((st.E_n, st.nHI_n), U)
    for _ in range(2):
        got = _static_residual(s, (st.E_n, st.nHI_n), U)
        scale = np.abs(ref) + np.abs(U) * 0 + 1e-300
        assert np.all(np.isfinite(got))
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)
        # a different state in between must not leak into the next call
        _static_residual(s, (st.E_n * 2, st.nHI_n), U)
    s.close()


def test_static_residual_rejects_oversized_grid():
    from paper_0908_2654_gb300 import _rt
    from paper_0908_2654_gb300.solver import Solver
    w = W.stromgren_static(n=16)
    s = Solver(w, precision="fp64")
    d = _rt.GridDesc.from_buffer_copy(s.desc)
    d.nx = d.ny = d.nz = 40   # 64000 cells > 32768
    st = s.state()
    inp = s.inputs()
    code = _rt.lib().rt_residual_static(ctypes.byref(d), ctypes.byref(inp), ctypes.byref(st), ctypes.byref(st),
                                        _rt.ptr(s.ec), _rt.ptr(s.ec), _rt.ptr(s.ec))
    s.close()
    assert code == _rt.RT_EINVAL
