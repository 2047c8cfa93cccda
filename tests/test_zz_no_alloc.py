"""The allocation-free residual entry point against the allocating one.

rt_residual_static serves callers that cannot allocate device memory (an application that
owns the whole device memory budget through its own pool allocator, or a loop that must not
take the synchronisation an allocation can cause): its scratch is a fixed device array inside
the library.  These tests call it through the C ABI and check
  * its output against rt_residual's on the same inputs, twice in a row (the array keeps the
    first call's contents, which the second call must not depend on);
  * that a call changes the device's free memory by nothing (no allocation of any kind);
  * that the calling thread's current device is the same after the call;
  * that oversized grids and device ordinals outside the supported range are rejected.
Collected last so that a run stopping at the first failure has run every other test already.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402
from oracle import driver  # noqa: E402


def _prepare(s, U_n, U):
    """Device inputs and outputs of one call, all allocated before the call."""
    u = s.units
    En, nn = s.to_device(U_n[0], u.u_E), s.to_device(U_n[1], u.u_n)
    ec, n, E = s.to_device(U[0], u.u_v**2), s.to_device(U[1], u.u_n), s.to_device(U[2], u.u_E)
    out = [torch.full_like(E, float("nan")) for _ in range(3)]
    keep = (En, nn, ec, n, E, torch.zeros_like(En))
    return dict(inp=s.inputs(), s0=s.state(En, nn, keep[5]), s1=s.state(E, n, ec), out=out, keep=keep)


def _call(s, c):
    from paper_0908_2654_gb300 import _rt
    fe, fn, fE = c["out"]
    return _rt.lib().rt_residual_static(ctypes.byref(s.desc), ctypes.byref(c["inp"]), ctypes.byref(c["s0"]),
                                        ctypes.byref(c["s1"]), _rt.ptr(fe), _rt.ptr(fn), _rt.ptr(fE))


def _to_cgs(s, c):
    u = s.units
    fe, fn, fE = c["out"]
    return np.stack([fe.cpu().numpy() * u.u_v**2, fn.cpu().numpy() * u.u_n, fE.cpu().numpy() * u.u_E])


@pytest.mark.parametrize("make", [
    lambda: W.random_state((12, 10, 7), seed=3, periodic=(False, True, False), isothermal=False),
    lambda: W.stromgren_static(n=16),
])
def test_static_residual_matches_rt_residual_twice(make):
    from paper_0908_2654_gb300 import _rt
    from paper_0908_2654_gb300.solver import Solver
    w = make()
    st = driver.Run(w).make_step()
    rng = np.random.default_rng(7)
    U = np.stack([1e8 * rng.standard_normal(st.shape) * (0 if w["isothermal"] else 1),
                  st.nHI_n * (1 + 0.1 * rng.random(st.shape)).clip(0, 1 / (st.nHI_n / st.n_H).max()),
                  st.E_n * (1 + 0.3 * rng.random(st.shape))])
    s = Solver(w, precision="fp64")
    ref = s.residual((st.E_n, st.nHI_n), U)
    same = _prepare(s, (st.E_n, st.nHI_n), U)
    other = _prepare(s, (st.E_n * 2, st.nHI_n), U)
    _rt.check(_call(s, same), "rt_residual_static")          # first call: per-device set-up
    torch.cuda.synchronize()
    for _ in range(2):
        free0 = torch.cuda.mem_get_info(s.dev)[0]
        _rt.check(_call(s, same), "rt_residual_static")
        free1 = torch.cuda.mem_get_info(s.dev)[0]
        assert free1 == free0, "the call changed the device's free memory"
        got = _to_cgs(s, same)
        assert np.all(np.isfinite(got))
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)
        # a different state in between must not leak into the next call
        _rt.check(_call(s, other), "rt_residual_static")
    s.close()


def test_static_residual_restores_current_device():
    from paper_0908_2654_gb300 import _rt
    from paper_0908_2654_gb300.solver import Solver
    w = W.stromgren_static(n=8)
    st = driver.Run(w).make_step()
    s = Solver(w, precision="fp64")
    c = _prepare(s, (st.E_n, st.nHI_n), (np.zeros(st.shape), st.nHI_n, st.E_n))
    before = torch.cuda.current_device()
    _rt.check(_call(s, c), "rt_residual_static")
    assert torch.cuda.current_device() == before
    s.close()


def test_static_residual_rejects_oversized_grid_and_bad_device():
    from paper_0908_2654_gb300 import _rt
    from paper_0908_2654_gb300.solver import Solver
    w = W.stromgren_static(n=16)
    s = Solver(w, precision="fp64")
    st = s.state()
    inp = s.inputs()
    for field, value in (("nx", 40), ("device", 64), ("device", -1)):
        d = _rt.GridDesc.from_buffer_copy(s.desc)
        if field == "nx":
            d.nx = d.ny = d.nz = value      # 64000 cells > 32768
        else:
            d.device = value
        code = _rt.lib().rt_residual_static(ctypes.byref(d), ctypes.byref(inp), ctypes.byref(st), ctypes.byref(st),
                                            _rt.ptr(s.ec), _rt.ptr(s.ec), _rt.ptr(s.ec))
        assert code == _rt.RT_EINVAL, (field, value)
    s.close()
