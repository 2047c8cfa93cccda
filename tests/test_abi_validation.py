"""Host-side argument checking of the C ABI (include/rt.h), run without a GPU.

Every entry point checks its arguments before any CUDA call. An invalid descriptor,
invalid step inputs, null handles and out-of-range arguments must return RT_EINVAL with
a detail message, whether or not a device is present.

The checks that pass host pointers in place of device arrays run only where no GPU is
visible. There, a check that wrongly let them through would only fail with RT_ECUDA.
"""
import ctypes

import pytest

torch = pytest.importorskip("torch")

from paper_0908_2654_gb300 import _rt  # noqa: E402


@pytest.fixture(scope="module")
def L():
    import os
    if not os.path.exists(_rt.LIB_PATH):
        import importlib
        importlib.import_module("paper_0908_2654_gb300.build").build()
    try:
        return _rt.lib()
    except OSError as e:   # the CUDA runtime may be absent on a machine without a driver
        pytest.skip(f"library not loadable here: {e}")


def _desc(**kw):
    d = _rt.GridDesc()
    d.nx = d.ny = d.nz = 8
    d.dx = 1.0
    for k in range(6):
        d.bc[k] = _rt.RT_BC_PERIODIC
    d.u_x = d.u_t = d.u_g = 1.0
    d.theta = 0.51
    d.precision = _rt.RT_MIXED
    d.isothermal = 1
    d.T_iso = 1e4
    d.spectrum = _rt.RT_SPECTRUM_BLACKBODY
    d.T_B = 1e5
    d.recomb = _rt.RT_RECOMB_CONST
    d.cooling = 1
    d.limiter = _rt.RT_LIMITER_LAGGED
    d.E_min = 1e-35
    d.newton_tol, d.max_newton = 1e-8, 40
    d.lin_rtol, d.max_lin = 1e-3, 200
    d.mg_nu1 = d.mg_nu2 = 4
    for k, v in kw.items():
        if k == "bc":
            for i, b in enumerate(v):
                d.bc[i] = b
        else:
            setattr(d, k, v)
    return d


nan = float("nan")
BAD_DESCRIPTORS = [
    dict(nx=0), dict(nz=-4), dict(dx=0.0), dict(dx=-1.0), dict(dx=nan), dict(u_x=0.0), dict(u_t=nan),
    dict(u_g=-1.0), dict(theta=0.0), dict(theta=1.5), dict(theta=nan), dict(bc=(0, 0, 7, 7, 0, 0)),
    dict(bc=(0, 1, 0, 0, 0, 0)), dict(bc=(2, 0, 0, 0, 0, 0)), dict(bc=(0, 0, 0, 0, 1, -1)),
    dict(precision=5), dict(mg_nu1=0), dict(mg_nu2=0), dict(max_newton=0), dict(max_lin=0),
    dict(newton_tol=0.0), dict(newton_tol=nan), dict(lin_rtol=-1.0), dict(helium=2),
    dict(helium=1, Y=1.0), dict(helium=1, Y=-0.1), dict(helium=1, Y=nan),
    dict(nx=2048, ny=2048, nz=1024),     # 2^32 cells: above the 2^31 cell limit
]


@pytest.mark.parametrize("bad", BAD_DESCRIPTORS, ids=[",".join(f"{k}={v}" for k, v in b.items()) for b in BAD_DESCRIPTORS])
def test_init_grid_rejects_invalid_descriptor(L, bad):
    h = ctypes.c_void_p(0x1234)
    rc = L.rt_init_grid(ctypes.byref(_desc(**bad)), ctypes.byref(h))
    assert rc == _rt.RT_EINVAL
    assert not h.value                     # the output handle is cleared
    assert L.rt_last_error_detail().decode()


def test_init_grid_rejects_null_arguments(L):
    h = ctypes.c_void_p()
    assert L.rt_init_grid(None, ctypes.byref(h)) == _rt.RT_EINVAL
    assert L.rt_init_grid(ctypes.byref(_desc()), None) == _rt.RT_EINVAL


def test_null_grid_handle_is_rejected_by_every_entry_point(L):
    """Every entry point rejects a NULL grid with RT_EINVAL and records its own detail text
    (checked against a different error's text recorded just before)."""
    inp, st, st2 = _rt.StepInputs(), _rt.State(), _rt.State()
    stats = _rt.StepStats()
    r = ctypes.c_double()
    n = ctypes.c_int()
    B = ctypes.byref
    calls = {
        "rt_implicit_step": lambda: L.rt_implicit_step(None, B(inp), B(st), B(stats)),
        "rt_residual": lambda: L.rt_residual(None, B(inp), B(st), B(st2), None, None, None),
        "rt_residual_helium": lambda: L.rt_residual_helium(None, B(inp), B(st), B(st2), None, None, None, None,
                                                           None),
        "rt_schur_system": lambda: L.rt_schur_system(None, B(inp), B(st), B(st2), None, None, None, None, None),
        "rt_schur_solve": lambda: L.rt_schur_solve(None, None, None, 1e-6, 10, B(n)),
        "rt_adjoint_step": lambda: L.rt_adjoint_step(None, B(inp), B(st), B(st2), B(st), B(st2), None, None),
        "rt_advect": lambda: L.rt_advect(None, B(inp), B(st), B(st2), None, None, B(r)),
        "rt_advect_adjoint": lambda: L.rt_advect_adjoint(None, B(inp), B(st), B(st2)),
        "rt_fold_energy": lambda: L.rt_fold_energy(None, None, None),
        "rt_grey_constants": lambda: L.rt_grey_constants(None, B(r), None, None),
        "rt_set_profiling": lambda: L.rt_set_profiling(None, 1),
        "rt_get_profile": lambda: L.rt_get_profile(None, None, 0, B(n)),
    }
    for name, call in calls.items():
        assert L.rt_eval_elementary(9, None, None, 1, None) == _rt.RT_EINVAL
        marker = L.rt_last_error_detail().decode()
        assert call() == _rt.RT_EINVAL, name
        detail = L.rt_last_error_detail().decode()
        assert detail and detail != marker, name
    L.rt_destroy_grid(None)                # a no-op


def test_elementary_function_arguments(L):
    assert L.rt_eval_elementary(4, None, None, 1, None) == _rt.RT_EINVAL    # no function 4
    assert L.rt_eval_elementary(-1, None, None, 1, None) == _rt.RT_EINVAL
    assert L.rt_eval_elementary(0, None, None, -1, None) == _rt.RT_EINVAL
    assert L.rt_eval_elementary(0, None, None, 5, None) == _rt.RT_EINVAL    # n > 0 needs both arrays
    assert L.rt_eval_elementary(1, None, None, 0, None) == _rt.RT_OK        # empty input: nothing to do


def test_error_strings_are_distinct(L):
    codes = range(8)
    names = [L.rt_error_string(c).decode() for c in codes]
    assert len(set(names)) == len(names)
    assert L.rt_error_string(99).decode() == "unknown error"


no_gpu = pytest.mark.skipif(torch.cuda.is_available(), reason="passes host pointers in place of device arrays")


def _static_args(nsrc=0, a=1.0, dt=1.0, adot=0.0, rho=True):
    buf = (ctypes.c_double * 8)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    inp = _rt.StepInputs()
    inp.rho_b = p if rho else None
    inp.e_h = p
    inp.a, inp.dt, inp.adot = a, dt, adot
    inp.nsrc = nsrc
    st = _rt.State(p, p, p, None, None)
    return buf, inp, st


@no_gpu
@pytest.mark.parametrize("kw", [dict(a=0.0), dict(a=-1.0), dict(dt=0.0), dict(dt=nan), dict(adot=nan),
                                dict(adot=float("inf")), dict(nsrc=-1), dict(nsrc=3), dict(rho=False)],
                         ids=["a=0", "a<0", "dt=0", "dt=nan", "adot=nan", "adot=inf", "nsrc<0", "nsrc-no-list",
                              "no-rho"])
def test_step_inputs_are_checked_before_any_device_work(L, kw):
    buf, inp, st = _static_args(**kw)
    p = ctypes.cast(buf, ctypes.c_void_p)
    rc = L.rt_residual_static(ctypes.byref(_desc(nx=2, ny=2, nz=2)), ctypes.byref(inp), ctypes.byref(st),
                              ctypes.byref(st), p, p, p)
    assert rc == _rt.RT_EINVAL, L.rt_last_error_detail().decode()


@no_gpu
def test_static_residual_limits(L):
    buf, inp, st = _static_args()
    p = ctypes.cast(buf, ctypes.c_void_p)
    big = _desc(nx=64, ny=64, nz=16)       # 65536 cells: above the static scratch
    assert L.rt_residual_static(ctypes.byref(big), ctypes.byref(inp), ctypes.byref(st), ctypes.byref(st),
                                p, p, p) == _rt.RT_EINVAL
    he = _desc(nx=2, ny=2, nz=2, helium=1, Y=0.24)
    assert L.rt_residual_static(ctypes.byref(he), ctypes.byref(inp), ctypes.byref(st), ctypes.byref(st),
                                p, p, p) == _rt.RT_EINVAL
    assert L.rt_residual_static(ctypes.byref(_desc(nx=2, ny=2, nz=2)), ctypes.byref(inp), ctypes.byref(st),
                                ctypes.byref(st), p, None, p) == _rt.RT_EINVAL
    bad_theta = _desc(nx=2, ny=2, nz=2, theta=2.0)
    assert L.rt_residual_static(ctypes.byref(bad_theta), ctypes.byref(inp), ctypes.byref(st), ctypes.byref(st),
                                p, p, p) == _rt.RT_EINVAL


@pytest.mark.parametrize("spectrum,T_B", [("mono", 1e5), ("blackbody", 1e4), ("blackbody", 3e4), ("blackbody", 1e5),
                                          ("blackbody", 3e5), ("blackbody", 1e6)])
def test_library_grey_constants_match_oracle(L, spectrum, T_B):
    """The library's own host quadrature of the grey constants (Eq. grey_definition, composite
    Gauss-Legendre) against the oracle's adaptive quadrature, hydrogen and helium, through
    rt_spectrum_constants (no CUDA call)."""
    from oracle import spectrum as S
    out = (ctypes.c_double * 7)()
    code = _rt.RT_SPECTRUM_MONO if spectrum == "mono" else _rt.RT_SPECTRUM_BLACKBODY
    assert L.rt_spectrum_constants(code, T_B, out) == _rt.RT_OK
    h = S.grey_constants(spectrum, T_B)
    he = S.helium_grey_constants(spectrum, T_B)
    ref = [h["sigma_E"], h["sigma_G"], h["eps_src"], he["sigma_E_HeI"], he["sigma_G_HeI"], he["sigma_E_HeII"],
           he["sigma_G_HeII"]]
    for k, (got, want) in enumerate(zip(out, ref)):
        assert got == pytest.approx(want, rel=1e-11, abs=0.0), k


def test_spectrum_constants_arguments(L):
    out = (ctypes.c_double * 7)()
    assert L.rt_spectrum_constants(7, 1e5, out) == _rt.RT_EINVAL
    assert L.rt_spectrum_constants(_rt.RT_SPECTRUM_BLACKBODY, 0.0, out) == _rt.RT_EINVAL
    assert L.rt_spectrum_constants(_rt.RT_SPECTRUM_BLACKBODY, nan, out) == _rt.RT_EINVAL
    assert L.rt_spectrum_constants(_rt.RT_SPECTRUM_BLACKBODY, 1e5, None) == _rt.RT_EINVAL
