"""ctypes binding of the C ABI in include/rt.h (argument marshalling only).

Loads the in-tree library ``lib/librtfld.so``; a missing library is an error (there is
no fallback).  Tensors passed to the wrappers must be contiguous CUDA tensors of the
documented dtype; their device pointers go straight to the library.
"""
import ctypes
import os

# imported before the library is loaded: the process's CUDA runtime is then the one PyTorch
# loads, and the library binds to that same libcudart
import torch  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "librtfld.so")

RT_OK, RT_EINVAL, RT_ENOMEM, RT_ECUDA, RT_ENOCONV, RT_ELINESEARCH, RT_ENONFINITE, RT_ELINEAR = range(8)
RT_BC_PERIODIC, RT_BC_REFLECT, RT_BC_OUTFLOW = 0, 1, 2
RT_BC_WALL = RT_BC_REFLECT
RT_FP64, RT_MIXED = 0, 1
RT_SPECTRUM_MONO, RT_SPECTRUM_BLACKBODY = 0, 1
RT_RECOMB_CONST, RT_RECOMB_HG97 = 0, 1
RT_LIMITER_LAGGED, RT_LIMITER_CONST = 0, 1


class GridDesc(ctypes.Structure):
    """rt_grid_desc: grid shape, units, physics switches and solver parameters."""

    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dx", ctypes.c_double),
        ("bc", ctypes.c_int * 6),
        ("u_x", ctypes.c_double), ("u_t", ctypes.c_double), ("u_g", ctypes.c_double),
        ("theta", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("isothermal", ctypes.c_int), ("T_iso", ctypes.c_double),
        ("spectrum", ctypes.c_int), ("T_B", ctypes.c_double),
        ("recomb", ctypes.c_int), ("cooling", ctypes.c_int), ("helium", ctypes.c_int), ("Y", ctypes.c_double),
        ("limiter", ctypes.c_int), ("D_const", ctypes.c_double),
        ("E_min", ctypes.c_double),
        ("newton_tol", ctypes.c_double), ("max_newton", ctypes.c_int),
        ("lin_rtol", ctypes.c_double), ("max_lin", ctypes.c_int),
        ("mg_nu1", ctypes.c_int), ("mg_nu2", ctypes.c_int),
        ("device", ctypes.c_int), ("stream", ctypes.c_void_p),
    ]


class StepInputs(ctypes.Structure):
    """rt_step_inputs: the hydro state, expansion and sources of one step (device pointers)."""

    _fields_ = [
        ("rho_b", ctypes.c_void_p), ("e_h", ctypes.c_void_p),
        ("vx", ctypes.c_void_p), ("vy", ctypes.c_void_p), ("vz", ctypes.c_void_p),
        ("clump", ctypes.c_void_p),
        ("a", ctypes.c_double), ("adot", ctypes.c_double), ("dt", ctypes.c_double),
        ("nsrc", ctypes.c_int),
        ("src_cell", ctypes.c_void_p), ("src_ndot", ctypes.c_void_p),
    ]


class State(ctypes.Structure):
    """rt_state: E, n_HI, e_c (and n_HeI, n_HeII on helium grids), device pointers."""

    _fields_ = [("E", ctypes.c_void_p), ("n_HI", ctypes.c_void_p), ("e_c", ctypes.c_void_p),
                ("n_HeI", ctypes.c_void_p), ("n_HeII", ctypes.c_void_p)]


class StepStats(ctypes.Structure):
    """rt_step_stats: Newton, line-search and CG counts, norms and their histories."""

    _fields_ = [
        ("newton_iters", ctypes.c_int), ("residual_evals", ctypes.c_int),
        ("linear_iters", ctypes.c_int), ("line_search_cuts", ctypes.c_int),
        ("norm0", ctypes.c_double), ("norm", ctypes.c_double), ("change_norm", ctypes.c_double),
        ("kernel_launches", ctypes.c_int),
        ("nhist", ctypes.c_int),
        ("hist_norm", ctypes.c_double * 64),
        ("hist_lam", ctypes.c_double * 64),
        ("hist_cg", ctypes.c_int * 64),
    ]

    def as_dict(self):
        """The counters and the used part of each history as a plain dict."""
        d = {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("hist")}
        d["hist_norm"] = list(self.hist_norm[: self.nhist])
        d["hist_lam"] = list(self.hist_lam[: self.nhist])
        d["hist_cg"] = list(self.hist_cg[: min(self.newton_iters + 1, 64)])
        return d


class KernelProfile(ctypes.Structure):
    """rt_kernel_profile: launches, event time and algorithmic bytes of one kernel class."""

    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double)]


_lib = None

EXPORTS = ["rt_init_grid", "rt_implicit_step", "rt_residual", "rt_schur_system", "rt_schur_solve",
           "rt_adjoint_step", "rt_fold_energy", "rt_destroy_grid", "rt_error_string",
           "rt_last_error_detail", "rt_grey_constants", "rt_set_profiling", "rt_get_profile",
           "rt_residual_static", "rt_eval_elementary", "rt_advect", "rt_advect_adjoint", "rt_residual_helium",
           "rt_spectrum_constants"]


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"librtfld.so not built ({LIB_PATH}); run python -m paper_0908_2654_gb300.build")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    L.rt_init_grid.argtypes = [P(GridDesc), P(ctypes.c_void_p)]
    L.rt_implicit_step.argtypes = [ctypes.c_void_p, P(StepInputs), P(State), P(StepStats)]
    L.rt_residual.argtypes = [ctypes.c_void_p, P(StepInputs), P(State), P(State)] + [ctypes.c_void_p] * 3
    L.rt_residual_helium.argtypes = [ctypes.c_void_p, P(StepInputs), P(State), P(State)] + [ctypes.c_void_p] * 5
    L.rt_schur_system.argtypes = [ctypes.c_void_p, P(StepInputs), P(State), P(State)] + [ctypes.c_void_p] * 5
    L.rt_schur_solve.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                 P(ctypes.c_int)]
    L.rt_adjoint_step.argtypes = [ctypes.c_void_p, P(StepInputs), P(State), P(State), P(State), P(State),
                                  ctypes.c_void_p, ctypes.c_void_p]
    L.rt_fold_energy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.rt_advect.argtypes = [ctypes.c_void_p, P(StepInputs), P(State), P(State), ctypes.c_void_p, ctypes.c_void_p,
                            P(ctypes.c_double)]
    L.rt_advect_adjoint.argtypes = [ctypes.c_void_p, P(StepInputs), P(State), P(State)]
    L.rt_destroy_grid.argtypes = [ctypes.c_void_p]
    L.rt_destroy_grid.restype = None
    L.rt_error_string.argtypes = [ctypes.c_int]
    L.rt_error_string.restype = ctypes.c_char_p
    L.rt_last_error_detail.argtypes = []
    L.rt_last_error_detail.restype = ctypes.c_char_p
    L.rt_grey_constants.argtypes = [ctypes.c_void_p] + [P(ctypes.c_double)] * 3
    L.rt_set_profiling.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.rt_eval_elementary.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p]
    L.rt_residual_static.argtypes = [P(GridDesc), P(StepInputs), P(State), P(State)] + [ctypes.c_void_p] * 3
    L.rt_get_profile.argtypes = [ctypes.c_void_p, P(KernelProfile), ctypes.c_int, P(ctypes.c_int)]
    L.rt_spectrum_constants.argtypes = [ctypes.c_int, ctypes.c_double, P(ctypes.c_double)]
    for name in EXPORTS:
        if name not in ("rt_destroy_grid", "rt_error_string", "rt_last_error_detail"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


class RTError(RuntimeError):
    """A non-zero return code of the library, with its message and detail text."""

    def __init__(self, code, where):
        L = lib()
        self.code = code
        msg = L.rt_error_string(code).decode()
        detail = L.rt_last_error_detail().decode()
        super().__init__(f"{where}: {msg} ({detail})")


def check(code, where):
    """Raise RTError unless code is RT_OK."""
    if code != RT_OK:
        raise RTError(code, where)


def ptr(t):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())
