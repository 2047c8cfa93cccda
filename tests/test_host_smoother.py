"""The red-black Gauss-Seidel sweep of the multigrid levels (rbpass.cuh), compiled for the host
and run launch by launch, block by block, on the colour-split storage of a level against a plain
red-black Gauss-Seidel sweep in natural order written from its definition: update every cell of
the first colour from its neighbours' old values, x_i = (b_i + sum_faces w_f x_nb) / diag_i, then
every cell of the other colour from the new values.  Also: the colour-split index is a bijection,
the split operator fills every entry, the zero start, each pass setting exactly the cells of its
colour, every index in range, rows shorter and longer than a block, periodic and reflecting axes;
the trilinear cell-centred prolongation of a natural or colour-split coarse vector; and the
coarse solver's colouring, which gives no two neighbours one colour, odd periodic axes included."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("host") / "smoother_host.so")
    subprocess.run([nvcc, "-x", "cu", "-std=c++17", "--expt-relaxed-constexpr", "-O2", "-shared", "-Xcompiler",
                    "-fPIC", "-gencode", "arch=compute_103a,code=sm_103a", os.path.join(HERE, "host", "smoother_host.cu"),
                    "-o", out], check=True, capture_output=True)
    return ctypes.CDLL(out)


def _operator(shape, per, rng, dtype):
    """diag, wx, wy, wz of a diagonally dominant 7-point operator ([z][y][x]); face couplings of
    the last cell along a non-periodic axis are zero (boundary faces)."""
    w = [rng.uniform(0.5, 2.0, shape) for _ in range(3)]
    for d, ax in ((0, 2), (1, 1), (2, 0)):
        if not per[d]:
            sl = [slice(None)] * 3
            sl[ax] = -1
            w[d][tuple(sl)] = 0.0
    nb = sum(w[d] + np.roll(w[d], 1, axis=ax) for d, ax in ((0, 2), (1, 1), (2, 0)))
    diag = nb + rng.uniform(0.1, 1.0, shape)
    return [a.astype(dtype) for a in (diag, *w)]


def _neighbour_sum(w, x):
    """sum over the six faces of w_f x_nb (np.roll wraps; boundary couplings are zero)."""
    wx, wy, wz = w
    s = np.zeros_like(x)
    for wd, ax in ((wx, 2), (wy, 1), (wz, 0)):
        s = s + wd * np.roll(x, -1, axis=ax) + np.roll(wd, 1, axis=ax) * np.roll(x, 1, axis=ax)
    return s


def _rbgs_reference(diag, w, b, x, first):
    z, y, xx = np.indices(x.shape)
    par = (xx + y + z) % 2
    x = x.astype(np.float64).copy()
    for c in (first, 1 - first):
        new = (b + _neighbour_sum(w, x)) / diag
        x[par == c] = new[par == c]
    return x


def _prolong_reference(xc, fshape, per):
    """Trilinear cell-centred prolongation: weights 3/4 and 1/4 from the coarse cell holding the
    fine cell and its neighbour on the fine cell's side (itself at a non-periodic edge)."""
    nz, ny, nx = fshape
    cz, cy, cx = xc.shape
    out = np.zeros(fshape)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                idx = []
                for c, n, p in ((x, cx, per[0]), (y, cy, per[1]), (z, cz, per[2])):
                    C = c >> 1
                    o = C + 1 if c & 1 else C - 1
                    if not (0 <= o < n):
                        o = (o + n) % n if p else C
                    idx.append((C, o))
                (X, X2), (Y, Y2), (Z, Z2) = idx
                v = 0.0
                for wz_, zz in ((0.75, Z), (0.25, Z2)):
                    for wy_, yy in ((0.75, Y), (0.25, Y2)):
                        for wx_, xx in ((0.75, X), (0.25, X2)):
                            v += wz_ * wy_ * wx_ * xc[zz, yy, xx]
                out[z, y, x] = v
    return out


def _sweep(lib, dtype, shape, per, diag, w, b, xin, first, zero, quad=1):
    nz, ny, nx = shape
    fn = lib.sweep_host_f64 if dtype == np.float64 else lib.sweep_host_f32
    fn.restype = ctypes.c_longlong
    arr = lambda a: np.ascontiguousarray(a, dtype=dtype)
    args = [arr(diag), *[arr(v) for v in w], arr(b)]
    x = np.array(xin, dtype=dtype, copy=True)
    bad = fn(nx, ny, nz, (ctypes.c_int * 3)(*per), *[a.ctypes.data_as(ctypes.c_void_p) for a in args],
             x.ctypes.data_as(ctypes.c_void_p), first, zero, quad)
    return x, bad


# (nz, ny, nx), periodic (x, y, z): split levels have even dimensions
CASES = [((20, 32, 64), (True, True, True)), ((24, 40, 40), (False, False, False)),
         ((4, 6, 8), (False, True, False)), ((10, 18, 36), (True, False, True)),
         ((12, 20, 34), (False, False, True)), ((8, 8, 8), (True, True, True)),
         ((6, 4, 300), (True, False, False)), ((2, 8, 2), (False, True, False)),
         ((24, 6, 8), (True, True, False)), ((2, 2, 258), (True, True, True))]


@pytest.mark.parametrize("quad", [1, 0])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("shape,per", CASES)
def test_sweep_equals_red_black_gauss_seidel(lib, shape, per, dtype, quad):
    """quad = 1: two pairs per thread wherever nx is a multiple of 4; quad = 0: one pair."""
    rng = np.random.default_rng(13 + sum(shape))
    diag, *w = _operator(shape, per, rng, dtype)
    b = rng.standard_normal(shape).astype(dtype)
    x0 = rng.standard_normal(shape).astype(dtype)
    tol = 1e-13 if dtype == np.float64 else 2e-6
    for first, zero, xin in ((0, 0, x0), (1, 0, x0), (0, 1, np.zeros(shape))):
        ref = _rbgs_reference(diag, w, b, xin, first)
        start = np.full(shape, np.nan) if zero else xin
        got, bad = _sweep(lib, dtype, shape, per, diag, w, b, start, first, zero, quad)
        assert bad == 0
        np.testing.assert_allclose(got, ref, rtol=tol, atol=tol * np.abs(ref).max())


@pytest.mark.parametrize("fn", ["prolong_host", "prolong_pair_host"])
@pytest.mark.parametrize("csplit", [0, 1])
@pytest.mark.parametrize("shape,per", [CASES[0], CASES[1], CASES[3], ((40, 24, 48), (False, False, True)),
                                       ((4, 2, 2), (True, True, True))])
def test_prolongation_is_trilinear(lib, shape, per, csplit, fn):
    rng = np.random.default_rng(7)
    cshape = tuple(n // 2 for n in shape)
    xc = rng.standard_normal(cshape)
    nz, ny, nx = shape
    out = np.zeros(shape)
    bad = getattr(lib, fn)(nx, ny, nz, (ctypes.c_int * 3)(*per), xc.ctypes.data_as(ctypes.c_void_p), cshape[2],
                           cshape[1], cshape[0], csplit, out.ctypes.data_as(ctypes.c_void_p))
    assert bad == 0
    np.testing.assert_allclose(out, _prolong_reference(xc, shape, per), rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("dims,per", [((8, 6, 4), (1, 1, 1)), ((5, 4, 6), (1, 0, 1)), ((5, 5, 5), (1, 1, 1)),
                                      ((3, 7, 1), (1, 1, 1)), ((1, 1, 5), (0, 0, 1)), ((7, 3, 9), (0, 0, 0)),
                                      ((2, 3, 3), (1, 1, 0)), ((9, 1, 1), (1, 0, 0))])
def test_coarse_colouring_has_no_neighbour_conflict(lib, dims, per):
    ncol = ctypes.c_int(0)
    lib.colour_conflicts.restype = ctypes.c_longlong
    bad = lib.colour_conflicts(*dims, (ctypes.c_int * 3)(*per), ctypes.byref(ncol))
    assert bad == 0
    odd_per = any(p and n % 2 for n, p in zip(dims, per))
    assert ncol.value == (3 if odd_per else 2)


@pytest.mark.parametrize("shape,per", [c for c in CASES if c[0][2] % 2 == 0])
def test_pair_residuals_equal_b_minus_Sx(lib, shape, per):
    rng = np.random.default_rng(23)
    diag, *w = _operator(shape, per, rng, np.float64)
    b = rng.standard_normal(shape)
    x = rng.standard_normal(shape)
    nz, ny, nx = shape
    out = np.zeros(shape)
    lib.resid_host.restype = ctypes.c_longlong
    args = [np.ascontiguousarray(a) for a in (diag, *w, b, x)]
    bad = lib.resid_host(nx, ny, nz, (ctypes.c_int * 3)(*per), *[a.ctypes.data_as(ctypes.c_void_p) for a in args],
                         out.ctypes.data_as(ctypes.c_void_p))
    assert bad == 0
    want = b - (diag * x - _neighbour_sum(w, x))
    np.testing.assert_allclose(out, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
