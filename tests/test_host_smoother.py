"""The fused red-black Gauss-Seidel sweep of the multigrid levels (smoother.cuh), compiled for
the host and run CTA by CTA in the order its barriers impose, against a plain red-black
Gauss-Seidel sweep written from its definition: update every cell of the first colour from its
neighbours' old values, x_i = (b_i + sum_faces w_f x_nb) / diag_i, then every cell of the other
colour from the new values.  Also: the fused coarse-grid correction (old iterate plus the
trilinear cell-centred prolongation of a coarse vector), the zero start, every global index in
range, several z chunks and tiles cut by the grid's edge, periodic and reflecting axes."""
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


def _call_tma(lib, dtype, shape, per, diag, w, b, xin, first, zero, zc, grid=5):
    nz, ny, nx = shape
    fn = lib.sweep_tma_host_f64 if dtype == np.float64 else lib.sweep_tma_host_f32
    fn.restype = ctypes.c_longlong
    arr = lambda a: np.ascontiguousarray(a, dtype=dtype)
    args = [arr(diag), *[arr(v) for v in w], arr(b), arr(xin)]
    out = np.full(shape, np.nan, dtype=dtype)
    perc = (ctypes.c_int * 3)(*per)
    bad = fn(nx, ny, nz, perc, *[a.ctypes.data_as(ctypes.c_void_p) for a in args], out.ctypes.data_as(ctypes.c_void_p),
             first, zero, zc, grid)
    return out, bad


def _call_queue(lib, dtype, shape, per, diag, w, b, xin, first, zero):
    nz, ny, nx = shape
    fn = lib.sweep_queue_host_f64 if dtype == np.float64 else lib.sweep_queue_host_f32
    fn.restype = ctypes.c_longlong
    arr = lambda a: np.ascontiguousarray(a, dtype=dtype)
    args = [arr(diag), *[arr(v) for v in w], arr(b)]
    x = np.array(xin, dtype=dtype, copy=True)
    perc = (ctypes.c_int * 3)(*per)
    bad = fn(nx, ny, nz, perc, *[a.ctypes.data_as(ctypes.c_void_p) for a in args], x.ctypes.data_as(ctypes.c_void_p),
             first, zero)
    return x, bad


def _call(lib, dtype, shape, per, diag, w, b, xin, first, zero, zc, xc=None, nth=256, grid=7):
    nz, ny, nx = shape
    fn = lib.sweep_host_f64 if dtype == np.float64 else lib.sweep_host_f32
    fn.restype = ctypes.c_longlong
    arr = lambda a: np.ascontiguousarray(a, dtype=dtype)
    args = [arr(diag), *[arr(v) for v in w], arr(b), arr(xin)]
    out = np.full(shape, np.nan, dtype=dtype)
    perc = (ctypes.c_int * 3)(*per)
    cshape = xc.shape if xc is not None else (1, 1, 1)
    xcp = arr(xc).ctypes.data_as(ctypes.c_void_p) if xc is not None else None
    bad = fn(nx, ny, nz, perc, *[a.ctypes.data_as(ctypes.c_void_p) for a in args], out.ctypes.data_as(ctypes.c_void_p),
             first, zero, zc, xcp, cshape[2], cshape[1], cshape[0], nth, grid)
    return out, bad


CASES = [((20, 32, 64), (True, True, True), 4), ((24, 40, 40), (False, False, False), 0),
         ((4, 6, 8), (False, True, False), 0), ((10, 18, 36), (True, False, True), 3),
         ((12, 20, 34), (False, False, True), 5), ((8, 8, 8), (True, True, True), 0)]


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("shape,per,zc", CASES)
def test_fused_sweep_equals_red_black_gauss_seidel(lib, shape, per, zc, dtype):
    rng = np.random.default_rng(sum(shape))
    diag, *w = _operator(shape, per, rng, dtype)
    b = rng.standard_normal(shape).astype(dtype)
    x0 = rng.standard_normal(shape).astype(dtype)
    tol = 1e-13 if dtype == np.float64 else 2e-6
    for first in (0, 1):
        ref = _rbgs_reference(diag, w, b, x0, first)
        got, bad = _call(lib, dtype, shape, per, diag, w, b, x0, first, 0, zc, grid=1 if first else 7)
        assert bad == 0
        np.testing.assert_allclose(got, ref, rtol=tol, atol=tol * np.abs(ref).max())
    ref0 = _rbgs_reference(diag, w, b, np.zeros(shape), 0)
    got, bad = _call(lib, dtype, shape, per, diag, w, b, np.full(shape, np.nan), 0, 1, zc)
    assert bad == 0
    np.testing.assert_allclose(got, ref0, rtol=tol, atol=tol * np.abs(ref0).max())


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("shape,per,zc", CASES)
def test_tensor_copy_sweep_equals_red_black_gauss_seidel(lib, shape, per, zc, dtype):
    """The sweep fed by bulk tensor copies (boxes with zeros outside the grid, wrapped edges of
    periodic axes patched, planes copied ahead into a ring of slots), its copies emulated in the
    kernel's order, against the plain sweep's definition."""
    rng = np.random.default_rng(3 + sum(shape))
    diag, *w = _operator(shape, per, rng, dtype)
    b = rng.standard_normal(shape).astype(dtype)
    x0 = rng.standard_normal(shape).astype(dtype)
    tol = 1e-13 if dtype == np.float64 else 2e-6
    for first in (0, 1):
        ref = _rbgs_reference(diag, w, b, x0, first)
        got, bad = _call_tma(lib, dtype, shape, per, diag, w, b, x0, first, 0, zc, grid=1 if first else 5)
        assert bad == 0
        np.testing.assert_allclose(got, ref, rtol=tol, atol=tol * np.abs(ref).max())
    ref0 = _rbgs_reference(diag, w, b, np.zeros(shape), 1)
    got, bad = _call_tma(lib, dtype, shape, per, diag, w, b, np.full(shape, np.nan), 1, 1, zc)
    assert bad == 0
    np.testing.assert_allclose(got, ref0, rtol=tol, atol=tol * np.abs(ref0).max())


QCASES = CASES + [((40, 16, 16), (True, False, True), 0), ((37, 8, 10), (False, True, False), 0),
                  ((24, 6, 8), (True, True, False), 0)]


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("shape,per,zc", QCASES)
def test_queued_in_place_sweep_equals_red_black_gauss_seidel(lib, shape, per, zc, dtype):
    """The in-place sweep whose two colour passes are cut into slab chunks and queued (R0, R1,
    B0, R2, B1, ...; periodic z: B0 last), run item by item in queue order, against the plain
    sweep's definition; every second-pass chunk finds the first passes over its own and the
    neighbouring slabs complete, and every index lies in the grid (odd nz too)."""
    rng = np.random.default_rng(11 + sum(shape))
    diag, *w = _operator(shape, per, rng, dtype)
    b = rng.standard_normal(shape).astype(dtype)
    x0 = rng.standard_normal(shape).astype(dtype)
    tol = 1e-13 if dtype == np.float64 else 2e-6
    for first in (0, 1):
        ref = _rbgs_reference(diag, w, b, x0, first)
        got, bad = _call_queue(lib, dtype, shape, per, diag, w, b, x0, first, 0)
        assert bad == 0
        np.testing.assert_allclose(got, ref, rtol=tol, atol=tol * np.abs(ref).max())
    ref0 = _rbgs_reference(diag, w, b, np.zeros(shape), 0)
    got, bad = _call_queue(lib, dtype, shape, per, diag, w, b, np.full(shape, np.nan), 0, 1)
    assert bad == 0
    np.testing.assert_allclose(got, ref0, rtol=tol, atol=tol * np.abs(ref0).max())


@pytest.mark.parametrize("slab", [0, 3, 4])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("shape,per,zc", QCASES)
def test_slab_ordered_passes_equal_red_black_gauss_seidel(lib, shape, per, zc, dtype, slab):
    """In-place colour passes launched slab by slab (R0, R1, B0, R2, B1, ...; periodic z: B0
    last), every launch's threads in turn, against the plain sweep's definition; each second pass
    follows the first passes over its own and the neighbouring slabs; indices in range."""
    nz, ny, nx = shape
    rng = np.random.default_rng(13 + sum(shape))
    diag, *w = _operator(shape, per, rng, dtype)
    b = rng.standard_normal(shape).astype(dtype)
    x0 = rng.standard_normal(shape).astype(dtype)
    tol = 1e-13 if dtype == np.float64 else 2e-6
    fn = lib.sweep_pass_host_f64 if dtype == np.float64 else lib.sweep_pass_host_f32
    fn.restype = ctypes.c_longlong
    arr = lambda a: np.ascontiguousarray(a, dtype=dtype)
    for first, zero, xin in ((0, 0, x0), (1, 0, x0), (0, 1, np.zeros(shape))):
        ref = _rbgs_reference(diag, w, b, xin, first)
        x = np.array(np.full(shape, np.nan) if zero else xin, dtype=dtype, copy=True)
        args = [arr(diag), *[arr(v) for v in w], arr(b)]
        bad = fn(nx, ny, nz, (ctypes.c_int * 3)(*per), *[a.ctypes.data_as(ctypes.c_void_p) for a in args],
                 x.ctypes.data_as(ctypes.c_void_p), first, zero, slab)
        assert bad == 0
        np.testing.assert_allclose(x, ref, rtol=tol, atol=tol * np.abs(ref).max())


def test_queue_plan(lib):
    """Slabs of 8 planes (all of a thinner grid), chunks of 8192 cells' rows: 256^3 gives 32 slabs
    of 8 planes x 8 row blocks of 32 rows."""
    out = (ctypes.c_int * 5)()
    lib.queue_plan(256, 256, 256, 1, out)
    assert list(out) == [8, 32, 32, 8, 64]
    lib.queue_plan(16, 16, 4, 0, out)
    assert list(out) == [4, 1, 16, 1, 4]


@pytest.mark.parametrize("shape,per,zc", [CASES[0], CASES[1], CASES[3], CASES[4]])
def test_fused_sweep_with_coarse_correction(lib, shape, per, zc):
    rng = np.random.default_rng(7)
    dtype = np.float64
    diag, *w = _operator(shape, per, rng, dtype)
    b = rng.standard_normal(shape)
    x0 = rng.standard_normal(shape)
    cshape = tuple(n // 2 for n in shape)
    xc = rng.standard_normal(cshape)
    ref = _rbgs_reference(diag, w, b, x0 + _prolong_reference(xc, shape, per), 1)
    got, bad = _call(lib, dtype, shape, per, diag, w, b, x0, 1, 0, zc, xc=xc)
    assert bad == 0
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def test_chunking_fills_the_resident_ctas(lib):
    """Work items of 16 planes while they fill the resident CTAs (256^3: 8 x 32 columns, 16 chunks,
    4096 items), halved down to 4 planes for small levels."""
    lib.sweep_chunk_planes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_longlong]
    assert lib.sweep_chunk_planes(256, 256, 256, 912) == 16
    assert lib.sweep_chunk_planes(64, 64, 64, 912) == 4
    assert lib.sweep_chunk_planes(16, 16, 2, 912) == 2
