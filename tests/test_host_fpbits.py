"""The bit-pattern conversions of the multigrid's level-0 casts (fpbits.cuh), compiled for the
host, against NumPy's IEEE-754 arithmetic: x 2^-e rounded to FP32 (NumPy rounds ties to even,
the bit version ties away from zero, so the two may differ by one unit in the last place exactly
at ties, which are planted and checked), values below the FP32 normal range (and FP64
subnormal inputs) flushed to zero, f 2^e widened to FP64 exactly where the result is a normal
FP64 number and to zero below, the exponent e of frexp, and non-finite values kept non-finite."""
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
    out = str(tmp_path_factory.mktemp("host") / "fpbits_host.so")
    subprocess.run([nvcc, "-x", "cu", "-std=c++17", "-O2", "-shared", "-Xcompiler", "-fPIC", "-gencode",
                    "arch=compute_103a,code=sm_103a", os.path.join(HERE, "host", "fpbits_host.cu"), "-o", out],
                   check=True)
    return ctypes.CDLL(out)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _to_float(lib, v, e):
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.empty(v.size, np.float32)
    lib.to_float_scaled_host(v.size, _ptr(v), e, _ptr(out))
    return out


def _from_float(lib, f, e):
    f = np.ascontiguousarray(f, dtype=np.float32)
    out = np.empty(f.size, np.float64)
    lib.from_float_scaled_host(f.size, _ptr(f), e, _ptr(out))
    return out


@pytest.mark.parametrize("e", [0, 7, -30, 300, -900])
def test_scaled_narrowing_matches_ieee_rounding(lib, e):
    rng = np.random.default_rng(5 + abs(e))
    mag = 2.0 ** rng.uniform(-140, 0, 200000)          # |v 2^-e| in (2^-140, 1]
    v = np.ldexp(mag * rng.choice([-1.0, 1.0], mag.size), e)
    got = _to_float(lib, v, e)
    want = np.ldexp(v, -e).astype(np.float32)
    normal = (np.abs(np.ldexp(v, -e)) >= 2.0**-126) & (np.abs(v) >= 2.0**-1022)
    assert np.all(got[~normal] == 0.0)
    np.testing.assert_array_equal(got[normal], want[normal])


def test_ties_round_away_from_zero(lib):
    # fraction ending in exactly half an FP32 unit: 1 + (2k+1) 2^-24
    k = np.arange(0, 1000, dtype=np.float64)
    v = np.concatenate([1.0 + (2 * k + 1) * 2.0**-24, -(1.0 + (2 * k + 1) * 2.0**-24)])
    got = _to_float(lib, v, 0).astype(np.float64)
    away = np.sign(v) * (np.abs(v) + 2.0**-24)
    np.testing.assert_array_equal(got, away)


@pytest.mark.parametrize("e", [0, 12, -40, 900, -900])
def test_scaled_widening_is_exact(lib, e):
    rng = np.random.default_rng(17)
    f = (rng.standard_normal(100000) * 2.0 ** rng.uniform(-120, 120, 100000)).astype(np.float32)
    got = _from_float(lib, f, e)
    want = np.ldexp(f.astype(np.float64), e)
    keep = (np.abs(f) >= np.float32(2.0**-126)) & (np.abs(want) >= 2.0**-1022)
    np.testing.assert_array_equal(got[keep], want[keep])
    assert np.all(got[~keep] == 0.0)


def test_exponent_is_frexps(lib):
    rng = np.random.default_rng(3)
    v = 2.0 ** rng.uniform(-1000, 1000, 10000) * rng.uniform(0.5, 1.0, 10000)
    out = np.empty(v.size, np.int32)
    lib.pow2_exponent_host(v.size, _ptr(v), _ptr(out))
    np.testing.assert_array_equal(out, np.frexp(v)[1])
    assert np.all(v < np.ldexp(1.0, out))
    special = np.array([0.0, -1.0, np.inf, np.nan])
    out2 = np.empty(4, np.int32)
    lib.pow2_exponent_host(4, _ptr(special), _ptr(out2))
    assert list(out2) == [0, 0, 0, 0]


def test_non_finite_values_stay_non_finite(lib):
    v = np.array([np.inf, -np.inf, np.nan])
    got = _to_float(lib, v, 3)
    assert got[0] == np.inf and got[1] == -np.inf and np.isnan(got[2])
    back = _from_float(lib, got, 3)
    assert back[0] == np.inf and back[1] == -np.inf and np.isnan(back[2])
