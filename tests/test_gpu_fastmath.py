"""The table-driven FP64 exp and log used by the rate fits against NumPy (glibc) and the CUDA
math library: at most 2 units in the last place over the ranges the rates use and beyond,
and the special values."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _eval(fn, x):
    from paper_0908_2654_gb300 import _rt
    xd = torch.as_tensor(np.ascontiguousarray(x, np.float64)).cuda()
    yd = torch.empty_like(xd)
    _rt.check(_rt.lib().rt_eval_elementary(fn, _rt.ptr(xd), _rt.ptr(yd), xd.numel(), None), "rt_eval_elementary")
    return yd.cpu().numpy()


def _ulp_err(a, ref):
    ok = np.isfinite(ref) & (ref != 0)
    return np.max(np.abs(a[ok] - ref[ok]) / np.spacing(np.abs(ref[ok])))


def test_exp_within_two_ulp():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-745, 709.7, 200000), rng.uniform(-1, 1, 100000), rng.uniform(-1e-8, 1e-8, 1000),
                        np.arange(-700, 700, 0.0108304), [0.0, 1.0, -1.0, 700.0, -708.0]])
    y = _eval(0, x)
    assert _ulp_err(y, np.exp(x)) <= 2.0
    assert _ulp_err(y, _eval(2, x)) <= 2.0
    sp = _eval(0, np.array([np.inf, -np.inf, np.nan, 710.0, -746.0, -740.0]))
    assert sp[0] == np.inf and sp[1] == 0.0 and np.isnan(sp[2]) and sp[3] == np.inf and sp[4] == 0.0
    assert sp[5] == pytest.approx(np.exp(-740.0), rel=1e-6)       # subnormal range


def test_log_within_two_ulp():
    rng = np.random.default_rng(1)
    x = np.concatenate([10 ** rng.uniform(-307, 307, 200000), rng.uniform(0.5, 2.0, 100000),
                        1 + rng.uniform(-1e-6, 1e-6, 10000), [1.0, 2.0, 0.5, 1e4, 3.15614e5]])
    y = _eval(1, x)
    assert _ulp_err(y, np.log(x)) <= 2.0
    assert _ulp_err(y, _eval(3, x)) <= 2.0
    assert _eval(1, np.array([1.0]))[0] == 0.0
    sp = _eval(1, np.array([0.0, -1.0, np.inf, np.nan, 5e-320]))
    assert sp[0] == -np.inf and np.isnan(sp[1]) and sp[2] == np.inf and np.isnan(sp[3])
    assert sp[4] == pytest.approx(np.log(5e-320), rel=1e-12)       # subnormal argument
