"""The tables of the table-driven exp and log (csrc/fastmath_tables.cuh) are what their
committed generator writes, and every entry is the correctly rounded value it claims to be.

Each entry is checked with 60-digit arithmetic from Python's decimal module, a route
independent of the generator's mpmath:
* kExpTable[j] = 2^(j/64);
* kLogHi + kLogLo = ln F, with kLogHi the double nearest ln F;
* kLogInv = 1/F, for F = j/128 on [0.75, 1.5];
* the split constants of ln 2 and ln 2 / 64.
No GPU is needed."""
import decimal
import importlib.util
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_0908_2654_gb300", "csrc")
TABLES = os.path.join(CSRC, "fastmath_tables.cuh")

D = decimal.Context(prec=60)
LN2 = D.ln(decimal.Decimal(2))


def _arrays():
    text = open(TABLES).read()
    out = {}
    for name, body in re.findall(r"const double (\w+)\[\d+\] = \{(.*?)\};", text, flags=re.S):
        out[name] = [float(v) for v in body.replace("\n", " ").split(",") if v.strip()]
    for name, v in re.findall(r"constexpr double (\w+) = ([^;]+);", text):
        out[name] = float(v)
    out["kLogJ0"] = int(re.search(r"constexpr int kLogJ0 = (\d+);", text).group(1))
    return out


def _nearest(x):
    """The double nearest a Decimal (float(str) rounds correctly)."""
    return float(str(x))


def test_committed_tables_are_the_generators_output():
    pytest.importorskip("mpmath")
    spec = importlib.util.spec_from_file_location("gen_fastmath_tables", os.path.join(CSRC, "gen_fastmath_tables.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    assert gen.render() == open(TABLES).read()


def test_exp_table_is_correctly_rounded():
    t = _arrays()["kExpTable"]
    assert len(t) == 64
    for j, v in enumerate(t):
        assert v == _nearest(D.exp(D.multiply(D.divide(decimal.Decimal(j), 64), LN2))), j


def test_log_tables_are_correctly_rounded_and_split():
    a = _arrays()
    j0 = a["kLogJ0"]
    hi, lo, inv = a["kLogHi"], a["kLogLo"], a["kLogInv"]
    assert j0 == 96 and len(hi) == len(lo) == len(inv) == 97      # F = j/128 on [0.75, 1.5]
    for i in range(97):
        F = D.divide(decimal.Decimal(i + j0), 128)
        lnF = D.ln(F)
        assert hi[i] == _nearest(lnF), i
        assert lo[i] == _nearest(D.subtract(lnF, decimal.Decimal(hi[i]))), i
        assert inv[i] == 128.0 / (i + j0), i                      # one correctly rounded division
    assert hi[128 - j0] == 0.0 and lo[128 - j0] == 0.0            # F = 1


@pytest.mark.parametrize("hi_name,lo_name,scale", [("kLn2Hi", "kLn2Lo", 1), ("kLn2By64Hi", "kLn2By64Lo", 64)])
def test_split_constants(hi_name, lo_name, scale):
    a = _arrays()
    hi, lo = a[hi_name], a[lo_name]
    v = D.divide(LN2, scale)
    # hi holds at most 29 significant bits, so k * hi is exact for |k| < 2^24
    m, _ = decimal.Decimal(hi).as_integer_ratio()
    assert (m // (m & -m)).bit_length() <= 29
    assert lo == _nearest(D.subtract(v, decimal.Decimal(hi)))
    assert abs(lo) < abs(hi) * 2.0**-28
    assert a["kInvLn2x64"] == _nearest(D.divide(64, LN2))
