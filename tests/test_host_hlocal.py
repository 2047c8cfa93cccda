"""The Newton kernel's hydrogen local equations with written-out partial derivatives
(hlocal.cuh), compiled for the host, against the dual-number evaluation of the same equations
(physics.cuh local_solutions<Dual<3>>, the form the GPU residual and Schur parity tests check
against the oracle): S_e, S_n and their six partials in (e_c, n_HI, E), over random cell states
spanning ionised and neutral gas, cold and hot gas (the 1 K temperature floor included), bright
and floor-level radiation, isothermal and non-isothermal, with and without cooling."""
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
    out = str(tmp_path_factory.mktemp("host") / "hlocal_host.so")
    subprocess.run([nvcc, "-x", "cu", "-std=c++17", "--expt-relaxed-constexpr", "-O2", "-shared", "-Xcompiler",
                    "-fPIC", "-gencode", "arch=compute_103a,code=sm_103a", os.path.join(HERE, "host", "hlocal_host.cu"),
                    "-o", out], check=True, capture_output=True)
    return ctypes.CDLL(out)


def _states(rng, n):
    rho = 10 ** rng.uniform(-2, 2, n)                          # n_H in normalised units
    x = 10 ** rng.uniform(-7, 0, n)                            # neutral fraction
    nHI = x * rho
    y0 = rho * np.clip(x * 10 ** rng.uniform(-1, 1, n), 1e-8, 1.0)
    E0 = 10 ** rng.uniform(-12, 2, n)
    E = E0 * 10 ** rng.uniform(-2, 2, n)
    E[: n // 10] = 1e-3 * 1e-12                                # at the radiation floor
    eh = 10 ** rng.uniform(-4, 2, n)
    ec = eh * rng.uniform(-0.5, 1.0, n)
    ec[n // 10: n // 5] = -0.9999 * eh[n // 10: n // 5]       # below the 1 K floor
    clump = rng.uniform(1.0, 3.0, n)
    return rho, y0, E0, eh, clump, ec, nHI, E


PRM = dict(a=0.2, dt=3.0, theta=0.51, kG=0.7, kT=2.0e4, kA=1.0e11, kH=5.0e-2, kC=3.0e25, un=1.0e-6, E_min=1e-12,
           T_iso=1.0e4, phi_e=2.9)


def _run(lib, st, iso, recomb, cooling):
    n = len(st[0])
    prm = np.array(list(PRM.values()) + [iso, recomb, cooling], dtype=np.float64)
    oh = np.zeros((8, n))
    od = np.zeros((8, n))
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in st]
    lib.hlocal_host(ctypes.c_int(n), prm.ctypes.data_as(ctypes.c_void_p),
                    *[a.ctypes.data_as(ctypes.c_void_p) for a in arrs],
                    oh.ctypes.data_as(ctypes.c_void_p), od.ctypes.data_as(ctypes.c_void_p))
    return oh, od


@pytest.mark.parametrize("iso,recomb,cooling", [(0, 1, 1), (0, 0, 1), (0, 1, 0), (1, 0, 0), (1, 1, 0)])
def test_written_out_partials_match_dual_numbers(lib, iso, recomb, cooling):
    """Values to rounding; every partial but dS_n/dE to 1e-11 of the largest partial of the same
    function.  dS_n/dE goes through the Riccati solution's derivative in the photo-ionisation
    rate, whose terms cancel where the radiation is weak compared with recombination (the two
    forms then differ in their rounding by up to 1e-6; see the next test for which is closer)."""
    rng = np.random.default_rng(31 + 7 * iso + recomb + 2 * cooling)
    st = _states(rng, 5000)
    oh, od = _run(lib, st, iso, recomb, cooling)
    assert np.all(np.isfinite(oh))
    np.testing.assert_allclose(oh[:2], od[:2], rtol=1e-13, atol=0)
    for rows in ((2, 3, 4), (5, 6, 7)):
        scale = np.max(np.abs(od[list(rows)]), axis=0) + 1e-300
        for k in rows:
            err = np.max(np.abs(oh[k] - od[k]) / scale)
            assert err < (1e-6 if k == 7 else 1e-11), (k, err)


def test_riccati_rate_derivative_as_accurate_as_dual_numbers(lib):
    """dS_n/dE of both forms against a 60-digit evaluation of the isothermal S_n (the exact
    solution of y' = A (n_H - y)^2 - G y over dt with G = c sigma_G pos(theta E + (1 - theta) E^n)
    / a^3, differentiated numerically at 60 digits), on the cells where the two forms disagree
    most and on random cells: the written-out form is no less accurate."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    rng = np.random.default_rng(38)
    st = _states(rng, 5000)
    oh, od = _run(lib, st, 1, 0, 0)
    rho, y0, E0, eh, clump, ec, nHI, E = st
    P = PRM

    def Sn(Ev, i):
        x = P["theta"] * Ev + (1 - P["theta"]) * mp.mpf(E0[i])
        Eb = (x + mp.sqrt(x * x + mp.mpf(P["E_min"]) ** 2)) / 2
        G = mp.mpf(P["kG"]) / mp.mpf(P["a"]) ** 3 * Eb
        A = mp.mpf(2.59e-13) * mp.mpf(P["kA"]) * mp.mpf(clump[i]) / mp.mpf(P["a"]) ** 3
        nH, y = mp.mpf(rho[i]), mp.mpf(y0[i])
        t = mp.mpf(P["dt"])
        # y(t) by separation of variables: the roots y1 < nH < y2 of A (nH - y)^2 - G y
        disc = mp.sqrt(G * G + 4 * nH * A * G)
        y1 = (2 * A * nH + G - disc) / (2 * A)
        y2 = (2 * A * nH + G + disc) / (2 * A)
        k = mp.exp(-A * (y2 - y1) * t)
        c = (y - y1) / (y - y2)
        return (y1 - y2 * c * k) / (1 - c * k)

    dis = np.abs(oh[7] - od[7]) / np.abs(od[7])
    cells = np.concatenate([np.argsort(dis)[-30:], rng.choice(len(dis), 30, replace=False)])
    eh_, ed_ = [], []
    for i in cells:
        ex = float(mp.diff(lambda e: Sn(e, int(i)), mp.mpf(E[i])))
        eh_.append(abs(oh[7, i] - ex) / abs(ex))
        ed_.append(abs(od[7, i] - ex) / abs(ex))
    assert max(eh_) <= 3 * max(ed_) + 1e-12, (max(eh_), max(ed_))
    assert np.median(eh_) <= 3 * np.median(ed_) + 1e-13
