"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: values the
paper prints (tests/golden/paper_values.json), closed forms, independent
numerical integration, brute-force derivatives or dense solves.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

import workloads as W
from oracle import constants as K
from oracle import cosmology as C
from oracle import diagnostics as D
from oracle import driver
from oracle import model as M
from oracle import newton as N
from oracle import newton as N_
from oracle import rates
from oracle import spectrum as S

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


# ----------------------------------------------------------------- paper values


def test_paper_constants():
    assert K.ALPHA_B_PAPER == GOLD["alpha_B_cm3_s"]["value"]
    assert K.HNU0 == pytest.approx(GOLD["hnu0_eV"]["value"] * K.EV, rel=1e-15)
    assert K.GAMMA == pytest.approx(GOLD["gamma"]["value"], rel=1e-15)
    assert W.E_FLOOR == GOLD["E_initial_erg_cm3"]["value"]
    assert M.E_MIN_DEFAULT == GOLD["E_initial_erg_cm3"]["value"]


def test_table1_densities_reproduce_quoted_rho_b0():
    """Omega_b rho_crit(H0) (1+z0)^3 of the z0 = 4 rows of Table 1 is the quoted rho_b0."""
    for q0, z0, L0, h, Om, OL, Ob in GOLD["table1"]["rows"]:
        assert Om == pytest.approx(2 * q0)        # q0 = Omega_m / 2 without Lambda
        if z0 == 4:
            rho = Ob * K.RHO_CRIT_H2 * h**2 * (1 + z0) ** 3
            assert rho == pytest.approx(GOLD["rho_b0_g_cm3"][f"q0={q0}"], rel=2e-3)


def test_hg97_alpha_matches_paper_value_at_1e4K():
    assert rates.alpha_B(1e4, "hg97") == pytest.approx(GOLD["alpha_B_cm3_s"]["value"], rel=2e-3)
    assert rates.alpha_B(1e4, "const") == GOLD["alpha_B_cm3_s"]["value"]


# ------------------------------------------------------------------ spectrum


def _bose_moment(n, x0, kmax=200):
    """int_{x0}^inf x^n / (e^x - 1) dx as the series sum_k e^{-k x0} P_n(x0, k)."""
    tot = 0.0
    for k in range(1, kmax):
        poly = sum(math.factorial(n) / math.factorial(n - j) * x0 ** (n - j) / k ** (j + 1)
                   for j in range(n + 1))
        tot += math.exp(-k * x0) * poly
    return tot


def test_blackbody_grey_constants_closed_forms():
    T_B = GOLD["T_B_K"]["value"]
    g = S.grey_constants("blackbody", T_B)
    kT = K.K_BOLTZ * T_B
    x0 = K.HNU0 / kT
    e3 = _bose_moment(3, x0)
    e2 = _bose_moment(2, x0)
    s0 = -math.log(-math.expm1(-x0))                          # int 1/(e^x-1)
    sm1 = sum(special.exp1(k * x0) for k in range(1, 200))     # int x^-1/(e^x-1)
    assert g["sigma_E"] == pytest.approx(K.SIGMA0 * x0**3 * s0 / e3, rel=1e-10)
    assert g["sigma_G"] == pytest.approx(K.SIGMA0 * x0**3 * sm1 / (kT * e3), rel=1e-10)
    assert g["eps_src"] == pytest.approx(kT * e3 / e2, rel=1e-10)
    # absorbed photons are softer than emitted ones, and both lie above the edge
    assert K.HNU0 < g["sigma_E"] / g["sigma_G"] < g["eps_src"]


def test_mono_grey_constants():
    g = S.grey_constants("mono")
    assert g["sigma_E"] == K.SIGMA0
    assert g["sigma_G"] * K.HNU0 == pytest.approx(K.SIGMA0, rel=1e-15)
    assert g["eps_src"] == K.HNU0
    # monochromatic edge photons deposit no heat
    assert g["sigma_E"] - K.HNU0 * g["sigma_G"] == pytest.approx(0.0, abs=1e-30)


# ------------------------------------------------------------- flux limiter


def test_limiter_limits():
    kap = 3.7e-22
    assert M.limiter_D(kap, 1e-12 * kap) == pytest.approx(K.C_LIGHT / (3 * kap), rel=1e-10)
    R = 1e12 * kap
    assert M.limiter_D(kap, R) * R == pytest.approx(K.C_LIGHT, rel=1e-10)    # |flux| -> c E
    assert M.limiter_D(0.0, 2.0) * 2.0 == pytest.approx(K.C_LIGHT, rel=1e-15)
    # flux never exceeds the free-streaming bound c E for any opacity
    for kT in (1e-30, 1e-24, 1e-20):
        for r in (1e-30, 1e-24, 1e-20, 1e-10):
            assert M.limiter_D(kT, r) * r <= K.C_LIGHT * (1 + 1e-12)


# ------------------------------------------------------------ local solutions


@pytest.mark.parametrize("case", range(8))
def test_riccati_matches_ode_integration(case):
    rng = np.random.default_rng(100 + case)
    nH = 10 ** rng.uniform(-4, -2)
    y0 = nH * 10 ** rng.uniform(-6, 0) * (1 - 1e-9)
    A = 10 ** rng.uniform(-17, -11)
    G = [0.0, 10 ** rng.uniform(-20, -10), 10 ** rng.uniform(-16, -12)][case % 3]
    if case == 7:
        A = 0.0
        G = 1e-14
    dt = 10 ** rng.uniform(12, 14.5)
    y = M.riccati_Sn(y0, nH, A, G, dt)
    sol = integrate.solve_ivp(lambda t, v: [A * (nH - v[0]) ** 2 - G * v[0]], (0, dt), [y0],
                              method="Radau", rtol=1e-12, atol=1e-18 * nH)
    assert float(y) == pytest.approx(sol.y[0, -1], rel=1e-8, abs=1e-14 * nH)


def test_riccati_equilibrium_root():
    nH, A, G = 2e-3, 3e-15, 5e-13
    yeq = M.riccati_Sn(0.5 * nH, nH, A, G, 1e30)      # t -> infinity
    assert A * (nH - yeq) ** 2 == pytest.approx(G * yeq, rel=1e-10)


def test_gas_energy_solution_matches_ode():
    """S_e with frozen G - Lambda solves de/dt = -2 (adot/a) e + g from e = 0."""
    H, g, dt = 3e-17, 4e-3, 2e15
    e = g * dt * M.phi1(2 * H * dt)
    sol = integrate.solve_ivp(lambda t, v: [-2 * H * v[0] + g], (0, dt), [0.0], rtol=1e-12, atol=1e-20)
    assert e == pytest.approx(sol.y[0, -1], rel=1e-9)
    assert M.phi1(0.0) == 1.0


# --------------------------------------------------- discrete radiation operator


def _uniform_step(n=(8, 6, 5), **kw):
    nx, ny, nz = n
    shape = (nz, ny, nx)
    base = dict(nx=nx, ny=ny, nz=nz, dx=3e21, periodic=(True, True, True),
                rho_b=np.full(shape, 1e-3 * K.M_H), e_h=np.full(shape, 1e12),
                v=tuple(np.zeros(shape) for _ in range(3)), clump=np.ones(shape),
                E_n=np.full(shape, 1e-20), nHI_n=np.full(shape, 0.5e-3), a=1.0, adot=0.0, dt=1e13,
                src_index=np.array([], np.int64), src_ndot=np.array([]),
                sigma_E=0.0, sigma_G=0.0, eps_src=K.HNU0)
    base.update(kw)
    return M.Step(**base)


def test_fourier_mode_amplification_is_exact():
    """Constant D, no opacity: a periodic Fourier mode decays by the theta-scheme factor
    (1 - (1-theta) dt mu) / (1 + theta dt mu), mu = D sum_d 4 sin^2(pi k_d / N_d) / (a dx)^2 + adot/a."""
    n = (8, 6, 5)
    k = (1, 2, 1)
    a, adot, dt, Dc, dx, theta = 0.4, 2e-17, 3e13, 5e28, 3e21, 0.51
    z, y, x = np.indices((n[2], n[1], n[0]))
    mode = np.cos(2 * np.pi * (k[0] * x / n[0] + k[1] * y / n[1] + k[2] * z / n[2]))
    En = 1e-20 * (2.0 + mode)
    st = _uniform_step(n, E_n=En, a=a, adot=adot, dt=dt, dx=dx, theta=theta, limiter="const", D_const=Dc)
    U, info = N.solve_step(st, tol=1e-13)
    mu = Dc * sum(4 * math.sin(math.pi * kd / nd) ** 2 for kd, nd in zip(k, n)) / (a * dx) ** 2 + adot / a
    mu0 = adot / a
    g = lambda m: (1 - (1 - theta) * dt * m) / (1 + theta * dt * m)
    expect = 1e-20 * (2.0 * g(mu0) + g(mu) * mode)
    np.testing.assert_allclose(U[2], expect, rtol=1e-11)


@pytest.mark.parametrize("theta", [0.51, 1.0])
def test_gaussian_spreading_variance_law(theta):
    """Constant-D diffusion of a Gaussian pulse, no opacity or expansion: the pulse's energy
    is conserved and its variance grows as sigma^2(t) = sigma_0^2 + 2 D t along the axis of
    the pulse.  For the discrete theta-scheme this holds exactly, step by step: summing
    x^2 times the 7-point Laplacian by parts gives 2 (a dx)^2 times the energy, at either
    time level, while the pulse stays clear of the periodic wrap (the implicit scheme's tails,
    geometric rather than Gaussian, are below 1e-16 of the peak there).  A wrong Laplacian weight, theta split or 1/a^2 changes the growth."""
    n = (64, 3, 3)
    a, dt, Dc, dx = 0.5, 2e13, 2e28, 3e21
    x = np.arange(n[0]) - 31.5
    sig0 = 1.6                                           # cells
    prof = np.exp(-0.5 * (x / sig0) ** 2)
    En = 1e-20 * np.broadcast_to(prof, (n[2], n[1], n[0])).copy()
    st = _uniform_step(n, E_n=En, a=a, adot=0.0, dt=dt, dx=dx, theta=theta, limiter="const", D_const=Dc)
    steps, E = 3, En
    for _ in range(steps):
        st.E_n = E
        U, _ = N.solve_step(st, tol=1e-14)
        E = U[2]
    ex = E.sum(axis=(0, 1))                              # profile along x
    m0_0, m0 = En.sum(axis=(0, 1)).sum(), ex.sum()
    var0 = float(np.sum(En.sum(axis=(0, 1)) * x**2) / m0_0)
    var = float(np.sum(ex * x**2) / m0)
    growth = 2.0 * Dc * steps * dt / (a * dx) ** 2      # cells^2
    assert m0 == pytest.approx(m0_0, rel=1e-12)
    assert var - var0 == pytest.approx(growth, rel=1e-9)
    assert 0.5 < growth < 4.0                            # a real spread, far from the wrap
    assert ex[0] < 1e-16 * ex.max() and ex[-1] < 1e-16 * ex.max()


def test_gaussian_spreading_converges_at_second_order():
    """The discrete solution of constant-D diffusion converges to the continuum Gaussian
    E = A sigma0 / sigma(t) exp(-x^2 / (2 sigma(t)^2)), sigma^2 = sigma0^2 + 2 D t, at second
    order.  The test uses Crank-Nicolson (theta = 1/2), halves dx and dt together, and checks
    that the max-norm error falls by about 4 at each refinement."""
    L, a, Dc = 48 * 3e21, 1.0, 2e28
    sig0 = L / 48 * 2.5                                   # 2.5 coarse cells
    t_end = 0.5 * sig0**2 / Dc                            # sigma^2 doubles
    errs = []
    for n, nsteps in ((48, 4), (96, 8), (192, 16)):
        dx = L / n
        x = (np.arange(n) + 0.5) * dx - 0.5 * L
        gauss = lambda t: np.exp(-x**2 / (2 * (sig0**2 + 2 * Dc * t))) * sig0 / np.sqrt(sig0**2 + 2 * Dc * t)
        En = 1e-20 * np.broadcast_to(gauss(0.0), (3, 3, n)).copy()
        st = _uniform_step((n, 3, 3), E_n=En, a=a, adot=0.0, dt=t_end / nsteps, dx=dx, theta=0.5,
                           limiter="const", D_const=Dc)
        E = En
        for _ in range(nsteps):
            st.E_n = E
            U, _ = N.solve_step(st, tol=1e-14)
            E = U[2]
        errs.append(np.max(np.abs(E[1, 1] / 1e-20 - gauss(t_end))))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.7 < r2 < 4.3, (errs, r1, r2)


def test_diffusion_conserves_energy_with_walls_and_periodic():
    rng = np.random.default_rng(3)
    for periodic in ((True, True, True), (False, True, False)):
        st = _uniform_step((7, 5, 4), periodic=periodic, sigma_E=6.3e-18)
        E = 10 ** rng.uniform(-25, -15, st.shape)
        nHI = 10 ** rng.uniform(-6, -3, st.shape)
        Ld = M.diffusion(st, E, M.opacity(st, nHI))
        assert abs(Ld.sum()) <= 1e-12 * np.abs(Ld).sum()


def _image_extension(E, lower, upper):
    """Periodic extension of a 1-D profile E (cells 0..N-1) whose rows 0..N-1 evolve like the
    bounded problem: a reflecting face is a mirror plane for E (even image about the face), an
    outflow face a node of an odd image about the ghost cell beyond it (which then holds 0)."""
    N = len(E)
    if (lower, upper) == ("reflect", "outflow"):          # even about face -1/2, odd about cell N
        half = np.concatenate([E, [0.0], -E[::-1]])
        return np.concatenate([half, half[::-1]])          # period 4N + 2
    if (lower, upper) == ("outflow", "reflect"):
        mirrored = _image_extension(E[::-1], "reflect", "outflow")[::-1]   # E in the last N cells
        return np.roll(mirrored, N)
    if (lower, upper) == ("outflow", "outflow"):          # odd about cell N and cell -1
        return np.concatenate([E, [0.0], -E[::-1], [0.0]])
    raise ValueError((lower, upper))


@pytest.mark.parametrize("theta", [0.51, 1.0])
@pytest.mark.parametrize("faces", [("reflect", "outflow"), ("outflow", "reflect"), ("outflow", "outflow")])
def test_outflow_and_reflecting_faces_match_image_solutions(faces, theta):
    """Constant-D diffusion on a bounded 1-D grid equals, row for row, the periodic problem whose
    initial data are extended by images: an even image about a reflecting face and an odd image
    about the ghost cell beyond an outflow face.  The periodic operator is itself pinned
    (Fourier modes, Gaussian spreading); the images are exact for the discrete scheme because
    it commutes with mirroring and with a change of sign.  A dropped ghost term, a ghost at the
    wrong distance or a flipped sign breaks the agreement."""
    N = 11
    a, adot, dt, Dc, dx = 0.6, 1e-17, 4e13, 3e28, 3e21
    rng = np.random.default_rng(17)
    E1 = 1e-20 * (1.0 + rng.random(N))
    bounded = _uniform_step((N, 1, 1), E_n=E1.reshape(1, 1, N).copy(), a=a, adot=adot, dt=dt, dx=dx,
                            theta=theta, limiter="const", D_const=Dc, periodic=(False, False, False),
                            bc=(faces[0], faces[1], "reflect", "reflect", "reflect", "reflect"))
    Eext = _image_extension(E1, *faces)
    L = len(Eext)
    ext = _uniform_step((L, 1, 1), E_n=Eext.reshape(1, 1, L).copy(), a=a, adot=adot, dt=dt, dx=dx, theta=theta,
                        limiter="const", D_const=Dc, periodic=(True, False, False))
    for _ in range(2):
        Ub, _ = N_.solve_step(bounded, tol=1e-12)
        Ue, _ = N_.solve_step(ext, tol=1e-12)
        np.testing.assert_allclose(Ub[2].ravel(), Ue[2].ravel()[:N], rtol=1e-11, atol=1e-13 * E1.max())
        bounded.E_n, ext.E_n = Ub[2], Ue[2]
    # and the bounded run really lost energy through its outflow face(s)
    assert bounded.E_n.sum() < E1.sum() * (1 - 1e-3)


def test_outflow_faces_lose_the_discrete_boundary_flux():
    """Summed over the cells, the FLD operator with outflow faces equals minus the flux through
    those faces alone (interior face fluxes cancel in pairs; reflecting faces carry none).  The
    flux through an outflow face is D (E_i - 0) / (a dx)^2 per unit cell volume with D from
    Eq. limiter between the cell and its empty ghost: face energy E_i / 2, hence R = 2 / (a dx),
    and kappa_T the cell's own opacity.  With no opacity the face carries the free-streaming
    limit of the limiter, c times the face energy: c E_i / 2."""
    rng = np.random.default_rng(5)
    shape = (3, 4, 5)
    bc = ("outflow", "outflow", "reflect", "outflow", "outflow", "reflect")
    for sigma in (6.3e-18, 0.0):
        st = _uniform_step((5, 4, 3), periodic=(False, False, False), bc=bc, sigma_E=sigma, a=0.7,
                           limiter="new")
        E = 10 ** rng.uniform(-22, -16, shape)
        nHI = 10 ** rng.uniform(-5, -2, shape)
        kap = M.opacity(st, nHI)
        adx = st.a * st.dx
        total = M.diffusion(st, E, kap).sum()
        loss = 0.0
        for (ax, side) in ((2, 0), (2, -1), (1, -1), (0, 0)):      # the outflow faces
            sl = [slice(None)] * 3
            sl[ax] = side
            Eb, kb = E[tuple(sl)], kap[tuple(sl)]
            D = M.limiter_D(kb, 2.0 / adx)
            if sigma == 0.0:
                np.testing.assert_allclose(D * Eb / adx, K.C_LIGHT * Eb / 2, rtol=1e-14)
            loss += np.sum(D * Eb) / adx**2
        assert total == pytest.approx(-loss, rel=1e-12)


@pytest.mark.parametrize("n,src", [((4, 3, 3), 4e-31), ((4, 3, 3), 0.0), ((1, 1, 5), 4e-31), ((2, 2, 2), 0.0),
                                   ((5, 1, 1), 4e-31)])
def test_absorption_of_uniform_field_matches_scalar_root(n, src):
    """Uniform gas and field: the step reduces to one scalar equation in E (brentq root), also
    with no sources and on the degenerate grids (one-cell-thin, 2^3)."""
    g = S.grey_constants("blackbody", 1e5)
    a, adot, dt, theta = 0.25, 1e-17, 2e13, 0.8
    nH, En, nHIn = 2e-4, 3e-16, 2e-8
    shape = (n[2], n[1], n[0])
    # axes under 3 cells get zero-flux walls (the oracle's periodic Jacobian colouring needs 3);
    # a uniform field stays uniform either way
    st = _uniform_step(n, a=a, adot=adot, dt=dt, theta=theta, rho_b=np.full(shape, nH * K.M_H),
                       E_n=np.full(shape, En), nHI_n=np.full(shape, nHIn),
                       periodic=tuple(nd >= 3 for nd in n), **g)
    # a uniform emissivity written as one source per cell (none when src = 0)
    st.src_index = np.arange(st.N) if src > 0 else np.zeros(0, np.int64)
    st.src_ndot = np.full(st.N, src * st.dx**3 / g["eps_src"]) if src > 0 else np.zeros(0)
    U, _ = N.solve_step(st, tol=1e-13)

    def Sn(E):
        Gam = K.C_LIGHT * g["sigma_G"] * (theta * E + (1 - theta) * En) / a**3
        return M.riccati_Sn(nHIn, nH, K.ALPHA_B_PAPER / a**3, Gam, dt)

    def h(E):
        kap = g["sigma_E"] * Sn(E) / a**3
        kap0 = g["sigma_E"] * nHIn / a**3
        H = adot / a
        return (E - En - dt * (1 - theta) * (-H * En + src - K.C_LIGHT * kap0 * En)
                - dt * theta * (-H * E + src - K.C_LIGHT * kap * E))

    from scipy.optimize import brentq
    assert h(1e-22) < 0 < h(1e-10)
    Estar = brentq(h, 1e-22, 1e-10, xtol=1e-40, rtol=1e-15)
    np.testing.assert_allclose(U[2], Estar, rtol=1e-10)
    np.testing.assert_allclose(U[1], Sn(Estar), rtol=1e-10)


# ----------------------------------------------------------- Newton machinery


def _smooth_state(shape, seed, isothermal=True):
    w = W.random_state(shape, seed=seed, isothermal=isothermal)
    r = driver.Run(w)
    st = r.make_step()
    z, y, x = np.indices(shape)
    # a smooth positive field so that derivatives are well conditioned
    st.E_n = 1e-18 * (1.5 + np.sin(x) * np.cos(0.7 * y + 0.3 * z))
    return st


def test_complex_step_jacobian_matches_central_differences():
    for iso in (True, False):
        st = _smooth_state((4, 3, 3), 5, isothermal=iso)
        U = N.initial_iterate(st)
        U[2] = st.E_n * 1.7
        U[0] = 3e9 if not iso else 0.0
        J = N.jacobian(st, U).toarray()
        Jfd = N.fd_jacobian_dense(st, U)
        scale = np.abs(Jfd).max(axis=1, keepdims=True) + 1e-300
        assert np.max(np.abs(J - Jfd) / scale) < 1e-5


def test_sparse_solve_matches_dense_lu_8cubed():
    w = W.stromgren_static(n=8)
    st = driver.Run(w).make_step()
    U = N.local_solve(st, N.initial_iterate(st))
    J = N.jacobian(st, U)
    f = M.residual(st, U).ravel()
    s1 = N.linear_solve(J, -f, "direct")
    s2 = np.linalg.solve(J.toarray(), -f)
    np.testing.assert_allclose(s1, s2, rtol=1e-9, atol=1e-12 * np.abs(s2).max())


def test_schur_system_reproduces_full_solve():
    st = _smooth_state((5, 4, 3), 7, isothermal=False)
    U = N.initial_iterate(st)
    U[2] = 1.3 * st.E_n
    U[0] = 1e9
    J = N.jacobian(st, U)
    f = M.residual(st, U)
    s = np.linalg.solve(J.toarray(), -f.ravel()).reshape(U.shape)
    S, r = N.schur_system(st, U)
    sE = np.linalg.solve(S.toarray(), r)
    np.testing.assert_allclose(sE, s[2].ravel(), rtol=1e-8, atol=1e-10 * np.abs(s[2]).max())
    # lagged limiter: the reduced operator is symmetric
    Sd = S.toarray()
    assert np.max(np.abs(Sd - Sd.T)) <= 1e-12 * np.abs(Sd).max()


def test_newton_converges_to_roundoff_nonisothermal():
    w = W.reionization_field(n=8, nsrc=2, box_mpc=14.4 * 8 / 256, ndot_total=1e52 * (8 / 256) ** 3)
    r = driver.Run(w)
    st = r.make_step()
    U, info = N.solve_step(st, tol=1e-11)
    assert info["iters"] <= 10
    f = M.residual(st, U)
    assert M.rms_norm(M.weights(st, U), f) <= 1e-11


# ---------------------------------------------------------------- cosmology


def test_lcdm_expansion_matches_friedmann_integration():
    cos = C.FlatLCDM(**W.LCDM)
    t0, t1 = cos.t_of_z(10.0), cos.t_of_z(4.0)
    sol = integrate.solve_ivp(lambda t, a: [cos.H0 * a[0] * math.sqrt(cos.Om / a[0] ** 3 + cos.OL)],
                              (t0, t1), [1 / 11.0], rtol=1e-12, atol=1e-15)
    assert cos.a(t1) == pytest.approx(sol.y[0, -1], rel=1e-9)
    assert cos.a(t1) == pytest.approx(0.2, rel=1e-12)
    assert cos.adot(t0) == pytest.approx(cos.H0 * (1 / 11) * math.sqrt(0.3 * 11**3 + 0.7), rel=1e-12)


@pytest.mark.parametrize("row", [0, 1, 2, 3])
def test_sg_closed_form_matches_ifront_ode(row):
    """Eqs. SG-solution/SG-tau/SG-F against direct integration of the I-front equation."""
    q0, z0, L0, h, Om, OL, Ob = GOLD["table1"]["rows"][row]
    cos = C.OpenNoLambda(q0, h * K.H100)
    nH0 = Ob * K.RHO_CRIT_H2 * h**2 * (1 + z0) ** 3 / K.M_H
    ndot = GOLD["Ndot_photons_s"]["value"]
    alpha = K.ALPHA_B_PAPER
    a0 = 1 / (1 + z0)
    t0 = cos.t_of_a(a0)
    n_c = nH0 * a0**3
    for abar in (1.5, 2.5):
        t1 = cos.t_of_a(a0 * abar)
        Vc = C.ifront_ode(t0, t1, cos.a, ndot, alpha, n_c)
        r_comoving = (3 * Vc / (4 * math.pi)) ** (1 / 3)
        r_sg = C.sg_ifront(abar, q0, z0, cos.H0, ndot, alpha, nH0)
        assert a0 * r_comoving == pytest.approx(r_sg, rel=1e-7)


def test_static_limit_of_ifront_ode():
    nH, ndot, alpha = 1e-3, 5e48, K.ALPHA_B_PAPER
    t = 0.7 / (alpha * nH)
    Vc = C.ifront_ode(0.0, t, lambda t: 1.0, ndot, alpha, nH)
    assert (3 * Vc / (4 * math.pi)) ** (1 / 3) == pytest.approx(C.static_ifront(t, ndot, alpha, nH), rel=1e-8)
    # paper numbers: R_s for the verification source at n_H = 1e-3
    assert C.stromgren_radius(ndot, alpha, nH) / K.KPC == pytest.approx(5.393, rel=1e-3)


# ------------------------------------------------ full runs against closed forms


@pytest.mark.slow
def test_static_stromgren_front():
    """16^3 octant, 20 steps of 0.01 t_rec (T_B = 1e5 K blackbody): the ionised volume
    follows R_s(1 - e^{-t/t_rec})^{1/3} with the grey model's ionising photon rate
    Ndot eps_src sigma_G / sigma_E (absorbed energy divided by the energy per
    absorbed photon; it equals Ndot for a monochromatic source)."""
    w = W.stromgren_static(n=16)
    r = driver.Run(w)
    g = r.grey
    neff = w["ndot_total"] * g["eps_src"] * g["sigma_G"] / g["sigma_E"]
    mono = S.grey_constants("mono")
    assert w["ndot_total"] * mono["eps_src"] * mono["sigma_G"] / mono["sigma_E"] == pytest.approx(
        w["ndot_total"], rel=1e-14)
    for _ in range(w["nsteps"]):
        r.advance(tol=1e-9)
    rI = D.ifront_radius(r.nHI, w["rho_b"] / K.M_H, w["dx"], True)
    rth = C.static_ifront(r.t, neff, K.ALPHA_B_PAPER, w["nH"])
    assert rI == pytest.approx(rth, rel=0.12)


@pytest.mark.slow
def test_cosmological_stromgren_front_16cubed():
    """LCDM I-front from z = 10 (16^3, 12 steps to z = 8) against the I-front ODE with the
    grey model's ionising photon rate (see test_static_stromgren_front)."""
    w = W.stromgren_cosmo(n=16, z0=10.0, z_end=8.0, nsteps=12)
    r = driver.Run(w)
    g = r.grey
    neff = w["ndot_total"] * g["eps_src"] * g["sigma_G"] / g["sigma_E"]
    for _ in range(w["nsteps"]):
        r.advance(tol=1e-9)
    cos = driver.cosmology_of(w)
    t0 = cos.t_of_z(10.0)
    Vc = C.ifront_ode(t0, r.t, cos.a, neff, K.ALPHA_B_PAPER, w["nH"])
    r_ode = (3 * Vc / (4 * math.pi)) ** (1 / 3)
    rI = D.ifront_radius(r.nHI, w["rho_b"] / K.M_H, w["dx"], True)
    assert rI == pytest.approx(r_ode, rel=0.12)


# ------------------------------------------------ equation of state, diagnostics, local solve


def test_temperature_is_the_monatomic_ideal_gas_temperature():
    """Eqs. eos + temperature with gamma = 5/3: a gas of n_tot = n_H + n_e particles per volume
    at temperature T holds (3/2) n_tot k T of internal energy per volume; with a bulk velocity
    the specific total energy adds |v|^2 / 2.  The oracle's temperature of that state is T."""
    shape = (2, 3, 4)
    rng = np.random.default_rng(4)
    rho = 10 ** rng.uniform(-28, -22, shape)
    nH = rho / K.M_H
    nHI = nH * rng.uniform(1e-6, 1.0, shape)
    T = 10 ** rng.uniform(1, 8, shape)
    v = tuple(rng.normal(0, 3e6, shape) for _ in range(3))
    n_tot = nH + (nH - nHI)
    e_h = 1.5 * n_tot * K.K_BOLTZ * T / rho + 0.5 * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2)
    st = M.Step(nx=4, ny=3, nz=2, dx=1.0, periodic=(True, True, True), rho_b=rho, e_h=e_h, v=v,
                clump=np.ones(shape), E_n=np.zeros(shape), nHI_n=nHI, a=1.0, adot=0.0, dt=1.0,
                src_index=np.array([], np.int64), src_ndot=np.array([]), sigma_E=0.0, sigma_G=0.0,
                eps_src=K.HNU0, isothermal=False)
    np.testing.assert_allclose(M.temperature(st, np.zeros(shape), nHI), T, rtol=1e-10)


def test_ifront_radius_of_a_resolved_sphere():
    """An octant holding a sphere of radius R about the corner, each cell ionised in proportion
    to the part of its volume inside the sphere (from 8^3 sub-cell samples): the equivalent-volume
    radius is R to the sampling error, and with whole-cell ionisation (cell centres inside) the
    error falls as the grid is refined."""
    R = 0.62
    for n in (16, 32):
        dx = 1.0 / n
        s = (np.arange(8) + 0.5) / 8.0
        z, y, x = np.indices((n, n, n))
        frac = np.zeros((n, n, n))
        for a in s:
            for b in s:
                for c in s:
                    frac += (((x + a) * dx) ** 2 + ((y + b) * dx) ** 2 + ((z + c) * dx) ** 2 <= R * R)
        frac /= 512.0
        nH = np.ones((n, n, n))
        rI = D.ifront_radius(nH * (1.0 - frac), nH, dx, True)
        assert rI == pytest.approx(R, rel=2e-3)
    errs = []
    for n in (16, 32, 64):
        dx = 1.0 / n
        z, y, x = np.indices((n, n, n))
        inside = (((x + 0.5) * dx) ** 2 + ((y + 0.5) * dx) ** 2 + ((z + 0.5) * dx) ** 2 <= R * R)
        nH = np.ones((n, n, n))
        errs.append(abs(D.ifront_radius(nH * (1.0 - inside), nH, dx, True) / R - 1.0))
    assert errs[2] < errs[0] and errs[2] < 0.01


def test_local_solve_matches_an_independent_root_finder():
    """The oracle's cell-local solution (damped 2x2 Newton) against SciPy's hybrid Powell method
    on the same local equations, started from the step's starting state, on sampled cells of a
    non-isothermal state: both find the same root."""
    from scipy import optimize
    st = _smooth_state((5, 4, 3), 12, isothermal=False)
    U = N.initial_iterate(st)
    U[2] = 2.0 * st.E_n
    Uo = N.local_solve(st, U)
    rng = np.random.default_rng(0)
    cells = rng.choice(st.N, 12, replace=False)
    se = np.maximum(M.internal_energy_h(st), M.E_FLOOR_INT())
    for c in cells:
        k = np.unravel_index(c, st.shape)

        def f(v):
            ec = np.full(st.shape, Uo[0][k]); n = np.full(st.shape, Uo[1][k])
            ec[k], n[k] = v[0] * se[k], v[1] * st.n_H[k]
            fe, fn = M.local_residual(st, ec, n, U[2])
            return [np.real(fe[k]) / se[k], np.real(fn[k]) / st.n_H[k]]

        sol = optimize.root(f, [0.0, st.nHI_n[k] / st.n_H[k]], method="hybr", tol=1e-14)
        assert sol.success
        assert sol.x[0] * se[k] == pytest.approx(Uo[0][k], rel=1e-8, abs=1e-10 * se[k])
        assert sol.x[1] * st.n_H[k] == pytest.approx(Uo[1][k], rel=1e-8, abs=1e-12 * st.n_H[k])
