"""Pins of the oracle's advection pre-step (step (iv), Eqs. enzo-chemical_ionization and
enzo-cons_radiation, donor-cell reading) against what the scheme's definition fixes: the
textbook one-dimensional upwind update, the exact shift at Courant number 1, conservation,
brute-force face loops on a tiny grid, first-order convergence to the exact translation, and
the conservation dual of the adjoint."""
import numpy as np
import pytest

from oracle import advection as A

AXES = (2, 1, 0)


def _uniform(shape, d, speed):
    v = [np.zeros(shape) for _ in range(3)]
    v[d] = np.full(shape, speed)
    return v


@pytest.mark.parametrize("d", [0, 1, 2])
@pytest.mark.parametrize("c", [0.3, -0.45])
def test_uniform_velocity_is_textbook_upwind(d, c):
    rng = np.random.default_rng(d)
    shape = (5, 6, 7)
    q = rng.random(shape)
    a, dt, dx = 0.5, 2.0, 3.0
    v = _uniform(shape, d, c * a * dx / dt)
    out = A.advect(q, v, a, dt, dx, (True, True, True))
    ax = AXES[d]
    if c > 0:
        ref = (1 - c) * q + c * np.roll(q, 1, ax)          # inflow from the '-' neighbour
    else:
        ref = (1 + c) * q - c * np.roll(q, -1, ax)         # inflow from the '+' neighbour
    assert np.allclose(out, ref, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_courant_one_is_an_exact_shift(d):
    q = 10 ** np.random.default_rng(1).uniform(-20, 0, (4, 5, 6))
    for sgn in (1.0, -1.0):
        out = A.advect(q, _uniform(q.shape, d, sgn), 1.0, 1.0, 1.0, (True, True, True))
        ref = np.roll(q, int(sgn), AXES[d])
        # q_i - (q_i - q_neighbour): exact up to the update's two roundings
        assert np.all(np.abs(out - ref) <= 4.5e-16 * np.maximum(np.abs(q), np.abs(ref)))


@pytest.mark.parametrize("periodic", [(True, True, True), (False, False, False), (True, False, True)])
def test_conserves_total_and_keeps_constants_under_uniform_flow(periodic):
    rng = np.random.default_rng(2)
    shape = (6, 5, 8)
    q = rng.random(shape)
    v = [rng.normal(size=shape) for _ in range(3)]
    cmax = A.max_courant(v, 1.0, 1.0, 1.0, periodic)
    dt = 0.9 / cmax
    out = A.advect(q, v, 1.0, dt, 1.0, periodic)
    assert abs(out.sum() - q.sum()) < 1e-13 * q.sum()
    assert out.min() >= 0.0                                # positivity at Courant <= 1
    if all(periodic):
        u = [np.full(shape, x) for x in (0.2, -0.1, 0.3)]
        assert np.allclose(A.advect(np.full(shape, 2.5), u, 1.0, 1.0, 1.0, periodic), 2.5, rtol=1e-15)


def _brute(q, v, a, dt, dx, periodic):
    """Face-by-face loops over a tiny grid, straight from the scheme's definition."""
    nz, ny, nx = q.shape
    n = (nx, ny, nz)
    out = q.copy()
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                p = [x, y, z]
                for d in range(3):
                    if p[d] + 1 == n[d] and not periodic[d]:
                        continue                           # wall face
                    r = list(p)
                    r[d] = (p[d] + 1) % n[d]
                    i, j = (p[2], p[1], p[0]), (r[2], r[1], r[0])
                    vf = 0.5 * (v[d][i] + v[d][j])
                    c = vf * dt / (a * dx)
                    flux = c * (q[i] if c > 0 else q[j])
                    out[i] -= flux
                    out[j] += flux
    return out


def test_matches_brute_force_face_loops_and_matrix():
    rng = np.random.default_rng(3)
    shape = (3, 4, 5)
    q = rng.random(shape)
    v = [rng.normal(size=shape) for _ in range(3)]
    per = (True, False, True)
    ref = _brute(q, v, 1.3, 0.2, 0.7, per)
    assert np.allclose(A.advect(q, v, 1.3, 0.2, 0.7, per), ref, rtol=1e-13, atol=1e-15)
    M = A.operator_matrix(shape, v, 1.3, 0.2, 0.7, per)
    assert np.allclose((M @ q.ravel()).reshape(shape), ref, rtol=1e-13, atol=1e-15)
    c = A.max_courant(v, 1.3, 0.2, 0.7, per)
    # brute-force Courant: outflow of each cell = M's diagonal deficit
    assert c == pytest.approx(float(np.max(1.0 - M.diagonal())), rel=1e-13)


def test_first_order_convergence_to_exact_translation():
    errs = []
    for n in (64, 128, 256):
        x = (np.arange(n) + 0.5) / n
        L, speed, T = 1.0, 1.0, 0.25
        dx = L / n
        dt = 0.5 * dx / speed
        q = np.exp(-((x - 0.3) / 0.05) ** 2)[None, None, :] * np.ones((1, 1, n))
        v = _uniform(q.shape, 0, speed)
        for _ in range(int(round(T / dt))):
            q = A.advect(q, v, 1.0, dt, dx, (True, True, True))
        exact = np.exp(-((x - 0.3 - speed * T) / 0.05) ** 2)
        errs.append(np.sum(np.abs(q[0, 0] - exact)) * dx)
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 1.5 < r1 < 2.3 and 1.6 < r2 < 2.3, errs


def test_adjoint_is_the_transpose_and_preserves_uniform_adjoints():
    rng = np.random.default_rng(4)
    shape = (4, 3, 6)
    v = [rng.normal(size=shape) for _ in range(3)]
    per = (False, True, False)
    dt = 0.8 / A.max_courant(v, 1.0, 1.0, 1.0, per)
    q, lam = rng.random(shape), rng.random(shape)
    lhs = np.sum(A.advect(q, v, 1.0, dt, 1.0, per) * lam)
    rhs = np.sum(q * A.advect_adjoint(lam, v, 1.0, dt, 1.0, per))
    assert lhs == pytest.approx(rhs, rel=1e-13)
    # conservation (1^T M = 1^T) means a uniform adjoint field is carried unchanged
    assert np.allclose(A.advect_adjoint(np.ones(shape), v, 1.0, dt, 1.0, per), 1.0, rtol=1e-14)
