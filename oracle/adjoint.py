"""Dense discrete adjoint of a multi-step run (oracle; test infrastructure only).

Each implicit step n maps the carried state X^n = (E^n, n_HI^n, e_h^n) to the root U of
f(U; X^n, p) = 0 (Eqs. gas_residual, chemistry_residual, radiation_residual), U = (e_c,
n_HI, E), and hands X^{n+1} = (E, n_HI, e_h^n + e_c) to the next step.  For an objective
J(X^K) the adjoint recursion of this map is

    J_U^T mu = lambda_U,   lambda_U = (lambda_eh, lambda_n, lambda_E) of X^{n+1},
    lambda^n = -J_X^T mu  (+ lambda_eh passed straight to e_h^n),
    dJ/dp   += -J_p^T mu,

with J_U = df/dU, J_X = df/dX^n and J_p = df/dp, all formed here densely by complex
steps (tiny grids only).  Parameters p: the photon rates Ndot_s of the sources and the
per-cell clumping factor C.  Objective: the volume-weighted ionised fraction
1 - mean(n_HI / n_H) of the final state.

With ``advect=True`` every step is preceded by the advection pre-step of n_HI and E
(``oracle.advection``, step (iv)), a linear map M: the implicit step starts from (M E, M n_HI,
e_h) with density M rho_b, and the adjoint of the pre-advection state is M^T applied to the
adjoint of the advected one (rho_b does not depend on the parameters, so it needs no adjoint;
the objective uses the final density).

Pinned in tests against central finite differences of the whole forward run.
"""
import numpy as np

from . import advection as ADV
from . import constants as K
from . import driver
from . import model as M
from . import newton as N


def ionised_fraction(nHI, nH):
    """Objective J of the gradient checks: the volume-averaged ionised fraction 1 - <n_HI/n_H>."""
    return float(1.0 - np.mean(nHI / nH))


def _step_from(run, X, p_ndot, p_clump):
    """Step object of ``run`` with carried state X = (E, nHI, e_h) and parameters p."""
    run.E, run.nHI, run.e_h = X
    st = run.make_step()
    st.src_ndot = p_ndot
    st.clump = p_clump
    return st


def _residual_of(st, U, X=None, ndot=None, clump=None):
    """f(U) with (optionally complex) start state X and parameters replaced."""
    import copy
    s2 = copy.copy(st)
    if X is not None:
        s2.E_n, s2.nHI_n, s2.e_h = X
    if ndot is not None:
        s2.src_ndot = ndot
    if clump is not None:
        s2.clump = clump
    return M.residual(s2, U).ravel()


def _advect_args(w, run):
    a, _ = driver.expansion(w, run.t + 0.5 * run.dt)
    return w["v"], a, run.dt, w["dx"], w["periodic"]


def forward(w, ndot, clump, nsteps, tol=1e-11, advect=False):
    """Run nsteps oracle steps; returns (J, checkpoints) with checkpoints[n] = (X^n, U^n, step,
    advection arguments or None), X^n the state the implicit step starts from."""
    run = driver.Run(w)
    X = (run.E.copy(), run.nHI.copy(), run.e_h.copy())
    ckpt = []
    for _ in range(nsteps):
        adv = _advect_args(w, run) if advect else None
        if adv:
            X = (ADV.advect(X[0], *adv), ADV.advect(X[1], *adv), X[2])
            run.rho_b = ADV.advect(run.rho_b, *adv)
        st = _step_from(run, X, ndot, clump)
        U, _ = N.solve_step(st, tol=tol)
        ckpt.append((X, U, st, adv))
        run.t += run.dt
        X = (U[2].copy(), U[1].copy(), X[2] + U[0])
    return ionised_fraction(X[1], run.rho_b / K.M_H), ckpt


def gradient(w, ndot, clump, nsteps, tol=1e-11, h=1e-30, advect=False):
    """(J, dJ/dNdot, dJ/dC) by the dense discrete adjoint."""
    Jval, ckpt = forward(w, ndot, clump, nsteps, tol, advect)
    shape = (w["nz"], w["ny"], w["nx"])
    Nc = int(np.prod(shape))
    nH = ckpt[-1][2].rho_b / K.M_H               # final density
    # lambda of the final carried state (E, nHI, e_h)
    lam_E = np.zeros(Nc)
    lam_n = (-1.0 / (Nc * nH)).ravel()
    lam_eh = np.zeros(Nc)
    g_ndot = np.zeros(len(ndot))
    g_clump = np.zeros(Nc)
    for X, U, st, adv in reversed(ckpt):
        Uc = np.asarray(U, float)
        JU = N.jacobian(st, Uc).toarray()
        lam_U = np.concatenate([lam_eh, lam_n, lam_E])
        mu = np.linalg.solve(JU.T, lam_U)
        # J_X by complex steps on the carried start state
        JX = np.zeros((3 * Nc, 3 * Nc))
        scales = [np.maximum(np.abs(X[0]), st.E_min), nH, np.maximum(np.abs(X[2]), 1.0)]
        for f in range(3):
            for k in range(Nc):
                Xc = [np.array(x, complex) for x in X]
                hs = h * scales[f].ravel()[k]
                Xc[f].ravel()[k] += 1j * hs
                JX[:, f * Nc + k] = np.imag(_residual_of(st, Uc, X=tuple(Xc))) / hs
        lamX = -JX.T @ mu                       # ordered (E, nHI, e_h) columns
        lam_E = lamX[:Nc]
        lam_n = lamX[Nc:2 * Nc]
        lam_eh = lamX[2 * Nc:] + lam_eh          # e_h^{n+1} = e_h^n + e_c passes lambda_eh through
        if adv:                                  # through the advection pre-step: M^T
            lam_E = ADV.advect_adjoint(lam_E.reshape(shape), *adv).ravel()
            lam_n = ADV.advect_adjoint(lam_n.reshape(shape), *adv).ravel()
        for s in range(len(ndot)):
            nd = np.array(ndot, complex)
            hs = h * abs(ndot[s])
            nd[s] += 1j * hs
            g_ndot[s] += -mu @ (np.imag(_residual_of(st, Uc, ndot=nd)) / hs)
        for k in range(Nc):
            cc = np.array(st.clump, complex)
            cc.ravel()[k] += 1j * h
            g_clump[k] += -mu @ (np.imag(_residual_of(st, Uc, clump=cc)) / h)
    return Jval, g_ndot, g_clump.reshape(shape)
