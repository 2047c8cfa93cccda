"""Root of f(U) = 0 for one implicit step, by a plain method (oracle; test infrastructure only).

Sec. "Algorithm": the time-evolved state U^{n+1} is the solution of f(U) = 0, found
by a globalised inexact Newton method whose linear systems J(U_k) S_k = -f(U_k) are
reduced by a Schur complement to a modified radiation equation.  The oracle reaches
the same root by the plainest route:

  * J(U) by complex steps, Im f(U + i h e_j) / h, on the full 3N unknowns (the
    columns are grouped by a colouring of the 7-point stencil so that no two
    columns in a group touch the same row);
  * each Newton step from a sparse direct solve of the full (unreduced) system;
  * the cell-local unknowns (e_c, n_HI) re-solved exactly from the local equations
    after each update of E (nonlinear elimination; n_HI then stays in (0, n_H));
  * step length halved until the RMS norm (Eq. rmsnorm, component-scaled) decreases.

``schur_system`` writes out the Schur complement S = J_EE - J_Eu J_uu^{-1} J_uE and
its right side -f_E + J_Eu J_uu^{-1} f_u with sparse algebra, for comparison with
the reduced system the CUDA path assembles.  There J holds the FLD coefficient D
fixed (``freeze=True``), the linearisation that keeps the reduced operator
symmetric for the conjugate-gradient solver the paper names.

Pinned by: complex-step Jacobian against central differences; the sparse solve
against a dense LU on 8^3 grids; convergence of f to round-off.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import model as M

_FIELDS = 3  # (e_c, n_HI, E)


def _colours_per_axis(n, periodic):
    if n <= 3:
        return n
    if not periodic:
        return 3
    for m in range(3, n + 1):
        if n % m == 0:
            return m
    return n


def _offsets():
    return [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]


def _neighbour(st, o):
    """Flat index of cell + o (offset in x, y, z) and whether it exists."""
    z, y, x = np.indices(st.shape)
    valid = np.ones(st.shape, bool)
    coords = []
    for d, (c, n) in enumerate(((x, st.nx), (y, st.ny), (z, st.nz))):
        cc = c + o[d]
        if st.periodic[d]:
            cc = cc % n
        else:
            valid &= (cc >= 0) & (cc < n)
            cc = np.clip(cc, 0, n - 1)
        coords.append(cc)
    flat = (coords[2] * st.ny + coords[1]) * st.nx + coords[0]
    return flat.ravel(), valid.ravel()


def _scales(st, U):
    e_c, nHI, E = np.real(U)
    s_e = np.maximum(np.abs(e_c), M.E_FLOOR_INT()) + 0 * E
    s_n = st.n_H + 0 * E
    s_E = np.maximum(np.abs(E), st.E_min)
    return np.stack([s_e, s_n, s_E]).reshape(_FIELDS, -1)


def jacobian(st, U, bE=None, freeze=False, h=1e-30, residual=None, scales=None):
    """Sparse 3N x 3N Jacobian of ``model.residual`` by coloured complex steps.

    Unknowns and equations are ordered [e_c (N), n_HI (N), E (N)], cells flat [z,y,x].
    ``residual`` / ``scales`` substitute another cell-local model with the same stencil
    (hydrogen + helium: ``oracle.helium``); the field count is U's first dimension.
    """
    if bE is None:
        bE = M.explicit_part(st)
    residual = M.residual if residual is None else residual
    scales = _scales if scales is None else scales
    nf = np.shape(U)[0]
    N = st.N
    for n, per in zip((st.nx, st.ny, st.nz), st.periodic):
        if per and n < 3:
            raise ValueError("oracle Jacobian needs >= 3 cells along a periodic axis")
    U = np.asarray(U, dtype=float)
    mx = _colours_per_axis(st.nx, st.periodic[0])
    my = _colours_per_axis(st.ny, st.periodic[1])
    mz = _colours_per_axis(st.nz, st.periodic[2])
    z, y, x = np.indices(st.shape)
    colour = ((x % mx) + mx * ((y % my) + my * (z % mz))).ravel()
    ncol = mx * my * mz
    scale = scales(st, U)
    nbrs = [_neighbour(st, o) for o in _offsets()]
    rows, cols, vals = [], [], []
    for fi in range(nf):
        for c in range(ncol):
            pert = np.zeros((nf, N), complex)
            sel = colour == c
            pert[fi, sel] = 1j * h * scale[fi, sel]
            Uc = U.astype(complex) + pert.reshape((nf,) + st.shape)
            fc = np.imag(residual(st, Uc, bE, freeze)).reshape(nf, N) / h
            for nb, valid in nbrs:
                r = np.nonzero(valid & (colour[nb] == c))[0]
                cc = nb[r]
                for fo in range(nf):
                    v = fc[fo, r] / scale[fi, cc]
                    nz = v != 0.0
                    rows.append(fo * N + r[nz])
                    cols.append(fi * N + cc[nz])
                    vals.append(v[nz])
    J = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nf * N, nf * N))
    return J


def fd_jacobian_dense(st, U, bE=None, rel=1e-6):
    """Dense central-difference Jacobian (tiny grids; used only to pin ``jacobian``)."""
    if bE is None:
        bE = M.explicit_part(st)
    N = st.N
    U = np.asarray(U, dtype=float)
    scale = _scales(st, U).ravel()
    flat = U.reshape(-1)
    J = np.zeros((_FIELDS * N, _FIELDS * N))
    for j in range(_FIELDS * N):
        hj = rel * scale[j]
        up = flat.copy(); up[j] += hj
        dn = flat.copy(); dn[j] -= hj
        fp = M.residual(st, up.reshape(U.shape), bE).ravel()
        fm = M.residual(st, dn.reshape(U.shape), bE).ravel()
        J[:, j] = (fp - fm) / (2 * hj)
    return J


def linear_solve(J, rhs, method="auto"):
    """Solve J s = rhs: sparse LU (SuperLU) or, for large systems, Jacobi-preconditioned BiCGStab."""
    n = J.shape[0]
    if method == "dense":
        return np.linalg.solve(J.toarray(), rhs)
    if method == "direct" or (method == "auto" and n <= 3 * 40**3):
        return spla.spsolve(J.tocsc(), rhs)
    dinv = 1.0 / J.diagonal()
    P = spla.LinearOperator(J.shape, matvec=lambda v: dinv * v)
    s, info = spla.bicgstab(J, rhs, M=P, rtol=1e-14, atol=0.0, maxiter=20000)
    if info != 0:
        raise RuntimeError(f"oracle BiCGStab did not converge (info={info})")
    return s


def fraction_to_boundary(st, U, S, tau=0.99):
    """Largest step in (0, 1] keeping E > 0, 0 < n_HI < n_H and e_int > 0, times tau."""
    e_c, nHI, E = np.real(U)
    se, sn, sE = S
    lam = 1.0
    with np.errstate(divide="ignore", invalid="ignore"):
        cand = [np.where(sE < 0, -E / sE, np.inf),
                np.where(sn < 0, -nHI / sn, np.inf),
                np.where(sn > 0, (st.n_H - nHI) / sn, np.inf)]
        if not st.isothermal:
            eint = M.internal_energy_h(st) + e_c
            cand.append(np.where(se < 0, -eint / se, np.inf))
    m = min(float(np.min(c)) for c in cand)
    if m <= 1.0:
        lam = tau * m
    return lam


def initial_iterate(st):
    """U_0 = (e_c^n = 0, n_HI*, E* + dt 4 pi eta): the advected state that step (v) starts
    from, with the step's emission added to E.  In a source cell the absorbed power
    c kappa(n_HI(E)) E is not monotone in E (the cell turns transparent as it ionises), so
    the step can have a neutral and an ionised branch; starting above both, Newton
    descends to the ionised one instead of stalling at the fold of the neutral one."""
    return np.stack([np.zeros(st.shape), st.nHI_n.copy(), st.E_n + st.dt * M.emissivity(st)])


def local_solve(st, U, tol=1e-14, maxit=60):
    """Solve the cell-local equations f_e = f_n = 0 for (e_c, n_HI) at fixed E.

    Isothermal runs: e_c = 0 and n_HI = S_n(E) directly.  Otherwise a per-cell damped
    2x2 Newton iteration with complex-step derivatives: each step is halved until the
    scaled local residual max(|f_e|/e_int, |f_n|/n_H) decreases, keeping 0 < n_HI <= n_H
    and the internal energy positive.
    """
    e_c, nHI, E = (np.array(x, float) for x in U)
    if st.isothermal:
        return np.stack([np.zeros_like(E), np.real(M.local_solutions(st, (e_c, nHI, E))[1]), E])
    h = 1e-30
    se = np.maximum(M.internal_energy_h(st), M.E_FLOOR_INT())
    sn = st.n_H
    eint_h = M.internal_energy_h(st)

    def scaled(fe, fn):         # max of the weighted local residual components
        return np.maximum(np.abs(fe) / se, np.abs(fn) / sn)

    nHI = np.clip(nHI, 1e-300, st.n_H)
    fe, fn = (np.real(x) for x in M.local_residual(st, e_c, nHI, E))
    r = scaled(fe, fn)
    for _ in range(maxit):
        active = r > tol
        if not np.any(active):
            break
        fe1, fn1 = M.local_residual(st, e_c + 1j * h * se, nHI, E)
        fe2, fn2 = M.local_residual(st, e_c, nHI + 1j * h * sn, E)
        a11, a21 = np.imag(fe1) / (h * se), np.imag(fn1) / (h * se)
        a12, a22 = np.imag(fe2) / (h * sn), np.imag(fn2) / (h * sn)
        det = a11 * a22 - a12 * a21
        de = np.where(active, -(a22 * fe - a12 * fn) / det, 0.0)
        dn = np.where(active, -(-a21 * fe + a11 * fn) / det, 0.0)
        lam = np.ones_like(e_c)
        todo = active.copy()
        for _ in range(40):
            ec_t = e_c + lam * de
            # keep the internal energy positive and the neutral density inside (0, n_H]
            ec_t = np.maximum(ec_t, -0.999 * eint_h)
            n_t = np.clip(nHI + lam * dn, 1e-300, st.n_H)
            fe_t, fn_t = (np.real(x) for x in M.local_residual(st, ec_t, n_t, E))
            r_t = scaled(fe_t, fn_t)
            ok = todo & (r_t < r)
            e_c = np.where(ok, ec_t, e_c)
            nHI = np.where(ok, n_t, nHI)
            fe = np.where(ok, fe_t, fe)
            fn = np.where(ok, fn_t, fn)
            r = np.where(ok, r_t, r)
            todo &= ~ok
            if not np.any(todo):
                break
            lam = np.where(todo, 0.5 * lam, lam)
        if np.any(todo & (r > 1e-9)):
            # no decrease along the Newton direction: the cell sits at its round-off floor
            # or needs more iterations; leave it for the next outer iteration
            pass
    return np.stack([e_c, nHI, E])


def solve_step(st, tol=1e-11, maxit=60, freeze=False, linear="auto", U0=None, verbose=False):
    """Globalised Newton iteration for f(U) = 0; returns (U, info).

    Each iteration solves the full linearised system J s = -f for the radiation
    update s_E and replaces the linear update of the cell-local unknowns by
    the exact solution of the local equations at the new E (nonlinear elimination:
    the reduced system's Jacobian is the Schur complement of J, so the E-step is the
    Newton step of the reduced problem).  Backtracking halves the step until the
    RMS norm decreases (Armijo, c = 1e-4).  Stops when the component-scaled RMS
    norm of f is <= tol.  The root does not depend on ``freeze``.
    """
    bE = M.explicit_part(st)
    U = initial_iterate(st) if U0 is None else np.array(U0, float)
    U = local_solve(st, U)
    hist = []
    for k in range(maxit + 1):
        f = M.residual(st, U, bE)
        w = M.weights(st, U)
        nrm = M.rms_norm(w, f)
        hist.append(nrm)
        if verbose:
            print(f"  oracle newton {k}: |f| = {nrm:.3e}")
        if not np.isfinite(nrm):
            raise FloatingPointError("oracle residual is not finite")
        if nrm <= tol:
            return U, dict(iters=k, hist=hist)
        if k == maxit:
            break
        J = jacobian(st, U, bE, freeze)
        S = linear_solve(J, -f.ravel(), linear).reshape(U.shape)
        sE = S[2]
        lam = 1.0
        for _ in range(40):
            Ut = U.copy()
            Ut[2] = U[2] + lam * sE
            Ut = local_solve(st, Ut)
            nt = M.rms_norm(w, M.residual(st, Ut, bE))
            if nt <= (1.0 - 1e-4 * lam) * nrm and nt < nrm:
                break
            lam *= 0.5
        else:
            if nrm <= 1e-9:
                # no further decrease is possible: the residual is at its round-off floor
                return U, dict(iters=k, hist=hist, floor=True)
            raise RuntimeError("oracle line search failed")
        U = Ut
    raise RuntimeError(f"oracle Newton did not converge: {hist[-5:]}")


def schur_system(st, U, bE=None):
    """(S, r): S = J_EE - J_Eu J_uu^-1 J_uE and r = -f_E + J_Eu J_uu^-1 f_u (sparse, N x N),
    u = (e_c, n_HI).

    The cell-local equations make J_uu block diagonal (one 2x2 block per cell, checked
    here); its inverse is formed block by block with numpy and the products are sparse.
    """
    if bE is None:
        bE = M.explicit_part(st)
    N = st.N
    J = jacobian(st, U, bE, freeze=True).tocsr()
    f = M.residual(st, U, bE).reshape(_FIELDS, N)
    Juu = J[: 2 * N, : 2 * N].tocoo()
    JuE = J[: 2 * N, 2 * N:]
    JEu = J[2 * N:, : 2 * N]
    JEE = J[2 * N:, 2 * N:]
    if np.any((Juu.row % N) != (Juu.col % N)):
        raise AssertionError("J_uu couples different cells")
    blocks = np.zeros((N, 2, 2))
    np.add.at(blocks, (Juu.row % N, Juu.row // N, Juu.col // N), Juu.data)
    inv = np.linalg.inv(blocks)
    cells = np.arange(N)
    rows = np.concatenate([a * N + cells for a in (0, 0, 1, 1)])
    cols = np.concatenate([b * N + cells for b in (0, 1, 0, 1)])
    vals = np.concatenate([inv[:, 0, 0], inv[:, 0, 1], inv[:, 1, 0], inv[:, 1, 1]])
    Juu_inv = sp.csr_matrix((vals, (rows, cols)), shape=(2 * N, 2 * N))
    S = JEE - JEu @ (Juu_inv @ JuE)
    r = -f[2] + JEu @ (Juu_inv @ f[:2].ravel())
    return sp.csr_matrix(S), r
