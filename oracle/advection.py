"""Advection pre-step of the species and radiation densities (oracle; test infrastructure only).

Sec. "Operator-Split Hydrodynamics with Radiative Feedback", step (iv): the baryon velocity v_b
carries the chemical number densities and the radiation energy density,

    d_t n_i + (1/a) div(n_i v_b) = 0,      d_t E + (1/a) div(E v_b) = 0

(Eqs. enzo-chemical_ionization and enzo-cons_radiation), giving the advected (n_i^*, E^*) from
which step (v) starts.  The baryon density moves with the same velocity (Eq. enzo-cons_mass,
here in its conservative form) and is transported with the same fluxes, so that n_HI / n_H stays
a convex combination of neighbouring fractions.  The paper hands this to the hydrodynamics code
(PPM); here it is the first-order donor-cell (upwind) finite-volume scheme, written out plainly:

  * the velocity on a face is the mean of the two cells' components normal to it;
  * the face Courant number is c_f = v_f dt / (a dx) (dx comoving, a the expansion factor);
  * the flux through the face is c_f times the density of the cell the flow leaves;
  * q*_i = q_i minus the net outward flux through the six faces of cell i;
  * on a wall axis the two boundary faces carry no flux.

Arrays are [z, y, x]; ``periodic`` is ordered (x, y, z) like the workloads.  Any consistent
units work: v, dt and dx only enter through the dimensionless c_f.

The map q -> q* is linear.  ``operator_matrix`` assembles it as a sparse matrix M from the
same definition, face by face, so the adjoint of the pre-step is M^T.
"""
import numpy as np
import scipy.sparse as sp

_AXES = (2, 1, 0)          # numpy axis of x, y, z


def face_courant(v, axis, periodic, a, dt, dx):
    """c_f on the '+' face of every cell along numpy axis ``axis`` (0 beyond a wall)."""
    c = 0.5 * (v + np.roll(v, -1, axis)) * dt / (a * dx)
    if not periodic:
        idx = [slice(None)] * 3
        idx[axis] = -1
        c[tuple(idx)] = 0.0
    return c


def advect(q, v, a, dt, dx, periodic):
    """q* of one donor-cell step.  v = (vx, vy, vz) arrays [z, y, x]."""
    q = np.asarray(q, dtype=np.float64)
    out = q.copy()
    for d in range(3):
        ax = _AXES[d]
        c = face_courant(np.asarray(v[d], np.float64), ax, periodic[d], a, dt, dx)
        up = np.where(c > 0, q, np.roll(q, -1, ax))       # the cell the flow leaves
        F = c * up                                        # flux through the '+' face
        out = out - (F - np.roll(F, 1, ax))               # '+' face out, '-' face in
    return out


def max_courant(v, a, dt, dx, periodic):
    """Largest per-cell sum of outflow Courant numbers (the donor-cell scheme keeps q >= 0
    and is stable while it is at most 1)."""
    tot = 0.0
    for d in range(3):
        ax = _AXES[d]
        c = face_courant(np.asarray(v[d], np.float64), ax, periodic[d], a, dt, dx)
        tot = tot + np.maximum(c, 0.0) + np.maximum(-np.roll(c, 1, ax), 0.0)
    return float(np.max(tot))


def operator_matrix(shape, v, a, dt, dx, periodic):
    """Sparse M with advect(q) = M q (flattened [z, y, x])."""
    nz, ny, nx = shape
    N = nx * ny * nz
    idx = np.arange(N).reshape(shape)
    rows, cols, vals = [np.arange(N)], [np.arange(N)], [np.ones(N)]
    for d in range(3):
        ax = _AXES[d]
        c = face_courant(np.asarray(v[d], np.float64), ax, periodic[d], a, dt, dx).ravel()
        i = idx.ravel()
        j = np.roll(idx, -1, ax).ravel()                  # the '+' neighbour
        donor = np.where(c > 0, i, j)
        # the face flux c q_donor leaves cell i and enters cell j
        rows += [i, j]
        cols += [donor, donor]
        vals += [-c, c]
    M = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    return M.tocsr()


def advect_adjoint(lam, v, a, dt, dx, periodic):
    """M^T lam: the adjoint of the pre-advection state from that of the advected state."""
    lam = np.asarray(lam, dtype=np.float64)
    M = operator_matrix(lam.shape, v, a, dt, dx, periodic)
    return (M.T @ lam.ravel()).reshape(lam.shape)
