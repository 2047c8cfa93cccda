"""Multi-step runs of the oracle on a workload from ``workloads`` (test infrastructure only).

Between steps the operator split of Sec. "Operator-Split Hydrodynamics with
Radiative Feedback" hands the implicit solve the hydro state; with no hydro the
only hand-over is the gas energy, e_h^{n+1} = e_h^n + e_c^{n+1}.  The expansion
factor of a step is taken at its midpoint time (reading: the paper does not say
where in the step a and adot are evaluated).
"""
import numpy as np

from . import constants as K
from . import cosmology as C
from . import model as M
from . import newton as N
from . import spectrum as S


def energy_from_temperature(T, rho_b, nHI, v):
    """Specific total energy for temperature T (Eqs. eos, temperature; X = 1)."""
    nH = rho_b / K.M_H
    e_int = K.K_BOLTZ * T * (2.0 * nH - nHI) / ((K.GAMMA - 1.0) * rho_b)
    return e_int + 0.5 * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2)


def cosmology_of(w):
    """The workload's expansion history (None for a static run): the Lambda-free models of
    Table 1 when the workload names q0, flat LCDM otherwise."""
    c = w.get("cosmology")
    if c is None:
        return None
    if "q0" in c:                               # the Lambda-free models of Table 1
        return C.OpenNoLambda(c["q0"], c["h"] * K.H100)
    return C.FlatLCDM(**c)


def time_grid(w):
    """(t0, dt) of a workload: static runs start at t = 0."""
    cos = cosmology_of(w)
    if cos is None:
        return 0.0, w["dt"]
    t0 = cos.t_of_z(w["z0"])
    if "z_end" in w:
        return t0, (cos.t_of_z(w["z_end"]) - t0) / w["nsteps"]
    return t0, w["dt"]


def expansion(w, t):
    """(a, da/dt) at time t; (1, 0) for a static run."""
    cos = cosmology_of(w)
    if cos is None:
        return 1.0, 0.0
    return float(cos.a(t)), float(cos.adot(t))


class Run:
    """State of a multi-step oracle run."""

    def __init__(self, w, theta=None):
        self.w = w
        self.theta = w.get("theta", 0.51) if theta is None else theta
        self.grey = S.grey_constants(w["spectrum"], w.get("T_B", 1e5))
        self.E = np.array(w["E"], float)
        self.nHI = np.array(w["nHI"], float)
        self.rho_b = np.array(w["rho_b"], float)
        self.e_h = energy_from_temperature(w["T0"], w["rho_b"], self.nHI, w["v"])
        self.t, self.dt = time_grid(w)
        self.step_index = 0

    def make_step(self, a=None, adot=None, dt=None):
        """The implicit step (v) from the current state: a and adot at the step's midpoint
        time unless given."""
        w = self.w
        if a is None:
            a, adot = expansion(w, self.t + 0.5 * self.dt)
        return M.Step(
            nx=w["nx"], ny=w["ny"], nz=w["nz"], dx=w["dx"], periodic=w["periodic"], bc=w.get("bc"),
            rho_b=self.rho_b, e_h=self.e_h, v=w["v"], clump=np.asarray(w["clump"], float),
            E_n=self.E, nHI_n=self.nHI, a=a, adot=adot, dt=self.dt if dt is None else dt,
            src_index=w["src_index"], src_ndot=w["src_ndot"],
            theta=self.theta, isothermal=w["isothermal"], T_iso=w["T_iso"], recomb=w["recomb"],
            **self.grey)

    def advance(self, tol=1e-11, **kw):
        """Solve one step (v) to the RMS norm tol and hand it over: E and n_HI replaced,
        e_h += e_c, t += dt.  Returns the root U and the Newton record."""
        st = self.make_step()
        U, info = N.solve_step(st, tol=tol, **kw)
        e_c, nHI, E = U
        self.E, self.nHI = E, nHI
        self.e_h = self.e_h + e_c
        self.t += self.dt
        self.step_index += 1
        return U, info
