"""Python driver around the C ABI: device buffers, unit conversion and the step loop.

``Solver`` owns one ``rt_grid`` and the device arrays of one problem.  Input fields are
given in CGS comoving units (the same form the workload generators produce); they are
converted once to the paper's normalised variables and kept on the GPU.  Every step of
the implicit solve runs inside the CUDA library; this module only marshals arguments.
"""
import ctypes

import numpy as np
import torch

from . import _rt
from .cosmology import from_dict as cosmology_from_dict
from .units import Units, specific_energy

_SPECTRA = {"mono": _rt.RT_SPECTRUM_MONO, "blackbody": _rt.RT_SPECTRUM_BLACKBODY}
_RECOMB = {"const": _rt.RT_RECOMB_CONST, "hg97": _rt.RT_RECOMB_HG97}
_BC = {"periodic": _rt.RT_BC_PERIODIC, "reflect": _rt.RT_BC_REFLECT, "outflow": _rt.RT_BC_OUTFLOW}


def _faces(w):
    """Boundary type of the six faces (x-, x+, y-, y+, z-, z+) of workload w: its ``bc`` entry, or
    from ``periodic`` (non-periodic axes reflect at both faces)."""
    if w.get("bc") is not None:
        return tuple(w["bc"])
    return tuple(t for p in w["periodic"] for t in (("periodic",) * 2 if p else ("reflect",) * 2))


class Solver:
    """Implicit FLD + ionisation + heating steps of one workload on one GPU.

    w: workload dict (see ``workloads``), fields in CGS comoving units.
    precision: "fp64" (FP64 multigrid) or "mixed" (FP32 multigrid inside FP64 Newton/CG).
    advect: run the advection pre-step (step (iv) for rho_b, n_HI and E) before every implicit
    step.
    """

    def __init__(self, w, precision="mixed", newton_tol=1e-8, lin_rtol=1e-3, max_newton=40, max_lin=200,
                 nu=(4, 4), theta=None, device=0, stream=None, limiter="lagged", D_const=0.0, E_min=1e-35,
                 advect=False):
        self.w = w
        self.dev = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.dev)
        nx, ny, nz = w["nx"], w["ny"], w["nz"]
        self.shape = (nz, ny, nx)
        self.units = Units.for_grid(w["dx"], float(np.mean(w["rho_b"])))
        u = self.units
        self.theta = w.get("theta", 0.51) if theta is None else theta
        d = _rt.GridDesc()
        d.nx, d.ny, d.nz = nx, ny, nz
        d.dx = w["dx"] / u.u_x
        for f, kind in enumerate(_faces(w)):
            d.bc[f] = _BC[kind]
        d.u_x, d.u_t, d.u_g = u.u_x, u.u_t, u.u_g
        d.theta = self.theta
        d.precision = _rt.RT_MIXED if precision == "mixed" else _rt.RT_FP64
        d.isothermal = int(w["isothermal"])
        d.T_iso = w.get("T_iso", 1e4)
        d.spectrum = _SPECTRA[w["spectrum"]]
        d.T_B = w.get("T_B", 1e5)
        d.recomb = _RECOMB[w["recomb"]]
        d.cooling = 1
        self.helium = bool(w.get("helium", False))
        d.helium = int(self.helium)
        d.Y = float(w.get("Y", 0.0)) if self.helium else 0.0
        d.limiter = _rt.RT_LIMITER_CONST if limiter == "const" else _rt.RT_LIMITER_LAGGED
        d.D_const = D_const
        d.E_min = E_min
        d.newton_tol = newton_tol
        d.max_newton = max_newton
        d.lin_rtol = lin_rtol
        d.max_lin = max_lin
        d.mg_nu1, d.mg_nu2 = nu
        d.device = device
        d.stream = ctypes.c_void_p(self.stream.cuda_stream)
        self.desc = d
        L = _rt.lib()
        h = ctypes.c_void_p()
        _rt.check(L.rt_init_grid(ctypes.byref(d), ctypes.byref(h)), "rt_init_grid")
        self.handle = h

        f64 = dict(dtype=torch.float64, device=self.dev)
        dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).to(**f64)
        self.rho = dev(w["rho_b"] / u.u_d)
        vt = tuple(np.asarray(v, np.float64) for v in w["v"])
        self.v = tuple(dev(v / u.u_v) for v in vt)
        self.has_v = any(np.any(v != 0) for v in vt)
        self.clump = torch.as_tensor(np.ascontiguousarray(w["clump"], dtype=np.float32)).to(self.dev)
        self.src_cell = torch.as_tensor(np.asarray(w["src_index"], np.int64)).to(self.dev)
        self.src_ndot = dev(np.asarray(w["src_ndot"], np.float64))
        self.E = dev(w["E"] / u.u_E)
        self.nHI = dev(w["nHI"] / u.u_n)
        self.ec = torch.zeros(self.shape, **f64)
        he = None
        if self.helium:
            self.nHeI = dev(w["nHeI"] / u.u_n)
            self.nHeII = dev(w["nHeII"] / u.u_n)
            he = (w["Y"], w["nHeI"], w["nHeII"])
        e_h = specific_energy(w["T0"], w["rho_b"], w["nHI"], vt, he)
        self.e_h = dev(e_h / u.u_v**2)
        # time
        cos = w.get("cosmology")
        self.cosmo = cosmology_from_dict(cos) if cos else None
        if self.cosmo is None:
            self.t, self.dt = 0.0, w["dt"]
        else:
            self.t = self.cosmo.t_of_z(w["z0"])
            self.dt = ((self.cosmo.t_of_z(w["z_end"]) - self.t) / w["nsteps"]) if "z_end" in w else w["dt"]
        self.stats = []
        self.advection = bool(advect)
        self._adv = None
        self.courant = None

    # ----------------------------------------------------------------- inputs
    def expansion(self, t):
        """(a, da/dt) at time t [s]; (1, 0) for a static run."""
        if self.cosmo is None:
            return 1.0, 0.0
        return self.cosmo.a(t), self.cosmo.adot(t)

    def inputs(self, a=None, adot=None, dt=None):
        """rt_step_inputs for a step of length dt [s] (default self.dt), a and adot at the
        step's midpoint unless given; device pointers into this solver's tensors."""
        if a is None:
            a, adot = self.expansion(self.t + 0.5 * self.dt)
        dt = self.dt if dt is None else dt
        u = self.units
        s = _rt.StepInputs()
        s.rho_b = _rt.ptr(self.rho)
        s.e_h = _rt.ptr(self.e_h)
        if self.has_v:
            s.vx, s.vy, s.vz = (_rt.ptr(v) for v in self.v)
        s.clump = _rt.ptr(self.clump)
        s.a, s.adot, s.dt = a, adot * u.u_t, dt / u.u_t
        s.nsrc = int(self.src_cell.numel())
        s.src_cell = _rt.ptr(self.src_cell) if s.nsrc else None
        s.src_ndot = _rt.ptr(self.src_ndot) if s.nsrc else None
        return s

    def state(self, E=None, nHI=None, ec=None, nHeI=None, nHeII=None):
        """rt_state over the given normalised device tensors (default: the solver's own)."""
        st = _rt.State()
        st.E = _rt.ptr(self.E if E is None else E)
        st.n_HI = _rt.ptr(self.nHI if nHI is None else nHI)
        st.e_c = _rt.ptr(self.ec if ec is None else ec)
        if self.helium:
            st.n_HeI = _rt.ptr(self.nHeI if nHeI is None else nHeI)
            st.n_HeII = _rt.ptr(self.nHeII if nHeII is None else nHeII)
        return st

    # ------------------------------------------------------------------- steps
    def step(self, fold=True, advect=None):
        """One implicit step (v) in place (after the advection pre-step if ``advect``, default
        the solver's setting), then e_h += e_c; returns the step statistics.  On error the
        state is unchanged (the pre-step writes scratch buffers that are swapped in only when
        the implicit step succeeds)."""
        L = _rt.lib()
        stats = _rt.StepStats()
        inp = self.inputs()
        adv = (self.advection if advect is None else advect) and self.has_v
        if adv:
            sc = self._advect_to_scratch(inp)
            inp.rho_b = _rt.ptr(sc[2])
            st = self.state(sc[0], sc[1], None, *sc[3:5])
        else:
            st = self.state()
        code = L.rt_implicit_step(self.handle, ctypes.byref(inp), ctypes.byref(st), ctypes.byref(stats))
        if code != _rt.RT_OK:
            err = _rt.RTError(code, "rt_implicit_step")
            err.stats = stats.as_dict()
            raise err
        if adv:
            self._swap_advected()
        if fold and not self.w["isothermal"]:
            _rt.check(L.rt_fold_energy(self.handle, _rt.ptr(self.e_h), _rt.ptr(self.ec)), "rt_fold_energy")
        self.t += self.dt
        self.stats.append(stats.as_dict())
        return self.stats[-1]

    # failures after which a smaller step is worth trying
    RETRY_CODES = (_rt.RT_ENOCONV, _rt.RT_ELINESEARCH, _rt.RT_ENONFINITE, _rt.RT_ELINEAR)

    def advance(self, t_end, tau_tol=1e-3, dt_max=None, growth=2.0, max_halvings=30, newton_target=8):
        """Steps from the current time to t_end with the time step chosen from the solution
        change: after a step with scaled change eps (``change_norm`` of the step statistics),
        the next step is dt min(growth, tau_tol / eps), capped by dt_max and t_end.  A step the
        solver fails on is retried with half the step (the state is unchanged on failure); the
        step after a retry does not grow, nor does one after a step that needed more than
        ``newton_target`` Newton iterations (beyond 1.5 x that target it shrinks by 0.7).
        Starts from the solver's current dt and leaves the next proposed step there; returns
        [(t, dt, stats)] of the accepted steps (stats gain ``rejected``: retries before it)."""
        out = []
        dt = self.dt
        while self.t < t_end * (1.0 - 1e-12):
            dt = min(dt, t_end - self.t)
            if dt_max is not None:
                dt = min(dt, dt_max)
            rejected = 0
            while True:
                self.dt = dt
                try:
                    st = self.step()
                    break
                except _rt.RTError as e:
                    if e.code not in self.RETRY_CODES or rejected >= max_halvings:
                        raise
                    rejected += 1
                    dt *= 0.5
            st["rejected"] = rejected
            out.append((self.t, dt, st))
            eps = st["change_norm"]
            factor = growth if eps <= tau_tol / growth else tau_tol / eps
            if rejected or st["newton_iters"] > newton_target:
                factor = min(factor, 1.0)
            if st["newton_iters"] > 1.5 * newton_target:
                factor = min(factor, 0.7)
            dt *= factor
            self.dt = dt            # the proposal carries over to the next call
        return out

    def _advect_to_scratch(self, inp):
        if self._adv is None:
            self._adv = tuple(torch.empty_like(self.E) for _ in range(5 if self.helium else 3))
        c = ctypes.c_double()
        src = self.state()
        dst = self.state(self._adv[0], self._adv[1], None, *(self._adv[3:5] if self.helium else ()))
        _rt.check(_rt.lib().rt_advect(self.handle, ctypes.byref(inp), ctypes.byref(src), ctypes.byref(dst),
                                      _rt.ptr(self.rho), _rt.ptr(self._adv[2]), ctypes.byref(c)), "rt_advect")
        self.courant = c.value
        return self._adv

    def _swap_advected(self):
        cur = (self.E, self.nHI, self.rho) + ((self.nHeI, self.nHeII) if self.helium else ())
        self.E, self.nHI, self.rho = self._adv[:3]
        if self.helium:
            self.nHeI, self.nHeII = self._adv[3:5]
        self._adv = cur

    def advect(self):
        """Advection pre-step (step (iv) for rho_b, n_HI, E and the helium species, donor
        cell) over this step's dt, in place; returns the largest Courant number."""
        self._advect_to_scratch(self.inputs())
        self._swap_advected()
        return self.courant

    # ---------------------------------------------------------- kernel access
    def to_device(self, a, scale):
        """A host array in CGS as a normalised FP64 device tensor (a / scale)."""
        return torch.as_tensor(np.ascontiguousarray(a / scale, dtype=np.float64)).to(self.dev)

    def residual(self, U_n, U, a=None, adot=None):
        """f(U) (CGS) for the step starting from U_n = (E, nHI); U = (e_c, nHI, E) in CGS."""
        u = self.units
        En, nn = self.to_device(U_n[0], u.u_E), self.to_device(U_n[1], u.u_n)
        ec, n, E = self.to_device(U[0], u.u_v**2), self.to_device(U[1], u.u_n), self.to_device(U[2], u.u_E)
        fe, fn, fE = (torch.empty_like(E) for _ in range(3))
        inp = self.inputs(a, adot)
        s0, s1 = self.state(En, nn, torch.zeros_like(En)), self.state(E, n, ec)
        _rt.check(_rt.lib().rt_residual(self.handle, ctypes.byref(inp), ctypes.byref(s0), ctypes.byref(s1),
                                        _rt.ptr(fe), _rt.ptr(fn), _rt.ptr(fE)), "rt_residual")
        return np.stack([fe.cpu().numpy() * u.u_v**2, fn.cpu().numpy() * u.u_n, fE.cpu().numpy() * u.u_E])

    def schur_system(self, U_n, U, a=None, adot=None):
        """(diag, wx, wy, wz, rhs[CGS]) of the reduced system at U (CGS inputs)."""
        u = self.units
        En, nn = self.to_device(U_n[0], u.u_E), self.to_device(U_n[1], u.u_n)
        ec, n, E = self.to_device(U[0], u.u_v**2), self.to_device(U[1], u.u_n), self.to_device(U[2], u.u_E)
        out = [torch.empty_like(E) for _ in range(5)]
        inp = self.inputs(a, adot)
        s0, s1 = self.state(En, nn, torch.zeros_like(En)), self.state(E, n, ec)
        _rt.check(_rt.lib().rt_schur_system(self.handle, ctypes.byref(inp), ctypes.byref(s0), ctypes.byref(s1),
                                            *[_rt.ptr(t) for t in out]), "rt_schur_system")
        d, wx, wy, wz, r = (t.cpu().numpy() for t in out)
        return d, wx, wy, wz, r * u.u_E

    def schur_solve(self, b, rtol=1e-10, max_iters=500):
        """Solve the last assembled reduced system for a right side b (normalised units)."""
        bt = torch.as_tensor(np.ascontiguousarray(b, dtype=np.float64)).to(self.dev)
        x = torch.zeros_like(bt)
        its = ctypes.c_int()
        _rt.check(_rt.lib().rt_schur_solve(self.handle, _rt.ptr(bt), _rt.ptr(x), rtol, max_iters, ctypes.byref(its)),
                  "rt_schur_solve")
        return x.cpu().numpy(), its.value

    def state_cgs(self):
        """(e_c, n_HI, E) in CGS; with helium (e_c, n_HI, n_HeI, n_HeII, E)."""
        u = self.units
        out = [self.ec.cpu().numpy() * u.u_v**2, self.nHI.cpu().numpy() * u.u_n]
        if self.helium:
            out += [self.nHeI.cpu().numpy() * u.u_n, self.nHeII.cpu().numpy() * u.u_n]
        return tuple(out + [self.E.cpu().numpy() * u.u_E])

    def residual_helium(self, U_n, U, a=None, adot=None):
        """f(U) (CGS, five components) for a helium grid; U_n = (E, nHI, nHeI, nHeII),
        U = (e_c, nHI, nHeI, nHeII, E), CGS."""
        u = self.units
        En, nn, h1n, h2n = (self.to_device(x, s) for x, s in zip(U_n, (u.u_E, u.u_n, u.u_n, u.u_n)))
        ec, n, h1, h2, E = (self.to_device(x, s) for x, s in zip(U, (u.u_v**2, u.u_n, u.u_n, u.u_n, u.u_E)))
        out = [torch.empty_like(E) for _ in range(5)]
        inp = self.inputs(a, adot)
        s0 = self.state(En, nn, torch.zeros_like(En), h1n, h2n)
        s1 = self.state(E, n, ec, h1, h2)
        _rt.check(_rt.lib().rt_residual_helium(self.handle, ctypes.byref(inp), ctypes.byref(s0), ctypes.byref(s1),
                                               *[_rt.ptr(t) for t in out]), "rt_residual_helium")
        scale = (u.u_v**2, u.u_n, u.u_n, u.u_n, u.u_E)
        return np.stack([t.cpu().numpy() * sc for t, sc in zip(out, scale)])

    def grey(self):
        """The grey constants the library derived (CGS): sigma_E, sigma_G, eps_src."""
        vals = [ctypes.c_double() for _ in range(3)]
        _rt.check(_rt.lib().rt_grey_constants(self.handle, *[ctypes.byref(v) for v in vals]), "rt_grey_constants")
        return dict(sigma_E=vals[0].value, sigma_G=vals[1].value, eps_src=vals[2].value)

    def set_profiling(self, on):
        """Enable (and reset) or disable the library's per-kernel event timing."""
        _rt.check(_rt.lib().rt_set_profiling(self.handle, int(on)), "rt_set_profiling")

    def profile(self):
        """{kernel class: {launches, ms, bytes}} accumulated since profiling was enabled."""
        buf = (_rt.KernelProfile * 32)()
        n = ctypes.c_int()
        _rt.check(_rt.lib().rt_get_profile(self.handle, buf, 32, ctypes.byref(n)), "rt_get_profile")
        return {buf[i].name.decode(): dict(launches=buf[i].launches, ms=buf[i].ms, bytes=buf[i].bytes)
                for i in range(min(n.value, 32))}

    def close(self):
        """Destroy the library grid (idempotent)."""
        if self.handle:
            _rt.lib().rt_destroy_grid(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
