"""Gradients of the ionised fraction through the implicit steps (torch.autograd.Function).

``IonizedFraction.apply(ndot, clump, workload, nsteps, options)`` runs ``nsteps`` implicit
steps (each after the advection pre-step when ``options`` has ``advect=True``) on the GPU from
the workload's initial state with the given source photon rates
(photons/s, float64 tensor) and per-cell clumping factor (float32 tensor [z, y, x]),
checkpointing the carried state before each step and the converged state after it, and
returns the final volume-weighted ionised fraction 1 - mean(n_HI / n_H).  Its backward pass
walks the checkpoints in reverse with rt_adjoint_step (the discrete adjoint of each step,
solved with the same Schur reduction and multigrid-preconditioned CG as the forward step) and
rt_advect_adjoint (the transpose of the advection pre-step)
and returns dJ/dNdot and dJ/dC.  The arithmetic runs in the CUDA library; this module
only keeps the checkpoints and marshals arguments.
"""
import ctypes

import numpy as np
import torch

from . import _rt
from .solver import Solver


def _advecting(s):
    return s.advection and s.has_v


def _run_forward(w, ndot, clump, nsteps, options):
    s = Solver(w, **options)
    s.src_ndot.copy_(ndot.to(s.dev, torch.float64))
    s.clump.copy_(clump.to(s.dev, torch.float32))
    ckpts = []
    for _ in range(nsteps):
        if _advecting(s):
            s.advect()
        # the state the implicit step starts from (after the advection pre-step) and its density
        X = (s.E.clone(), s.nHI.clone(), s.e_h.clone(), s.t, s.rho.clone() if _advecting(s) else None)
        s.step(advect=False)
        ckpts.append((X, (s.ec.clone(), s.nHI.clone(), s.E.clone())))
    J = 1.0 - torch.mean(s.nHI / s.rho)
    return s, ckpts, J


def adjoint_sweep(s, ckpts, lam_E, lam_n, lam_eh, nsrc):
    """Accumulate dJ/dNdot, dJ/dC over the checkpointed steps, last step first."""
    L = _rt.lib()
    g_ndot = torch.zeros(nsrc, dtype=torch.float64, device=s.dev)
    g_clump = torch.zeros(s.shape, dtype=torch.float32, device=s.dev)
    lam = _rt.State()
    lam.E, lam.n_HI, lam.e_c = _rt.ptr(lam_E), _rt.ptr(lam_n), _rt.ptr(lam_eh)
    for X, U in reversed(ckpts):
        E0, n0, eh0, t0, rho0 = X
        ec1, n1, E1 = U
        inp = s.inputs(*s.expansion(t0 + 0.5 * s.dt))
        inp.e_h = _rt.ptr(eh0)
        if rho0 is not None:
            inp.rho_b = _rt.ptr(rho0)
        s0 = s.state(E0, n0, torch.zeros_like(E0))
        s1 = s.state(E1, n1, ec1)
        code = L.rt_adjoint_step(s.handle, ctypes.byref(inp), ctypes.byref(s0), ctypes.byref(s1),
                                 ctypes.byref(lam), ctypes.byref(lam), _rt.ptr(g_ndot) if nsrc else None,
                                 _rt.ptr(g_clump))
        _rt.check(code, "rt_adjoint_step")
        if rho0 is not None:
            # through the advection pre-step: the transpose of its linear map
            out_E, out_n = torch.empty_like(lam_E), torch.empty_like(lam_n)
            dst = s.state(out_E, out_n, lam_eh)
            _rt.check(L.rt_advect_adjoint(s.handle, ctypes.byref(inp), ctypes.byref(lam), ctypes.byref(dst)),
                      "rt_advect_adjoint")
            lam_E, lam_n = out_E, out_n
            lam.E, lam.n_HI = _rt.ptr(lam_E), _rt.ptr(lam_n)
    return g_ndot, g_clump


class IonizedFraction(torch.autograd.Function):
    """J = volume-averaged ionised fraction after nsteps implicit steps, as a function of the
    source rates and the clumping field; backward runs the discrete adjoint of every step
    (rt_adjoint_step, and rt_advect_adjoint with advection) from the forward checkpoints."""

    @staticmethod
    def forward(ctx, ndot, clump, w, nsteps, options):
        """Run the forward steps on the GPU, keeping the per-step checkpoints for backward."""
        s, ckpts, J = _run_forward(w, ndot, clump, nsteps, options or {})
        ctx.solver = s
        ctx.ckpts = ckpts
        ctx.nsrc = int(ndot.numel())
        ctx.devices = (ndot.device, clump.device)
        return J.detach().to(ndot.device)

    @staticmethod
    def backward(ctx, gJ):
        """dJ/dNdot and dJ/dC by the adjoint sweep; frees the forward solver."""
        s = ctx.solver
        lam_E = torch.zeros_like(s.E)
        lam_n = -1.0 / (s.rho.numel() * s.rho)       # dJ/dn_HI of the final state
        lam_eh = torch.zeros_like(s.E)
        g_ndot, g_clump = adjoint_sweep(s, ctx.ckpts, lam_E, lam_n.contiguous(), lam_eh, ctx.nsrc)
        s.close()
        ctx.solver = None
        ctx.ckpts = None
        gJ = gJ.to(g_ndot.device)
        return ((gJ * g_ndot).to(ctx.devices[0]), (gJ * g_clump).to(torch.float32).to(ctx.devices[1]),
                None, None, None)


def ionized_fraction(ndot, clump, w, nsteps, **options):
    """Final volume-weighted ionised fraction after nsteps implicit steps (differentiable in
    ndot and clump)."""
    return IonizedFraction.apply(ndot, clump, w, nsteps, options)
