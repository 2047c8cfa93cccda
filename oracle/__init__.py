"""Plain FP64 CPU oracle for the coupled implicit radiation / ionization / heating step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
Python binding) imports, links or executes anything in this package.  The only
callers are ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py``.

The oracle works directly in CGS comoving units (the paper normalises units only
to keep floating-point values in range, which FP64 on the CPU does not need), so
it also checks the product's unit normalisation independently.

What it computes, with the paper passage each module follows:

* ``constants``  -- physical constants (CGS).
* ``spectrum``   -- grey averages over the fixed spectrum chi_E(nu) from the
  hydrogen edge to infinity (Sec. "Physical Model", Eq. grey_definition and the
  T_B = 1e5 K blackbody that follows it; monochromatic 13.6 eV source of the
  verification section).
* ``rates``      -- case-B recombination, photo-heating and the cooling terms
  entering G - Lambda (Sec. "Physical Model", rates cited there).
* ``model``      -- the flux limiter (Eq. limiter), the local solutions S_e, S_n
  (Eqs. gas_residual, chemistry_residual) and the nonlinear residual f(U)
  of step (v) (Eqs. RT-cons_energy .. radiation_residual).
* ``newton``     -- the root of f(U) by a plain full-system Newton method with a
  complex-step Jacobian and sparse direct solves; the Schur complement of the
  linearised system written out with sparse algebra (Sec. "Algorithm"); the
  RMS norm of Eq. rmsnorm.
* ``helium``     -- the same step for hydrogen + helium gas (Eq. electron_density's helium
  case; species n_HI, n_HeI, n_HeII with the rest by conservation).
* ``advection``  -- the donor-cell advection pre-step of step (iv) and its transpose.
* ``multigroup`` -- the step with G radiation groups: Eq. cons_radiation_multifreq integrated
  over frequency groups with the fixed spectrum kept within each group (Sec. "Physical Model").
* ``adjoint``    -- the dense discrete adjoint of a multi-step run.
* ``cosmology``  -- a(t) for the verification cosmologies, the Shapiro-Giroux
  I-front closed form (Eqs. SG-stromgren_radius, SG-solution, SG-tau, SG-F)
  and the expanding-universe I-front ODE.
* ``diagnostics``-- I-front radius of a computed field.
* ``adjoint``    -- dense discrete adjoint of a short run on tiny grids.

Parity status per function is stated in each module's header.  Functions whose
values no paper passage or mathematical fact pins are marked "parity unpinned":
the temperature-dependent recombination fit away from 1e4 K and the cooling
rates (``rates``).
"""
