"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module only builds inputs (grids, fields, source lists, time-step settings)
in CGS comoving units.  It contains none of the solver's arithmetic: no rates,
no unit normalisation, no equation of state.  Temperatures are handed out as
temperatures; each side converts them to gas energy with its own code.

The fixed-step workloads use the two-level parameter theta = 1: with the paper's
theta = 0.51 and steps this long, stiff absorption modes change sign every step and
the nonlinear solve fails to converge (the paper avoids that regime with its
time-step error control, which these fixed-step runs do not have).  Random-state
parity cases use theta = 0.51.

Workloads (sizes and values follow the paper's verification and reionization
set-ups; the reionization field stands in for the paper's Enzo initial
conditions, which are not available):

* ``stromgren_static``   -- isothermal Stromgren sphere in a static universe:
  uniform n_H = 1e-3 cm^-3 in a 6.6 kpc box, x_HI = 0.9999, T = 1e4 K,
  E = 1e-35 erg/cm^3, one corner source of 5e48 photons/s (one octant of it is
  inside the box: reflecting lower faces, Ndot/8 emitted into the octant; outflow at the
  upper faces, as in the paper's verification problem).
* ``stromgren_cosmo``    -- the same source in a comoving box of 400 kpc at the
  mean baryon density of flat LCDM (Omega_m 0.3, Omega_b 0.04, h 0.7), z = 10.
* ``reionization_field`` -- periodic 14.4 Mpc comoving box at z = 9: log-normal
  density (ln rho Gaussian, P(k) ~ k^-2.5, sigma_ln = 1, mean preserved),
  Gaussian random peculiar velocities (sigma 30 km/s per component, same
  spectral shape), point sources on the highest density peaks (26-neighbour
  local maxima) with Ndot proportional to density (total 1e52 photons/s),
  3^3 ionised blocks (x_HI = 1e-4, T = 1e4 K) around sources, elsewhere
  x_HI = 0.9999 and T = 100 K.
* ``shapiro_giroux``     -- the four cosmological I-front problems of the verification
  section (Table 1: q0 in {0.5, 0.05}, z0 in {4, 10}, box L0 proper at z0, H0, Omega_b):
  uniform gas at Omega_b rho_crit (1+z0)^3 (the quoted rho_b0 for z0 = 4), fully neutral,
  T = 1e4 K (isothermal), E = 1e-35 erg/cm^3, one monochromatic 13.6 eV corner source of
  5e48 photons/s (octant, reflecting lower and outflow upper faces), case-B alpha = 2.59e-13,
  run from z0 to z = 0
  in steps evenly spaced in log t.
* ``random_state``       -- random but physical states on small grids, for
  element-wise parity of single kernels.
* ``with_helium``        -- the hydrogen + helium version of any of them (helium mass
  fraction Y = 0.24, helium singly ionised where hydrogen is ionised).
"""
import numpy as np

KPC = 3.0856775814913673e21
MPC = 1e3 * KPC
MYR = 3.15576e13
KM = 1e5
M_H = 1.6735575e-24            # g: rho_b = M_H n_H for hydrogen-only gas
ALPHA_B_PAPER = 2.59e-13       # cm^3/s, used only to express dt in recombination times
E_FLOOR = 1e-35                # erg/cm^3, initial radiation energy density (paper)

LCDM = dict(Omega_m=0.3, Omega_L=0.7, Omega_b=0.04, h=0.7)
RHO_CRIT_H2 = 1.8784723e-29    # g/cm^3 per h^2 (critical density today)


# boundaries of the verification problems: reflecting at the lower faces, outflow at the upper
# faces, per face in the order (x-, x+, y-, y+, z-, z+)
PAPER_BC = ("reflect", "outflow") * 3


def _base(n, L, periodic, bc=None):
    """Grid shape, cell width and boundaries; bc (six face types) overrides periodic, whose axes
    otherwise reflect at both faces."""
    nx, ny, nz = (n, n, n) if np.isscalar(n) else n
    if bc is None:
        bc = tuple(t for p in periodic for t in (("periodic",) * 2 if p else ("reflect",) * 2))
    bc = tuple(bc)
    periodic = tuple(bc[2 * d] == "periodic" for d in range(3))
    return dict(nx=int(nx), ny=int(ny), nz=int(nz), dx=float(L) / nx, periodic=periodic, bc=bc)


def stromgren_static(n=16, dt_over_trec=1e-2, nsteps=20, spectrum="blackbody", nH=1e-3,
                     box_kpc=6.6, ndot=5e48, theta=1.0, bc=PAPER_BC):
    """Static-universe Stromgren sphere (octant: reflecting lower faces, outflow upper faces,
    source in cell 0)."""
    w = _base(n, box_kpc * KPC, (False, False, False), bc)
    shape = (w["nz"], w["ny"], w["nx"])
    t_rec = 1.0 / (ALPHA_B_PAPER * nH)
    w.update(
        rho_b=np.full(shape, nH * M_H),
        T0=np.full(shape, 1e4),
        v=tuple(np.zeros(shape) for _ in range(3)),
        clump=np.ones(shape, np.float32),
        E=np.full(shape, E_FLOOR),
        nHI=np.full(shape, 0.9999 * nH),
        src_index=np.array([0], np.int64),
        src_ndot=np.array([ndot / 8.0]),
        ndot_total=ndot, octant=True,
        cosmology=None, a0=1.0, dt=dt_over_trec * t_rec, nsteps=nsteps, t_rec=t_rec, nH=nH,
        isothermal=True, T_iso=1e4, recomb="const", spectrum=spectrum, T_B=1e5, theta=theta,
    )
    return w


def stromgren_cosmo(n=128, z0=10.0, z_end=4.0, nsteps=500, box_kpc_comoving=400.0, ndot=5e48,
                    spectrum="blackbody", theta=1.0, bc=PAPER_BC):
    """Cosmological Stromgren sphere in flat LCDM (octant, boundaries as stromgren_static); the
    driver advances a(t) from z0."""
    w = _base(n, box_kpc_comoving * KPC, (False, False, False), bc)
    shape = (w["nz"], w["ny"], w["nx"])
    nH = LCDM["Omega_b"] * RHO_CRIT_H2 * LCDM["h"] ** 2 / M_H
    w.update(
        rho_b=np.full(shape, nH * M_H),
        T0=np.full(shape, 1e4),
        v=tuple(np.zeros(shape) for _ in range(3)),
        clump=np.ones(shape, np.float32),
        E=np.full(shape, E_FLOOR),
        nHI=np.full(shape, 0.9999 * nH),
        src_index=np.array([0], np.int64),
        src_ndot=np.array([ndot / 8.0]),
        ndot_total=ndot, octant=True,
        cosmology=dict(LCDM), z0=z0, z_end=z_end, nsteps=nsteps, nH=nH,
        isothermal=True, T_iso=1e4, recomb="const", spectrum=spectrum, T_B=1e5, theta=theta,
    )
    return w


# Table 1 of the verification section: q0, z0, L0 [kpc, proper at z0], H0 [100 km/s/Mpc],
# Omega_m, Omega_Lambda, Omega_b
SG_TABLE1 = ((0.5, 4.0, 80.0, 0.5, 1.0, 0.0, 0.2),
             (0.05, 4.0, 60.0, 1.0, 0.1, 0.0, 0.1),
             (0.5, 10.0, 36.0, 0.5, 1.0, 0.0, 0.2),
             (0.05, 10.0, 27.0, 1.0, 0.1, 0.0, 0.1))


def shapiro_giroux(row, n=32, nsteps=200, ndot=5e48, theta=1.0, bc=PAPER_BC):
    """Row ``row`` of Table 1 (see the module docstring); comoving box L0 (1 + z0)."""
    q0, z0, L0, h, Om, OL, Ob = SG_TABLE1[row]
    w = _base(n, L0 * KPC * (1.0 + z0), (False, False, False), bc)
    shape = (w["nz"], w["ny"], w["nx"])
    nH = Ob * RHO_CRIT_H2 * h**2 / M_H            # comoving (proper at z0: times (1 + z0)^3)
    w.update(
        rho_b=np.full(shape, nH * M_H),
        T0=np.full(shape, 1e4),
        v=tuple(np.zeros(shape) for _ in range(3)),
        clump=np.ones(shape, np.float32),
        E=np.full(shape, E_FLOOR),
        nHI=np.full(shape, nH),
        src_index=np.array([0], np.int64),
        src_ndot=np.array([ndot / 8.0]),
        ndot_total=ndot, octant=True,
        cosmology=dict(q0=q0, h=h), z0=z0, z_end=0.0, nsteps=nsteps, time_steps="log", nH=nH,
        sg=dict(q0=q0, z0=z0, L0_kpc=L0, h=h, Omega_b=Ob),
        isothermal=True, T_iso=1e4, recomb="const", spectrum="mono", T_B=1e5, theta=theta,
    )
    return w


def with_helium(w, Y=0.24):
    """Hydrogen + helium version of workload w: helium mass fraction Y (n_H = (1 - Y) rho / m_H,
    n_He = Y rho / (4 m_H)), the hydrogen neutral fraction kept, and helium singly ionised
    where hydrogen is ionised (n_HeI = x_HI n_He, n_HeII = (1 - x_HI) n_He, no HeIII)."""
    w = dict(w)
    rho = np.asarray(w["rho_b"], float)
    xHI = np.asarray(w["nHI"], float) * M_H / rho
    nHe = Y * rho / (4.0 * M_H)
    w.update(helium=True, Y=Y, nHI=xHI * (1.0 - Y) * rho / M_H, nHeI=xHI * nHe, nHeII=(1.0 - xHI) * nHe)
    return w


def _gaussian_field(shape, slope, rng):
    """Zero-mean unit-variance Gaussian random field with P(k) ~ k^slope (k = 0 removed)."""
    nz, ny, nx = shape
    kz = np.fft.fftfreq(nz)[:, None, None]
    ky = np.fft.fftfreq(ny)[None, :, None]
    kx = np.fft.rfftfreq(nx)[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    amp = k2 ** (slope / 4.0)
    amp[0, 0, 0] = 0.0
    noise = rng.standard_normal(shape)
    g = np.fft.irfftn(np.fft.rfftn(noise) * amp, s=shape, axes=(0, 1, 2))
    g -= g.mean()
    return g / g.std()


def _local_maxima(rho):
    """Boolean mask of cells strictly greater than their 26 periodic neighbours."""
    m = np.ones(rho.shape, bool)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dz == dy == dx == 0:
                    continue
                m &= rho > np.roll(rho, (dz, dy, dx), axis=(0, 1, 2))
    return m


def reionization_field(n=256, nsrc=2000, seed=9001, box_mpc=14.4, z0=9.0, dt_myr=1.0, nsteps=100,
                       ndot_total=1e52, sigma_ln=1.0, slope=-2.5, v_sigma_kms=30.0, theta=1.0):
    """Reionization-like periodic field at z0 (shapes and recipe in the module docstring)."""
    w = _base(n, box_mpc * MPC, (True, True, True))
    shape = (w["nz"], w["ny"], w["nx"])
    rng = np.random.default_rng(seed)
    g = _gaussian_field(shape, slope, rng) * sigma_ln
    nH_mean = LCDM["Omega_b"] * RHO_CRIT_H2 * LCDM["h"] ** 2 / M_H
    rho = nH_mean * M_H * np.exp(g - 0.5 * sigma_ln**2)
    v = tuple(_gaussian_field(shape, slope, np.random.default_rng(seed + 1 + i)) * v_sigma_kms * KM
              for i in range(3))
    peaks = np.flatnonzero(_local_maxima(rho))
    order = np.lexsort((peaks, -rho.ravel()[peaks]))      # densest first, ties by index
    src = np.sort(peaks[order[:nsrc]])
    ndot = rho.ravel()[src] / rho.ravel()[src].sum() * ndot_total
    xHI = np.full(shape, 0.9999)
    T0 = np.full(shape, 100.0)
    zc, yc, xc = np.unravel_index(src, shape)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                idx = ((zc + dz) % shape[0], (yc + dy) % shape[1], (xc + dx) % shape[2])
                xHI[idx] = 1e-4
                T0[idx] = 1e4
    w.update(
        rho_b=rho, T0=T0, v=v, clump=np.ones(shape, np.float32),
        E=np.full(shape, E_FLOOR), nHI=xHI * rho / M_H,
        src_index=src.astype(np.int64), src_ndot=ndot, ndot_total=ndot_total, octant=False,
        cosmology=dict(LCDM), z0=z0, dt=dt_myr * MYR, nsteps=nsteps,
        isothermal=False, T_iso=1e4, recomb="hg97", spectrum="blackbody", T_B=1e5, theta=theta,
    )
    return w


def random_state(shape, seed=0, periodic=(True, True, True), isothermal=True, nsrc=3, box_kpc=100.0,
                 theta=0.51, dt_myr=None, bc=None):
    """A random physical state for element-wise kernel parity.

    Densities n_H in [1e-4, 1e-2] cm^-3, neutral fractions log-uniform in [1e-6, 1),
    E log-uniform over 1e-30 .. 1e-12 erg/cm^3 (with smooth and rough parts),
    T in [100, 3e4] K, clumping in [1, 3], velocities ~ 10 km/s.
    """
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    w = _base((nx, ny, nz), box_kpc * KPC, periodic, bc)
    nH = 10 ** rng.uniform(-4, -2, shape)
    xHI = 10 ** rng.uniform(-6, -1e-6, shape)
    E = 10 ** rng.uniform(-30, -12, shape)
    w.update(
        rho_b=nH * M_H,
        T0=10 ** rng.uniform(2, np.log10(3e4), shape),
        v=tuple(rng.normal(0, 10 * KM, shape) for _ in range(3)),
        clump=rng.uniform(1, 3, shape).astype(np.float32),
        E=E, nHI=xHI * nH,
        src_index=rng.choice(nx * ny * nz, size=nsrc, replace=False).astype(np.int64),
        src_ndot=10 ** rng.uniform(46, 49, nsrc),
        ndot_total=None, octant=False,
        cosmology=None, a0=1.0, dt=(rng.uniform(0.1, 2.0) if dt_myr is None else dt_myr) * MYR,
        nsteps=1, isothermal=isothermal, T_iso=1e4, recomb="const" if isothermal else "hg97",
        spectrum="blackbody", T_B=1e5, theta=theta,
    )
    return w
