/*
 * rt.h -- C ABI of the GB300 implicit radiation / ionisation / heating solver.
 *
 * The library advances one operator-split step (v) of Norman, Reynolds & So,
 * "Cosmological Radiation Hydrodynamics with Enzo" (Sec. "Algorithm",
 * subsection "Operator-Split Hydrodynamics with Radiative Feedback"): it solves
 * the coupled system of Eqs. RT-cons_energy, RT-chemical_ionization and
 * RT-cons_radiation for U = (e_c, n_HI, E) on a uniform Cartesian grid by
 * driving the residual of Eqs. gas_residual, chemistry_residual and
 * radiation_residual to zero with a globalised inexact Newton method.  Each
 * Newton system is reduced by a Schur complement to a modified radiation
 * equation (a 7-point symmetric operator in E), solved by conjugate gradients
 * preconditioned with geometric multigrid.  Hydrogen-only gas (N_s = 1), or hydrogen +
 * helium (N_s = 3: n_HI, n_HeI, n_HeII; rt_grid_desc.helium) with Eq. electron_density's
 * helium case.
 *
 * Units.  All fields are in the paper's normalised comoving variables
 * (Eqs. units, scalings, proper_vars): x~ = x/u_x, t~ = t/u_t, rho~ = rho/u_d,
 * e~ = e/u_v^2, E~ = E/u_E with u_d = u_g/u_x^3, u_v = u_x/u_t, u_E = u_d u_v^2;
 * number densities n~ = n/u_n with u_n = u_d/m_H (so n~_H = rho~ for X = 1).
 * E and n are comoving densities (proper = comoving / a^3), v_b is the proper
 * peculiar velocity.  Source rates are photons per second (physical).
 *
 * Memory.  Every array argument is a DEVICE pointer to a contiguous FP64 array
 * of nx*ny*nz values in [z][y][x] order (x fastest) unless stated otherwise,
 * owned by the caller.  The library owns its workspace (allocated in
 * rt_init_grid, freed in rt_destroy_grid) and enqueues all work on the stream
 * given in the descriptor; every call returns after synchronising that stream.
 *
 * Errors.  Functions return RT_OK (0) or one of the positive codes below; no C++
 * exception crosses the ABI.  On any error the caller's output arrays are left
 * unchanged; rt_error_string() gives a message.  The last error's detail text is
 * available from rt_last_error_detail().
 */
#ifndef RT_H
#define RT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RT_OK 0
#define RT_EINVAL 1        /* invalid argument or grid shape                         */
#define RT_ENOMEM 2        /* device allocation failed                               */
#define RT_ECUDA 3         /* a CUDA call failed                                     */
#define RT_ENOCONV 4       /* Newton did not reach newton_tol within max_newton      */
#define RT_ELINESEARCH 5   /* backtracking could not reduce the residual norm        */
#define RT_ENONFINITE 6    /* a residual or linear-solver quantity became NaN/Inf    */
#define RT_ELINEAR 7       /* the linear solver did not reach lin_rtol in max_lin    */

/* Boundary type of a face (Sec. "Verification tests": reflecting at the lower faces, outflow at
 * the upper faces).  PERIODIC must be set on both faces of an axis.  REFLECT (alias WALL): no
 * flux through the face.  OUTFLOW: radiation leaves freely -- the cell beyond the face is an empty
 * ghost (E = 0) holding a copy of the boundary cell's gas, and the face's flux-limited diffusion
 * coefficient follows Eq. limiter between the two (free-streaming limit: c E / 2 per unit area). */
enum { RT_BC_PERIODIC = 0, RT_BC_REFLECT = 1, RT_BC_WALL = 1, RT_BC_OUTFLOW = 2 };
enum { RT_FP64 = 0, RT_MIXED = 1 };                     /* multigrid precision          */
enum { RT_SPECTRUM_MONO = 0, RT_SPECTRUM_BLACKBODY = 1 };
enum { RT_RECOMB_CONST = 0, RT_RECOMB_HG97 = 1 };
enum { RT_LIMITER_LAGGED = 0, RT_LIMITER_CONST = 1 };

/* Grid and solver description (rt_init_grid copies it). */
typedef struct {
    int nx, ny, nz;       /* cells per axis; each level coarsened by 2 while all dims are even
                             and the level has more cells than the coarse-level bound (4096
                             FP32 / 2048 FP64); a level above that bound with an odd dim is
                             rejected with RT_EINVAL                                         */
    double dx;            /* comoving cell width, normalised (cm / u_x)                     */
    int bc[6];            /* boundary per face (x-, x+, y-, y+, z-, z+): RT_BC_PERIODIC on both
                             faces of an axis, else RT_BC_REFLECT or RT_BC_OUTFLOW per face   */
    double u_x, u_t, u_g; /* unit factors of Eq. units: cm, s, g                               */
    double theta;         /* two-level time parameter of Eq. radiation_residual (paper: 0.51) */
    int precision;        /* RT_FP64 or RT_MIXED (FP32 multigrid inside FP64 Newton/CG)       */
    int isothermal;       /* 1: T = T_iso and f_e = e_c                                        */
    double T_iso;         /* K                                                               */
    int spectrum;         /* RT_SPECTRUM_MONO (13.6 eV) or RT_SPECTRUM_BLACKBODY              */
    double T_B;           /* blackbody temperature, K                                        */
    int recomb;           /* RT_RECOMB_CONST (alpha_B = 2.59e-13) or RT_RECOMB_HG97           */
    int cooling;          /* non-isothermal runs: 1 = include Lambda                          */
    int helium;           /* 0: hydrogen only (n_H = rho / m_H); 1: hydrogen + helium with
                             mass fraction Y (n_H = (1-Y) rho / m_H, n_He = Y rho / (4 m_H)),
                             species n_HI, n_HeI, n_HeII in the state, n_e = n_HII + n_HeII +
                             2 n_HeIII (Eq. electron_density with number densities)          */
    double Y;             /* helium mass fraction, 0 <= Y < 1 (helium = 1)                   */
    int limiter;          /* RT_LIMITER_LAGGED (Eq. limiter at the step's start state) or
                             RT_LIMITER_CONST (D = D_const, a test mode)                      */
    double D_const;       /* proper diffusion coefficient for RT_LIMITER_CONST, cm^2/s        */
    double E_min;         /* radiation floor of the limiter and rate smoothing, erg/cm^3
                             (paper's initial value 1e-35); 0 selects 1e-35                  */
    double newton_tol;    /* RMS norm (Eq. rmsnorm, component-scaled) at which Newton stops   */
    int max_newton;       /* Newton iterations per step                                      */
    double lin_rtol;      /* relative reduction of the weighted Schur residual per solve      */
    int max_lin;          /* CG iterations per Newton system                                 */
    int mg_nu1, mg_nu2;   /* red-black Gauss-Seidel sweeps before / after coarse correction  */
    int device;           /* CUDA device ordinal                                             */
    void* stream;         /* cudaStream_t to enqueue on (NULL = legacy default stream)       */
} rt_grid_desc;

/* Per-step inputs from the rest of the operator split (steps (i)-(iv)); device pointers. */
typedef struct {
    const double* rho_b;  /* comoving baryon density (normalised)                            */
    const double* e_h;    /* specific total gas energy after hydro (normalised)              */
    const double* vx;     /* proper peculiar velocity components (normalised); NULL = 0      */
    const double* vy;
    const double* vz;
    const float* clump;   /* clumping factor on the recombination term; NULL = 1             */
    double a, adot, dt;   /* expansion factor, da/dt~ and step length in normalised time     */
    int nsrc;             /* number of point sources                                         */
    const int64_t* src_cell;  /* DEVICE: flat [z][y][x] index of each source's cell          */
    const double* src_ndot;   /* DEVICE: ionising photons per second of each source           */
} rt_step_inputs;

/* Caller-owned state, device pointers, normalised units. */
typedef struct {
    double* E;            /* radiation energy density                                        */
    double* n_HI;         /* neutral hydrogen number density                                 */
    double* e_c;          /* gas energy correction of step (v) (specific)                    */
    double* n_HeI;        /* helium grids only: neutral and singly ionised helium number     */
    double* n_HeII;       /* densities (n_HeIII = n_He - n_HeI - n_HeII); unused otherwise   */
} rt_state;

#define RT_STATS_HIST 64
typedef struct {
    int newton_iters;     /* accepted Newton updates                                         */
    int residual_evals;   /* fused residual/Jacobian evaluations (incl. rejected trials)     */
    int linear_iters;     /* CG iterations summed over the step                              */
    int line_search_cuts; /* step halvings                                                   */
    double norm0;         /* RMS norm of f at the initial iterate                            */
    double norm;          /* RMS norm of f at the returned state                             */
    double change_norm;   /* RMS over the 3N (helium: 5N) unknowns of the step's change,
                             scaled like the norm (E by max(|E^{n+1}|, |E^n|, E_floor), n_HI
                             by n_H, helium by n_He, e_c by the hydro internal energy): the
                             measure a time-step controller
                             compares with its tolerance (0 unless the step succeeded)      */
    int kernel_launches;  /* kernels this call launched                                      */
    int nhist;            /* entries used in the histories below                             */
    double hist_norm[RT_STATS_HIST];  /* per evaluation: RMS norm (trial norms use the weights
                                         of the current iterate)                             */
    double hist_lam[RT_STATS_HIST];   /* per evaluation: step length of the trial (0 = start) */
    int hist_cg[RT_STATS_HIST];       /* per Newton iteration: CG iterations (negative when the
                                         requested reduction was not reached)                 */
} rt_step_stats;

typedef struct rt_grid rt_grid;   /* opaque */

/* Allocate workspace and precompute the grey spectral constants (Eq. grey_definition) and
 * unit factors.  *out receives the handle (NULL on error).  All descriptor checks run before
 * any CUDA call.  Errors: RT_EINVAL (shape, units, parameters), RT_ENOMEM, RT_ECUDA. */
int rt_init_grid(const rt_grid_desc* desc, rt_grid** out);

/* One implicit step (v): on entry *inout holds the advected state (E*, n_HI*, and n_HeI*,
 * n_HeII* on helium grids; e_c is ignored and taken as 0), on success it holds U^{n+1} with
 * f(U^{n+1}) below newton_tol.
 * stats may be NULL.  It describes the attempt on success, on RT_ENOCONV and RT_ELINESEARCH,
 * and on any error the linear solve returns.  It is left as the caller passed it on argument
 * errors, on a non-finite residual evaluation and on CUDA errors outside the linear solve.
 * The hydro state in `in` is checked on the device first: a density that is not positive and
 * finite, a non-finite energy or (non-isothermal grids) a non-positive internal energy
 * e_h - |v|^2/2 in any cell gives RT_EINVAL before anything is written.
 * Errors: RT_EINVAL, RT_ENOCONV, RT_ELINESEARCH, RT_ENONFINITE, RT_ELINEAR,
 * RT_ECUDA; *inout is unchanged on error. */
int rt_implicit_step(rt_grid* g, const rt_step_inputs* in, rt_state* inout, rt_step_stats* stats);

/* Residual f(U) = (f_e, f_n, f_E) of Eqs. gas_residual, chemistry_residual,
 * radiation_residual at the iterate U for the step that starts from U_n (E*, n_HI*).
 * Outputs are caller device arrays.  Errors: RT_EINVAL, RT_ECUDA. */
int rt_residual(rt_grid* g, const rt_step_inputs* in, const rt_state* U_n, const rt_state* U,
                double* f_e, double* f_n, double* f_E);

/* Schur complement of the Newton system at U (Sec. "Algorithm": the reduction to a modified
 * radiation equation; u = the cell-local unknowns, (e_c, n_HI) or on helium grids (e_c, n_HI,
 * n_HeI, n_HeII), which U and U_n must then carry):
 * S = J_EE - J_Eu J_uu^-1 J_uE as diag (per cell) and the three +x/+y/+z
 * face couplings w (S_ij = -w on the face between i and its + neighbour; S is symmetric), and
 * rhs = -f_E + J_Eu J_uu^-1 f_u.  The operator is also kept as the one rt_schur_solve uses.
 * Errors: RT_EINVAL, RT_ECUDA. */
int rt_schur_system(rt_grid* g, const rt_step_inputs* in, const rt_state* U_n, const rt_state* U,
                    double* diag, double* wx, double* wy, double* wz, double* rhs);

/* Solve S x = b for the operator of the last rt_schur_system call with multigrid-
 * preconditioned conjugate gradients (multigrid in the grid's precision) until the
 * residual's 2-norm falls below rtol times ||b||_2.  x: initial guess in, solution out.
 * *iters receives the CG iterations.  Errors: RT_EINVAL, RT_ELINEAR, RT_ENONFINITE, RT_ECUDA. */
int rt_schur_solve(rt_grid* g, const double* b, double* x, double rtol, int max_iters, int* iters);

/* Operator-split hand-over between steps without hydrodynamics: e_h += e_c (device arrays of
 * nx*ny*nz values).  Errors: RT_EINVAL, RT_ECUDA. */
int rt_fold_energy(rt_grid* g, double* e_h, const double* e_c);

/* Per-kernel timing.  While enabled, every kernel the library launches is bracketed by CUDA
 * events on the grid's stream and its algorithmic bytes (the arrays it must read and write,
 * counted once per launch) are recorded; rt_get_profile returns the totals per kernel class
 * accumulated since the last enable.  Timing adds two events per launch.  Errors: RT_EINVAL. */
typedef struct {
    char name[32];        /* kernel class                                                    */
    int launches;         /* launches recorded                                               */
    double ms;            /* summed event time of those launches                             */
    double bytes;         /* summed algorithmic bytes of those launches                      */
} rt_kernel_profile;
int rt_set_profiling(rt_grid* g, int on);
int rt_get_profile(rt_grid* g, rt_kernel_profile* out, int max_entries, int* n_entries);

/* Helium grids: rt_residual with the two helium species' residuals f_HeI, f_HeII as well
 * (all outputs optional, NULL skips).  U_n and U must carry n_HeI and n_HeII.  Errors as
 * rt_residual, and RT_EINVAL on a hydrogen-only grid. */
int rt_residual_helium(rt_grid* g, const rt_step_inputs* in, const rt_state* U_n, const rt_state* U,
                       double* f_e, double* f_n, double* f_HeI, double* f_HeII, double* f_E);

/* Diagnostic: evaluates the library's table-driven FP64 exp (fn 0) or log (fn 1) used by the
 * rate fits, or the CUDA math library's exp (fn 2) / log (fn 3), on n device values x into y,
 * on the given stream (NULL = legacy default stream).  Errors: RT_EINVAL, RT_ECUDA. */
int rt_eval_elementary(int fn, const double* x, double* y, long long n, void* stream);

/* Allocation-free residual.  The paper has no counterpart: this is a service for callers
 * that cannot allocate device memory -- an application that owns the whole device memory
 * budget through its own pool allocator (a library's own cudaMalloc there fails or fragments
 * that budget), or a real-time loop that must not take the device-wide synchronisation
 * cudaMalloc and cudaFree may cause.  It computes the same f(U) as rt_residual but takes the
 * descriptor instead of a grid handle and calls no cudaMalloc, cudaFree or allocating library
 * routine: its scratch is one file-scope device array of RT_RESIDUAL_STATIC_MAX_CELLS cells'
 * worth (about 2.2 MB), which every GPU that loads the library holds until the process exits.
 * Grids with more cells are rejected with RT_EINVAL, as are device ordinals outside 0..63.
 * The first call on a device looks up the array's device address on that device (and caches
 * it); make that first call before any stream capture, and make no call after a
 * cudaDeviceReset of that device.  Every call uses the same array and it keeps the last
 * call's contents: calls whose GPU work overlaps (other streams, other host threads on the
 * same device) race on it and must be serialised by the caller.
 * Arguments as rt_residual; desc->device and desc->stream select where the work runs; the
 * calling thread's current device is restored before the call returns.  The call returns
 * after synchronising desc->stream.  Hydrogen-only grids.
 * Errors: RT_EINVAL, RT_ECUDA. */
#define RT_RESIDUAL_STATIC_MAX_CELLS 32768
int rt_residual_static(const rt_grid_desc* desc, const rt_step_inputs* in, const rt_state* U_n,
                       const rt_state* U, double* f_e, double* f_n, double* f_E);

/* Discrete adjoint of one step (the step map of Sec. "Algorithm": U^{n+1} is the root of
 * f(U; X^n, p) = 0 with X^n = (E^n, n_HI^n, e_h^n) the state handed over by the operator split
 * and X^{n+1} = (E, n_HI, e_h^n + e_c)).  Given lam_np1 = dJ/dX^{n+1} for an objective J, it
 * solves the transposed Newton system at the converged state with the same Schur reduction and
 * multigrid-preconditioned CG as the forward step, and returns lam_n = dJ/dX^n through this
 * step.  The e_c slot of lam_np1 / lam_n holds the adjoint of the gas energy e_h.
 * U_n: the step's start state (E^n, n_HI^n; e_c unused); U_np1: its converged result
 * (rt_implicit_step output); in: the same inputs as that step (e_h = e_h^n).
 * g_ndot (nsrc values, may be NULL) and g_clump (nx*ny*nz FP32 values, may be NULL) are
 * ACCUMULATED: += dJ/dNdot_s [1/(photons/s)] and += dJ/dC of this step.  lam_n may alias
 * lam_np1.  All arrays are device arrays in the normalised units of the state.
 * Errors: RT_EINVAL, RT_ELINEAR, RT_ENONFINITE, RT_ECUDA. */
int rt_adjoint_step(rt_grid* g, const rt_step_inputs* in, const rt_state* U_n, const rt_state* U_np1,
                    const rt_state* lam_np1, rt_state* lam_n, double* g_ndot, float* g_clump);

/* Advection pre-step: step (iv) of the operator split (Sec. "Operator-Split Hydrodynamics with
 * Radiative Feedback") carries the densities with the baryon velocity,
 * d_t q + (1/a) div(q v_b) = 0 for q = n_HI, E (Eqs. enzo-chemical_ionization,
 * enzo-cons_radiation) and rho_b (Eq. enzo-cons_mass in conservative form), giving the advected
 * state step (v) starts from.  Scheme: first-order donor cell over in->dt at expansion factor
 * in->a.  On the face between a cell and its '+' neighbour,
 * c = (v_cell + v_neighbour)/2 * dt / (a dx) (zero on a wall face); the flux c * q of the cell
 * the flow leaves moves from one cell to the other.  Moving rho_b with the same fluxes keeps
 * n_HI <= n_H.  The gas energy e_h belongs to the hydrodynamics (pressure work,
 * Eq. enzo-cons_energy) and is not touched.
 * src: E, n_HI read (e_c unused; on helium grids n_HeI, n_HeII too).  dst: E, n_HI (and the
 * helium species) written.  rho_src / rho_dst: baryon density in and out (both NULL to leave
 * it alone).  No written array may overlap another argument array.
 * in->vx, vy, vz: device velocity components in the units of the state (NULL = 0); only
 * in->a, in->dt and the velocities are read from in.
 * courant_max (host pointer, may be NULL) receives the largest per-cell sum of outflow Courant
 * numbers.  If it exceeds 1 (the donor-cell bound for positivity and stability), nothing is
 * written and RT_EINVAL is returned.
 * Errors: RT_EINVAL, RT_ECUDA.  Synchronises the grid's stream. */
int rt_advect(rt_grid* g, const rt_step_inputs* in, const rt_state* src, rt_state* dst, const double* rho_src,
              double* rho_dst, double* courant_max);

/* Transpose of rt_advect's linear map (same inputs), for the adjoint of the operator split:
 * lam_star holds dJ/d(E*, n_HI*) of the advected state, lam receives dJ/d(E, n_HI) before
 * advection (e_c slots unused).  rho_b is not a differentiated variable (it does not depend on
 * the source rates or the clumping factor).  Hydrogen-only grids (RT_EINVAL with helium).
 * Same argument rules and errors as rt_advect. */
int rt_advect_adjoint(rt_grid* g, const rt_step_inputs* in, const rt_state* lam_star, rt_state* lam);

/* Free the grid's whole workspace; g is invalid afterwards.  NULL is a no-op. */
void rt_destroy_grid(rt_grid* g);
/* Static message for an error code ("unknown error" for codes outside the list). */
const char* rt_error_string(int code);
/* Detail text of the last error this library recorded on the calling host thread (a
 * per-thread buffer, overwritten by that thread's next error; empty if none). */
const char* rt_last_error_detail(void);

/* Grey constants the library derived at init, in CGS: sigma_E [cm^2], sigma_G [cm^2/erg],
 * eps_src [erg] (Eq. grey_definition with sigma ~ nu^-3).  Errors: RT_EINVAL. */
int rt_grey_constants(const rt_grid* g, double* sigma_E, double* sigma_G, double* eps_src);

/* The same grey constants without a grid (host computation only, no CUDA call): for the
 * spectrum (RT_SPECTRUM_MONO or RT_SPECTRUM_BLACKBODY at T_B kelvin, 0 < T_B < 1e9) it writes
 * seven values to the host array out, in CGS:
 *   [0] sigma_E [cm^2], [1] sigma_G [cm^2/erg], [2] eps_src [erg]  (hydrogen, as above);
 *   [3] sigma_E,HeI, [4] sigma_G,HeI, [5] sigma_E,HeII, [6] sigma_G,HeII  (the helium grey
 *   cross sections over the same spectrum, normalised by its energy above the hydrogen edge;
 *   zero for the 13.6 eV line).
 * Errors: RT_EINVAL. */
int rt_spectrum_constants(int spectrum, double T_B, double* out);

#ifdef __cplusplus
}
#endif
#endif
