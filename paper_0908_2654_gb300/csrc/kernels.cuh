// Kernel declarations and launch helpers shared by the host driver.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "physics.cuh"

// Maximum cells of the level that the single-CTA coarse solver takes over.
template <class T> struct TailMax;
template <> struct TailMax<float> { static const int value = 4096; };
template <> struct TailMax<double> { static const int value = 2048; };

#define RT_RED_SLOTS 4      // simultaneous sums per reduction
#define RT_MAX_PARTIALS 4096

struct Dims {
    int nx, ny, nz;
    int per[3];
    __host__ __device__ long long n() const { return (long long)nx * ny * nz; }
};

// ---- step setup
void launch_zero(double* p, long long n, cudaStream_t s);
// sets bit 1 of *d_err for a source index outside the grid (that source is skipped)
void launch_scatter_sources(double* src, const int64_t* cell, const double* ndot, int nsrc, double scale,
                            long long ncell, int* d_err, cudaStream_t s);
void launch_faces(const PhysParams& P, const double* E0, const double* n0, double* wx, double* wy, double* wz,
                  float* wxf, float* wyf, float* wzf, cudaStream_t s);
// the hydro state of the step (device pointers; velocities may be null)
struct HydroIn {
    const double* rho;
    const double* e_h;
    const double* vx;
    const double* vy;
    const double* vz;
};
// also writes per-block max |E_init| to partials (one slot) and sets bit 2 of *err where the
// hydro state is invalid (density not positive and finite, energy not finite, non-isothermal
// internal energy not positive); returns the number of blocks
int launch_setup(const PhysParams& P, const double* E0, const double* n0, const double* src, const double* wx,
                 const double* wy, const double* wz, double* bE, double* E_init, double* n_init, double* ec_init,
                 double* partials, const HydroIn& H, int* err, cudaStream_t s);

// ---- fused Newton evaluation
struct AssembleArgs {
    // trial iterate: E_t = E_cur + lam * step (step may be null); u from local solve
    const double* E_cur;
    const double* step;
    double lam;
    const double* n_guess;   // local-solve starting values (current iterate)
    const double* ec_guess;
    const double* Xe_cur;    // optional: d(e_c, n_HI)/dE = -(Xe, Xn) at the current iterate; the
    const double* Xn_cur;    // local solve then starts from the tangent predictor u - X lam s
    // given-iterate mode (parity entry points): u is taken from here, no local solve
    const double* n_given;
    const double* ec_given;
    // per-step data
    const double* E0;
    const double* n0;
    const double* rho;
    const double* e_h;
    const double* vx;
    const double* vy;
    const double* vz;
    const float* clump;
    const double* bE;
    const double* src;
    const double* wx;
    const double* wy;
    const double* wz;
    // outputs
    double* E_out;
    double* n_out;
    double* ec_out;
    double* diag;       // Schur diagonal
    double* rhs;        // Schur right side
    double* wE;         // norm weight of the trial (for the linear solver's residual norm)
    double* Xe_out;     // optional: X = J_uu^-1 J_uE at the trial (non-isothermal)
    double* Xn_out;
    double* fE_out;     // optional residual outputs (parity entry points)
    double* fn_out;
    double* fe_out;
    double* partials;   // RT_RED_SLOTS * nblocks block sums
};
int launch_assemble(const PhysParams& P, const AssembleArgs& A, bool given_u, cudaStream_t s);
// sum of squared scaled changes (E_cur, n_guess, ec_guess) against (E0, n0): one slot per block
int launch_change_norm(const PhysParams& P, const AssembleArgs& A, cudaStream_t s);

// ---- hydrogen + helium: the helium species next to AssembleArgs' hydrogen ones
struct HeliumArgs {
    const double* nHeI0;       // start of step
    const double* nHeII0;
    const double* HeI_guess;   // local-solve starting values (current iterate)
    const double* HeII_guess;
    const double* HeI_given;   // given-iterate mode
    const double* HeII_given;
    double* HeI_out;           // trial values
    double* HeII_out;
    double* fHeI_out;          // optional residual outputs
    double* fHeII_out;
};
int launch_assemble_he(const PhysParams& P, const AssembleArgs& A, const HeliumArgs& H, bool given_u,
                       cudaStream_t s);
// change norm with the helium species (HeI_guess / HeII_guess hold the new state)
int launch_change_norm_he(const PhysParams& P, const AssembleArgs& A, const HeliumArgs& H, cudaStream_t s);

// ---- advection pre-step (donor cell) and its transpose
struct AdvectArgs {
    int nx, ny, nz;
    int per[3];
    double k;              // dt / (a dx)
    const double* v[3];    // velocity components (null: zero)
    const double* qE;      // forward: E, n_HI; transpose: their adjoints after advection
    const double* qn;
    double* oE;
    double* on;
    const double* qr;      // optional third density moved by the forward map (rho_b), or null
    double* orh;
    const double* qh1;     // optional helium species moved by the forward map, or null
    const double* qh2;
    double* oh1;
    double* oh2;
    double* partials;      // Courant check: one block maximum per block
};
int launch_advect_courant(const AdvectArgs& A, cudaStream_t s);   // returns the number of blocks
void launch_advect(const AdvectArgs& A, bool transpose, cudaStream_t s);

// ---- elementary functions (fn 0: table exp, 1: table log, 2: CUDA exp, 3: CUDA log)
void launch_elementary(int fn, const double* x, double* y, long long n, cudaStream_t s);

// ---- discrete adjoint of one step
struct AdjointArgs {
    const double* rho;
    const double* e_h;
    const double* vx;
    const double* vy;
    const double* vz;
    const float* clump;
    const double* E0;        // start state
    const double* n0;
    const double* E;         // converged end state U = (e_c, n_HI, E)
    const double* nHI;
    const double* ec;
    const double* lam_E_in;  // adjoint of the hand-over state (E, n_HI, e_h)
    const double* lam_n_in;
    const double* lam_eh_in;
    double* rhs;             // reduced adjoint right side
    const double* muE;       // reduced adjoint solution
    double* lam_E_out;       // adjoint of the start state
    double* lam_n_out;
    double* lam_eh_out;
    float* g_clump;          // += dJ/dC
    double* g_ndot;          // += dJ/dNdot
    const int64_t* src_cell;
};
void launch_adj_rhs(const PhysParams& P, const AdjointArgs& A, cudaStream_t s);
void launch_adj_back(const PhysParams& P, const AdjointArgs& A, int nsrc, cudaStream_t s);

// ---- reductions (deterministic: block partials then one ordered pass)
void launch_finalize(const double* partials, int nblocks, int nslots, double* out, cudaStream_t s);
// slots [0, nsum) are summed, slots [nsum, nsum + nmax) are maxima
void launch_finalize_ext(const double* partials, int nblocks, int nsum, int nmax, double* out, cudaStream_t s);

// ---- CG vector kernels (FP64)
int launch_spmv_dot(const Dims& D, const double* diag, const double* wx, const double* wy, const double* wz,
                     const double* p, double* q, double* partials, cudaStream_t s);
int launch_residual_norm(const Dims& D, const double* diag, const double* wx, const double* wy, const double* wz,
                         const double* b, const double* x, double* r, const double* w, double* partials,
                         cudaStream_t s);
int launch_cg_update_xr(long long n, const double* scal, double* x, double* r, const double* p, const double* q,
                        const double* w, double* partials, cudaStream_t s);
int launch_dot2(long long n, const double* z, const double* r, const double* q, double* partials, cudaStream_t s);
void launch_p_update(long long n, const double* scal, const double* z, double* p, cudaStream_t s);
// multigrid operator diagonal: max(diag, sum of the 6 face couplings), i.e. sigma = max(sigma, 0)
template <class T>
void launch_mg_diag(const Dims& D, const double* diag, const double* wx, const double* wy, const double* wz, T* out,
                    cudaStream_t s);
void launch_copy(long long n, const double* a, double* b, cudaStream_t s);
void launch_add(long long n, const double* a, double* b, cudaStream_t s);   // b += a
// scalar bookkeeping on the device: scal[] holds alpha, beta and the dot products
void launch_cg_scalars(double* scal, const double* dots, int phase, cudaStream_t s);

// ---- multigrid (T = float or double)
// Every level but the last is smoothed and holds x and b colour-split (rbpass.cuh), with the
// smoother's copy of its operator in ds / w6; the last level, solved by the single-CTA solver,
// is in natural order.  diag / wx / wy / wz are the natural-order operator of every level.
template <class T>
struct Level {
    Dims d;
    T* diag;
    T* wx;
    T* wy;
    T* wz;
    T* dinv;   // colour-split inverse diagonal (split levels)
    T* w6;     // six face arrays of the colour-0 cells, n/2 each (split levels)
    T* x;      // current iterate
    T* b;
    int split; // x and b colour-split
};
template <class T>
void launch_coarsen(const Level<T>& f, const Level<T>& c, cudaStream_t s);
// dinv and w6 of a split level from its natural-order operator
template <class T>
void launch_split_level(const Level<T>& L, cudaStream_t s);
// one red-black Gauss-Seidel sweep of a split level's x in place as two colour passes
// (rbpass.cuh), the first from a zero iterate when zero_guess; returns the launches made
template <class T>
int launch_rbgs_inplace(const Level<T>& L, int first, bool zero_guess, cudaStream_t s);
// f.x += trilinear prolongation of c.x (f split)
template <class T>
void launch_prolong_add(const Level<T>& c, const Level<T>& f, cudaStream_t s);
// c.b = average over the 8 children of f.b - S f.x (f split)
template <class T>
void launch_resid_restrict(const Level<T>& f, const Level<T>& c, cudaStream_t s);
// level-0 vectors: out[level order] = a * 2^-k (k from *amax, or 0 when amax is null) and back
template <class Tin, class Tout>
void launch_to_level(const Dims& d, int split, const Tin* a, Tout* out, const double* amax, cudaStream_t s);
template <class Tin, class Tout>
void launch_from_level(const Dims& d, int split, const Tin* a, Tout* out, const double* amax, cudaStream_t s);
template <class T>
int launch_tail(const Level<T>& L, int ncycles, int nu, cudaStream_t s);
template <class T>
size_t tail_smem_bytes(const Dims& d);
