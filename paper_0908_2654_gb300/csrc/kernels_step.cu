// Per-step and per-Newton-iteration kernels of the implicit step (FP64).
//
//  k_faces       once per step: flux-limited face couplings w = dt theta D / (a dx)^2 on the
//                +x/+y/+z face of every cell, D from Eq. limiter at the step's starting state
//                (0 on boundary faces; an outflow face's coupling to its empty ghost is
//                recomputed where it is used, outflow_coupling).
//  k_setup       once per step: explicit part b_E of Eq. radiation_residual and the initial
//                iterate (E* + dt 4 pi eta, n_HI*, 0).
//  k_assemble    once per Newton trial, fused: trial E = E_k + lam s, exact solution of the
//                cell-local equations for (e_c, n_HI) at that E (with forward-mode
//                derivatives), radiation residual f_E (7-point), Schur diagonal and right side
//                of the reduced Newton system (Sec. "Algorithm"), and the block partial sums of
//                the component-scaled RMS norm (Eq. rmsnorm).
#include "cellgrid.cuh"
#include "kernels.cuh"
#include "hlocal.cuh"

namespace {

using namespace cellgrid;

__global__ void k_zero(double* p, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = 0.0;
}

__global__ void k_scatter(double* src, const int64_t* cell, const double* ndot, int nsrc, double scale,
                          long long ncell, int* err) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nsrc) return;
    long long c = cell[k];
    if (c < 0 || c >= ncell) {      // checked: an out-of-range source index is reported, not written
        atomicOr(err, 1);
        return;
    }
    atomicAdd(&src[c], scale * ndot[k]);
}

__global__ void k_faces(PhysParams P, const double* __restrict__ E0, const double* __restrict__ n0,
                        double* __restrict__ wx, double* __restrict__ wy, double* __restrict__ wz,
                        float* __restrict__ wxf, float* __restrict__ wyf, float* __restrict__ wzf) {
    const long long n = (long long)P.nx * P.ny * P.nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        cell_coords(i, P.nx, P.ny, x, y, z);
        const double Ei = E0[i];
        const double ki = kappa_start(P, n0, i);
        const long long sy = P.nx, sz = (long long)P.nx * P.ny;
        const long long base = i - x - (long long)y * sy - (long long)z * sz;
        long long j[3] = {base + up(x, P.nx, P.per[0]) + y * sy + z * sz,
                          base + x + up(y, P.ny, P.per[1]) * sy + z * sz,
                          base + x + y * sy + up(z, P.nz, P.per[2]) * sz};
        const bool wall[3] = {!P.per[0] && x == P.nx - 1, !P.per[1] && y == P.ny - 1, !P.per[2] && z == P.nz - 1};
        double w[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (wall[d]) {
                w[d] = 0.0;
            } else {
                const double D = limiter_face(P, Ei, E0[j[d]], ki, kappa_start(P, n0, j[d]));
                w[d] = P.wscale * D;
            }
        }
        wx[i] = w[0];
        wy[i] = w[1];
        wz[i] = w[2];
        if (wxf) {
            wxf[i] = (float)w[0];
            wyf[i] = (float)w[1];
            wzf[i] = (float)w[2];
        }
    }
}

__global__ void k_setup(PhysParams P, const double* __restrict__ E0, const double* __restrict__ n0,
                        const double* __restrict__ src, const double* __restrict__ wx, const double* __restrict__ wy,
                        const double* __restrict__ wz, double* __restrict__ bE, double* __restrict__ E_init,
                        double* __restrict__ n_init, double* __restrict__ ec_init, double* partials, HydroIn H,
                        int* err) {
    const long long n = (long long)P.nx * P.ny * P.nz;
    const double expl = (1.0 - P.theta) / P.theta;   // (1-theta) dt D/(a dx)^2 = expl * w
    double emax = 0.0;
    bool bad = false;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        // the hydro state handed over by the operator split: positive finite density, finite
        // energy and (non-isothermal gas) a positive internal energy
        const double rho = H.rho[i], eh = H.e_h[i];
        double v2 = 0.0;
        if (H.vx) v2 += H.vx[i] * H.vx[i];
        if (H.vy) v2 += H.vy[i] * H.vy[i];
        if (H.vz) v2 += H.vz[i] * H.vz[i];
        if (!(rho > 0.0) || !isfinite(rho) || !isfinite(eh) || !isfinite(v2) || (!P.isothermal && !(eh - 0.5 * v2 > 0.0)))
            bad = true;
        int x, y, z;
        cell_coords(i, P.nx, P.ny, x, y, z);
        const Stencil s = stencil(i, x, y, z, P.nx, P.ny, P.nz, P.per, wx, wy, wz);
        const double E = E0[i];
        const double lap = s.wxp * (E0[s.xp] - E) + s.wxm * (E0[s.xm] - E) + s.wyp * (E0[s.yp] - E) +
                           s.wym * (E0[s.ym] - E) + s.wzp * (E0[s.zp] - E) + s.wzm * (E0[s.zm] - E) -
                           outflow_coupling(P, E0, n0, i, x, y, z) * E;
        const double kap = kappa_start(P, n0, i);
        bE[i] = E + expl * lap + P.dt * (1.0 - P.theta) * (-P.H * E + src[i] - P.c * kap * E);
        const double Ei = E + P.dt * src[i];
        E_init[i] = Ei;
        n_init[i] = n0[i];
        ec_init[i] = 0.0;
        emax = fmax(emax, fabs(Ei));
    }
    if (bad) atomicOr(err, 2);
    __shared__ double sh[kBlock / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) emax = fmax(emax, __shfl_down_sync(0xffffffffu, emax, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = emax;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) m = fmax(m, sh[w]);
        partials[blockIdx.x] = m;
    }
}

// Local equations f_e = e_c - S_e, f_n = n - S_n at fixed E: solution, residual and the
// pieces of the Schur reduction, X = (J_uu^-1 J_uE)_n and Y = (J_uu^-1 f_u)_n.
struct LocalOut {
    double ec, n, fe, fn, X, Y, Xe;
};

template <bool ISO, bool GIVEN>
__device__ __forceinline__ LocalOut local_block(const PhysParams& P, const HCell& c, double E, double ec_in,
                                                double n_in, double inv_se, double inv_rho) {
    LocalOut o;
    if (ISO) {
        const HLocal L = h_local<true>(P, c, 0.0, n_in, E);
        o.ec = GIVEN ? ec_in : 0.0;
        o.n = GIVEN ? n_in : L.Sn;
        o.fe = o.ec;
        o.fn = o.n - L.Sn;
        o.X = -L.Sn_E;
        o.Y = o.fn;
        o.Xe = 0.0;
        return o;
    }
    // damped 2x2 Newton: steps are halved until max(|f_e|/e_int, |f_n|/n_H) decreases,
    // keeping 0 < n_HI <= n_H and the internal energy positive
    double ec = ec_in, n = n_in;
    if (!GIVEN) n = fmin(fmax(n, 1e-300), c.rho);
    HLocal L = h_local<false>(P, c, ec, n, E);
    double fe = ec - L.Se, fn = n - L.Sn;
    double r = fmax(fabs(fe) * inv_se, fabs(fn) * inv_rho);
    const int maxit = GIVEN ? 0 : 60;
    for (int it = 0; it < maxit && r > P.local_tol; ++it) {
        const double a11 = 1.0 - L.Se_e, a12 = -L.Se_n, a21 = -L.Sn_e, a22 = 1.0 - L.Sn_n;
        const double idet = 1.0 / (a11 * a22 - a12 * a21);
        const double de = -(a22 * fe - a12 * fn) * idet;
        const double dn_ = -(a11 * fn - a21 * fe) * idet;
        double lam = 1.0;
        bool moved = false;
        for (int k = 0; k < 40; ++k, lam *= 0.5) {
            const double ec_t = fmax(ec + lam * de, -0.999 * c.eh_kin);
            const double n_t = fmin(fmax(n + lam * dn_, 1e-300), c.rho);
            const HLocal Lt = h_local<false>(P, c, ec_t, n_t, E);
            const double fe_t = ec_t - Lt.Se, fn_t = n_t - Lt.Sn;
            const double r_t = fmax(fabs(fe_t) * inv_se, fabs(fn_t) * inv_rho);
            if (r_t < r) {
                ec = ec_t;
                n = n_t;
                L = Lt;
                fe = fe_t;
                fn = fn_t;
                r = r_t;
                moved = true;
                break;
            }
        }
        if (!moved) break;   // round-off floor
    }
    const double a11 = 1.0 - L.Se_e, a21 = -L.Sn_e;
    const double a12 = -L.Se_n, a22 = 1.0 - L.Sn_n;
    const double idet = 1.0 / (a11 * a22 - a12 * a21);
    const double be = -L.Se_E, bn = -L.Sn_E;
    o.ec = ec;
    o.n = n;
    o.fe = fe;
    o.fn = fn;
    o.X = (a11 * bn - a21 * be) * idet;
    o.Y = (a11 * fn - a21 * fe) * idet;
    o.Xe = (a22 * be - a12 * bn) * idet;
    return o;
}

// two CTAs per SM (128 registers a thread): twice the warps the FP64 pipe can switch between
template <bool ISO, bool GIVEN>
__global__ void __launch_bounds__(kBlock, 2) k_assemble(PhysParams P, AssembleArgs A) {
    const long long n = (long long)P.nx * P.ny * P.nz;
    const double inv_a3 = 1.0 / P.a3;
    const double kEa = P.kE * inv_a3;     // proper opacity per unit n_HI
    double acc[3] = {0.0, 0.0, 0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        cell_coords(i, P.nx, P.ny, x, y, z);
        const Stencil s = stencil(i, x, y, z, P.nx, P.ny, P.nz, P.per, A.wx, A.wy, A.wz);
        const double lam = A.lam;
        const double* Ec = A.E_cur;
        const double* st = A.step;
        auto Et = [&](long long j) { return st ? fma(lam, st[j], Ec[j]) : Ec[j]; };
        const double E = Et(i);
        const double wb = outflow_coupling(P, A.E0, A.n0, i, x, y, z);   // outflow faces (ghost E = 0)
        const double lap = s.wxp * (Et(s.xp) - E) + s.wxm * (Et(s.xm) - E) + s.wyp * (Et(s.yp) - E) +
                           s.wym * (Et(s.ym) - E) + s.wzp * (Et(s.zp) - E) + s.wzm * (Et(s.zm) - E) - wb * E;
        const double sumw = s.wxp + s.wxm + s.wyp + s.wym + s.wzp + s.wzm + wb;

        double v2 = 0.0;
        if (A.vx) v2 += A.vx[i] * A.vx[i];
        if (A.vy) v2 += A.vy[i] * A.vy[i];
        if (A.vz) v2 += A.vz[i] * A.vz[i];
        const HCell c = make_hcell(P, inv_a3, A.rho[i], A.n0[i], A.E0[i], A.e_h[i] - 0.5 * v2,
                                   A.clump ? (double)A.clump[i] : 1.0);
        const double inv_se = 1.0 / fmax(c.eh_kin, P.e_floor), inv_rho = c.inv_rho;

        double ec_in = GIVEN ? A.ec_given[i] : (A.ec_guess ? A.ec_guess[i] : 0.0);
        double n_in = GIVEN ? A.n_given[i] : A.n_guess[i];
        if (!GIVEN && !ISO && A.Xe_cur && st) {
            // tangent predictor: u(E + dE) ~ u(E) - X dE, from the elimination at the current iterate
            const double dE = lam * st[i];
            ec_in = fmax(ec_in - A.Xe_cur[i] * dE, -0.999 * c.eh_kin);
            n_in = fmin(fmax(n_in - A.Xn_cur[i] * dE, 1e-300), c.rho);
        }
        const LocalOut L = local_block<ISO, GIVEN>(P, c, E, ec_in, n_in, inv_se, inv_rho);

        const double kap = kEa * L.n;
        const double dtt = P.dt * P.theta;
        const double fE = E - A.bE[i] - lap - dtt * (-P.H * E + A.src[i] - P.c * kap * E);
        const double AEn = dtt * P.c * kEa * E;
        const double AEE = 1.0 + dtt * (P.H + P.c * kap) + sumw;
        const double dg = AEE - AEn * L.X;
        const double rh = -fE + AEn * L.Y;

        // the norm weights of E at the current iterate and at the trial from one reciprocal
        const double mEc = fmax(fmax(fabs(Ec[i]), c.E0), P.E_floor);
        const double mEt = fmax(fmax(fabs(E), c.E0), P.E_floor);
        const double wcw = 1.0 / (mEc * mEt);
        const double wEc = mEt * wcw, wEt = mEc * wcw;
        const double loc = (L.fn * inv_rho) * (L.fn * inv_rho) + (L.fe * inv_se) * (L.fe * inv_se);
        acc[0] += (wEc * fE) * (wEc * fE) + loc;
        acc[1] += (wEt * fE) * (wEt * fE) + loc;
        if (!isfinite(fE) || !isfinite(dg) || !isfinite(L.n) || !isfinite(L.ec)) acc[2] += 1.0;

        if (A.E_out) A.E_out[i] = E;
        if (A.n_out) A.n_out[i] = L.n;
        if (A.ec_out) A.ec_out[i] = L.ec;
        if (A.diag) A.diag[i] = dg;
        if (A.rhs) A.rhs[i] = rh;
        if (A.wE) A.wE[i] = wEt;
        if (A.fE_out) A.fE_out[i] = fE;
        if (A.fn_out) A.fn_out[i] = L.fn;
        if (A.fe_out) A.fe_out[i] = L.fe;
        if (A.Xe_out) {
            A.Xe_out[i] = L.Xe;
            A.Xn_out[i] = L.X;
        }
    }
    block_sums<3>(acc, A.partials);
}

// Sum over cells of the squared component-scaled change of (e_c, n_HI, E) over the step
// (e_c^n = 0; E scaled by max(|E^{n+1}|, |E^n|, E_floor), n_HI by n_H, e_c by the hydro
// state's internal energy): the time-step controller's measure of the solution change.
__global__ void __launch_bounds__(kBlock) k_change_norm(PhysParams P, AssembleArgs A) {
    const long long n = (long long)P.nx * P.ny * P.nz;
    double acc[1] = {0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double E1 = A.E_cur[i], E0 = A.E0[i];
        const double dE = (E1 - E0) / fmax(fmax(fabs(E1), fabs(E0)), P.E_floor);
        const double dn = (A.n_guess[i] - A.n0[i]) / A.rho[i];
        double de = 0.0;
        if (!P.isothermal) {
            double v2 = 0.0;
            if (A.vx) v2 += A.vx[i] * A.vx[i];
            if (A.vy) v2 += A.vy[i] * A.vy[i];
            if (A.vz) v2 += A.vz[i] * A.vz[i];
            de = A.ec_guess[i] / fmax(A.e_h[i] - 0.5 * v2, P.e_floor);
        }
        acc[0] += dE * dE + dn * dn + de * de;
    }
    block_sums<1>(acc, A.partials);
}

__global__ void k_finalize(const double* __restrict__ partials, int nblocks, int nslots, double* out) {
    __shared__ double sh[256];
    for (int k = 0; k < nslots; ++k) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partials[(size_t)k * nblocks + b];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[k] = sh[0];
        __syncthreads();
    }
}

__global__ void k_finalize_ext(const double* __restrict__ partials, int nblocks, int nsum, int nmax, double* out) {
    __shared__ double sh[256];
    for (int k = 0; k < nsum + nmax; ++k) {
        const bool is_max = k >= nsum;
        double s = is_max ? 0.0 : 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
            const double v = partials[(size_t)k * nblocks + b];
            s = is_max ? fmax(s, v) : s + v;
        }
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) sh[threadIdx.x] = is_max ? fmax(sh[threadIdx.x], sh[threadIdx.x + w])
                                                          : sh[threadIdx.x] + sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[k] = sh[0];
        __syncthreads();
    }
}

__global__ void k_elementary(int fn, const double* __restrict__ x, double* __restrict__ y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = x[i];
        y[i] = fn == 0 ? rt_exp(v) : fn == 1 ? rt_log(v) : fn == 2 ? exp(v) : log(v);
    }
}

int grid_for(long long n) {
    long long b = (n + kBlock - 1) / kBlock;
    const long long cap = 152LL * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

void launch_zero(double* p, long long n, cudaStream_t s) { k_zero<<<grid_for(n), kBlock, 0, s>>>(p, n); }

void launch_scatter_sources(double* src, const int64_t* cell, const double* ndot, int nsrc, double scale,
                            long long ncell, int* d_err, cudaStream_t s) {
    if (nsrc <= 0) return;
    k_scatter<<<(nsrc + 255) / 256, 256, 0, s>>>(src, cell, ndot, nsrc, scale, ncell, d_err);
}

void launch_faces(const PhysParams& P, const double* E0, const double* n0, double* wx, double* wy, double* wz,
                  float* wxf, float* wyf, float* wzf, cudaStream_t s) {
    const long long n = (long long)P.nx * P.ny * P.nz;
    k_faces<<<grid_for(n), kBlock, 0, s>>>(P, E0, n0, wx, wy, wz, wxf, wyf, wzf);
}

int launch_setup(const PhysParams& P, const double* E0, const double* n0, const double* src, const double* wx,
                 const double* wy, const double* wz, double* bE, double* E_init, double* n_init, double* ec_init,
                 double* partials, const HydroIn& H, int* err, cudaStream_t s) {
    const long long n = (long long)P.nx * P.ny * P.nz;
    const int g = grid_for(n);
    k_setup<<<g, kBlock, 0, s>>>(P, E0, n0, src, wx, wy, wz, bE, E_init, n_init, ec_init, partials, H, err);
    return g;
}

int launch_assemble(const PhysParams& P, const AssembleArgs& A, bool given_u, cudaStream_t s) {
    const long long n = (long long)P.nx * P.ny * P.nz;
    const int g = grid_for(n);
    if (P.isothermal) {
        if (given_u) k_assemble<true, true><<<g, kBlock, 0, s>>>(P, A);
        else k_assemble<true, false><<<g, kBlock, 0, s>>>(P, A);
    } else {
        if (given_u) k_assemble<false, true><<<g, kBlock, 0, s>>>(P, A);
        else k_assemble<false, false><<<g, kBlock, 0, s>>>(P, A);
    }
    return g;
}

int launch_change_norm(const PhysParams& P, const AssembleArgs& A, cudaStream_t s) {
    const long long n = (long long)P.nx * P.ny * P.nz;
    const int g = grid_for(n);
    k_change_norm<<<g, kBlock, 0, s>>>(P, A);
    return g;
}

void launch_elementary(int fn, const double* x, double* y, long long n, cudaStream_t s) {
    k_elementary<<<grid_for(n), kBlock, 0, s>>>(fn, x, y, n);
}

void launch_finalize(const double* partials, int nblocks, int nslots, double* out, cudaStream_t s) {
    k_finalize<<<1, 256, 0, s>>>(partials, nblocks, nslots, out);
}

void launch_finalize_ext(const double* partials, int nblocks, int nsum, int nmax, double* out, cudaStream_t s) {
    k_finalize_ext<<<1, 256, 0, s>>>(partials, nblocks, nsum, nmax, out);
}
