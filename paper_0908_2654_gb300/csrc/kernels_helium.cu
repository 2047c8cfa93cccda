// Fused Newton evaluation of the implicit step for hydrogen + helium gas (FP64).
//
// Like k_assemble for hydrogen alone, with the cell-local unknowns u = (e_c, n_HI, n_HeI,
// n_HeII): trial E = E_k + lam s, the local equations f_u = u - S(u, E) solved at that E by a
// damped 4x4 Newton iteration (isothermal: e_c = 0, a 3x3 one), the radiation residual f_E with
// the opacity kappa = (kE n_HI + kE1 n_HeI + kE2 n_HeII) / a^3, and the reduced (Schur)
// system's diagonal and right side: with A_Eu = dt theta c E / a^3 (0, kE, kE1, kE2),
// X = A_uu^-1 A_uE and Y = A_uu^-1 f_u, diag = A_EE - A_Eu.X and rhs = -f_E + A_Eu.Y.  The
// norm sums run over the N (N_s + 2) = 5 N unknowns (helium species scaled by n_He).
#include "cellgrid.cuh"
#include "helium.cuh"
#include "kernels.cuh"

namespace {

using namespace cellgrid;
using D5 = Dual<5>;   // lanes: e_c, n_HI, n_HeI, n_HeII, E

// Solves a x = b for two right sides by Gaussian elimination with partial pivoting (row swaps by
// selects keep every index static, so the arrays stay in registers).
__device__ __forceinline__ void solve4(double (&a)[4][4], double (&b)[4][2]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
        for (int i = k + 1; i < 4; ++i) {
            const bool sw = fabs(a[i][k]) > fabs(a[k][k]);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const double t = a[k][j];
                a[k][j] = sw ? a[i][j] : t;
                a[i][j] = sw ? t : a[i][j];
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const double t = b[k][j];
                b[k][j] = sw ? b[i][j] : t;
                b[i][j] = sw ? t : b[i][j];
            }
        }
        const double inv = 1.0 / a[k][k];
#pragma unroll
        for (int i = k + 1; i < 4; ++i) {
            const double m = a[i][k] * inv;
#pragma unroll
            for (int j = k; j < 4; ++j) a[i][j] -= m * a[k][j];
#pragma unroll
            for (int j = 0; j < 2; ++j) b[i][j] -= m * b[k][j];
        }
    }
#pragma unroll
    for (int k = 3; k >= 0; --k) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            double s = b[k][j];
#pragma unroll
            for (int i = k + 1; i < 4; ++i) s -= a[k][i] * b[i][j];
            b[k][j] = s / a[k][k];
        }
    }
}

struct LocalHe {
    double u[4], f[4], X[4], Y[4];
};

template <bool ISO>
__device__ __forceinline__ void eval_he(const PhysParams& P, const CellHe& c, const double (&u)[4], double E,
                                        double (&f)[4], double (&J)[4][4], double (&JE)[4]) {
    D5 S[4];
    local_solutions_he<D5>(P, c, dvar<5>(u[0], 0), dvar<5>(u[1], 1), dvar<5>(u[2], 2), dvar<5>(u[3], 3),
                           dvar<5>(E, 4), S[0], S[1], S[2], S[3]);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        f[i] = u[i] - S[i].v;
#pragma unroll
        for (int j = 0; j < 4; ++j) J[i][j] = (i == j ? 1.0 : 0.0) - S[i].d[j];
        JE[i] = -S[i].d[4];
    }
    if (ISO) {   // f_e = e_c = 0 and e_c does not enter the other equations
        f[0] = 0.0;
        JE[0] = 0.0;
#pragma unroll
        for (int j = 0; j < 4; ++j) J[0][j] = j == 0 ? 1.0 : 0.0;
    }
}

// the local residuals alone (line-search trials)
template <bool ISO>
__device__ __forceinline__ void eval_f_he(const PhysParams& P, const CellHe& c, const double (&u)[4], double E,
                                          double (&f)[4]) {
    double S[4];
    local_solutions_he<double>(P, c, u[0], u[1], u[2], u[3], E, S[0], S[1], S[2], S[3]);
#pragma unroll
    for (int i = 0; i < 4; ++i) f[i] = u[i] - S[i];
    if (ISO) f[0] = 0.0;
}

__device__ __forceinline__ double scaled_max(const double (&f)[4], const double (&inv)[4]) {
    return fmax(fmax(fabs(f[0]) * inv[0], fabs(f[1]) * inv[1]), fmax(fabs(f[2]) * inv[2], fabs(f[3]) * inv[3]));
}

__device__ __forceinline__ void clamp_he(const CellHe& c, double (&u)[4]) {
    u[0] = fmax(u[0], -0.999 * c.eh_kin);
    u[1] = fmin(fmax(u[1], 1e-300), c.nH);
    u[2] = fmin(fmax(u[2], 0.0), c.nHe);
    u[3] = fmin(fmax(u[3], 0.0), c.nHe - u[2]);
}

// damped Newton on the local equations at fixed E (GIVEN: no iteration, evaluate at u_in)
template <bool ISO, bool GIVEN>
__device__ __forceinline__ LocalHe local_block_he(const PhysParams& P, const CellHe& c, double E,
                                                  const double (&u_in)[4], const double (&inv)[4]) {
    LocalHe o;
    double u[4] = {u_in[0], u_in[1], u_in[2], u_in[3]};
    if (ISO) u[0] = 0.0;
    if (!GIVEN) clamp_he(c, u);
    double f[4], J[4][4], JE[4];
    eval_he<ISO>(P, c, u, E, f, J, JE);
    double r = scaled_max(f, inv);
    const int maxit = GIVEN ? 0 : 60;
    for (int it = 0; it < maxit && r > P.local_tol; ++it) {
        double a[4][4], b[4][2];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int j = 0; j < 4; ++j) a[i][j] = J[i][j];
            b[i][0] = -f[i];
            b[i][1] = 0.0;
        }
        solve4(a, b);
        // backtracking on the residuals alone; the Jacobian only at the accepted point
        double lam = 1.0;
        bool moved = false;
        for (int k = 0; k < 40; ++k, lam *= 0.5) {
            double ut[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) ut[i] = u[i] + lam * b[i][0];
            if (ISO) ut[0] = 0.0;
            clamp_he(c, ut);
            double ft[4];
            eval_f_he<ISO>(P, c, ut, E, ft);
            if (scaled_max(ft, inv) < r) {
#pragma unroll
                for (int i = 0; i < 4; ++i) u[i] = ut[i];
                moved = true;
                break;
            }
        }
        if (!moved) break;   // round-off floor
        eval_he<ISO>(P, c, u, E, f, J, JE);
        r = scaled_max(f, inv);
    }
    double a[4][4], b[4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) a[i][j] = J[i][j];
        b[i][0] = JE[i];
        b[i][1] = f[i];
    }
    solve4(a, b);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        o.u[i] = u[i];
        o.f[i] = f[i];
        o.X[i] = b[i][0];
        o.Y[i] = b[i][1];
    }
    return o;
}

template <bool ISO, bool GIVEN>
__global__ void __launch_bounds__(kBlock) k_assemble_he(PhysParams P, AssembleArgs A, HeliumArgs H) {
    const long long n = (long long)P.nx * P.ny * P.nz;
    const double nH_per_rho = 1.0 - P.Y, nHe_per_rho = 0.25 * P.Y;
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

        CellHe c;
        c.rho = A.rho[i];
        c.nH = nH_per_rho * c.rho;
        c.nHe = nHe_per_rho * c.rho;
        c.nHI0 = A.n0[i];
        c.nHeI0 = H.nHeI0[i];
        c.nHeII0 = H.nHeII0[i];
        c.E0 = A.E0[i];
        double v2 = 0.0;
        if (A.vx) v2 += A.vx[i] * A.vx[i];
        if (A.vy) v2 += A.vy[i] * A.vy[i];
        if (A.vz) v2 += A.vz[i] * A.vz[i];
        c.eh_kin = A.e_h[i] - 0.5 * v2;
        c.clump = A.clump ? (double)A.clump[i] : 1.0;
        const double se = fmax(c.eh_kin, P.e_floor);
        const double inv[4] = {1.0 / se, 1.0 / c.nH, c.nHe > 0.0 ? 1.0 / c.nHe : 0.0, c.nHe > 0.0 ? 1.0 / c.nHe : 0.0};

        double u_in[4];
        if (GIVEN) {
            u_in[0] = A.ec_given[i];
            u_in[1] = A.n_given[i];
            u_in[2] = H.HeI_given[i];
            u_in[3] = H.HeII_given[i];
        } else {
            u_in[0] = A.ec_guess ? A.ec_guess[i] : 0.0;
            u_in[1] = A.n_guess[i];
            u_in[2] = H.HeI_guess[i];
            u_in[3] = H.HeII_guess[i];
        }
        const LocalHe L = local_block_he<ISO, GIVEN>(P, c, E, u_in, inv);

        const double kap = (P.kE * L.u[1] + P.kE1 * L.u[2] + P.kE2 * L.u[3]) / P.a3;
        const double dtt = P.dt * P.theta;
        const double fE = E - A.bE[i] - lap - dtt * (-P.H * E + A.src[i] - P.c * kap * E);
        const double aE = dtt * P.c * E / P.a3;
        const double AEu[4] = {0.0, aE * P.kE, aE * P.kE1, aE * P.kE2};
        const double AEE = 1.0 + dtt * (P.H + P.c * kap) + sumw;
        double dg = AEE, rh = -fE;
#pragma unroll
        for (int k = 1; k < 4; ++k) {
            dg -= AEu[k] * L.X[k];
            rh += AEu[k] * L.Y[k];
        }

        const double wEc = 1.0 / fmax(fmax(fabs(Ec[i]), c.E0), P.E_floor);
        const double wEt = 1.0 / fmax(fmax(fabs(E), c.E0), P.E_floor);
        double loc = 0.0;
#pragma unroll
        for (int k = 0; k < 4; ++k) loc += (L.f[k] * inv[k]) * (L.f[k] * inv[k]);
        acc[0] += (wEc * fE) * (wEc * fE) + loc;
        acc[1] += (wEt * fE) * (wEt * fE) + loc;
        bool bad = !isfinite(fE) || !isfinite(dg);
#pragma unroll
        for (int k = 0; k < 4; ++k) bad = bad || !isfinite(L.u[k]);
        if (bad) acc[2] += 1.0;

        if (A.E_out) A.E_out[i] = E;
        if (A.n_out) A.n_out[i] = L.u[1];
        if (A.ec_out) A.ec_out[i] = L.u[0];
        if (H.HeI_out) H.HeI_out[i] = L.u[2];
        if (H.HeII_out) H.HeII_out[i] = L.u[3];
        if (A.diag) A.diag[i] = dg;
        if (A.rhs) A.rhs[i] = rh;
        if (A.wE) A.wE[i] = wEt;
        if (A.fE_out) A.fE_out[i] = fE;
        if (A.fe_out) A.fe_out[i] = L.f[0];
        if (A.fn_out) A.fn_out[i] = L.f[1];
        if (H.fHeI_out) H.fHeI_out[i] = L.f[2];
        if (H.fHeII_out) H.fHeII_out[i] = L.f[3];
    }
    block_sums<3>(acc, A.partials);
}

// solution change over a step (time-step control): the hydrogen terms plus the helium species
__global__ void __launch_bounds__(kBlock) k_change_norm_he(PhysParams P, AssembleArgs A, HeliumArgs H) {
    const long long n = (long long)P.nx * P.ny * P.nz;
    const double nH_per_rho = 1.0 - P.Y, nHe_per_rho = 0.25 * P.Y;
    double acc[1] = {0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double E1 = A.E_cur[i], E0 = A.E0[i];
        const double dE = (E1 - E0) / fmax(fmax(fabs(E1), fabs(E0)), P.E_floor);
        const double nH = nH_per_rho * A.rho[i], nHe = nHe_per_rho * A.rho[i];
        const double dn = (A.n_guess[i] - A.n0[i]) / nH;
        const double ih = nHe > 0.0 ? 1.0 / nHe : 0.0;
        const double d1 = (H.HeI_guess[i] - H.nHeI0[i]) * ih, d2 = (H.HeII_guess[i] - H.nHeII0[i]) * ih;
        double de = 0.0;
        if (!P.isothermal) {
            double v2 = 0.0;
            if (A.vx) v2 += A.vx[i] * A.vx[i];
            if (A.vy) v2 += A.vy[i] * A.vy[i];
            if (A.vz) v2 += A.vz[i] * A.vz[i];
            de = A.ec_guess[i] / fmax(A.e_h[i] - 0.5 * v2, P.e_floor);
        }
        acc[0] += dE * dE + dn * dn + d1 * d1 + d2 * d2 + de * de;
    }
    block_sums<1>(acc, A.partials);
}

int grid_for(long long n) {
    long long b = (n + kBlock - 1) / kBlock;
    const long long cap = 152LL * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

int launch_assemble_he(const PhysParams& P, const AssembleArgs& A, const HeliumArgs& H, bool given_u,
                       cudaStream_t s) {
    const int g = grid_for((long long)P.nx * P.ny * P.nz);
    if (P.isothermal) {
        if (given_u) k_assemble_he<true, true><<<g, kBlock, 0, s>>>(P, A, H);
        else k_assemble_he<true, false><<<g, kBlock, 0, s>>>(P, A, H);
    } else {
        if (given_u) k_assemble_he<false, true><<<g, kBlock, 0, s>>>(P, A, H);
        else k_assemble_he<false, false><<<g, kBlock, 0, s>>>(P, A, H);
    }
    return g;
}

int launch_change_norm_he(const PhysParams& P, const AssembleArgs& A, const HeliumArgs& H, cudaStream_t s) {
    const int g = grid_for((long long)P.nx * P.ny * P.nz);
    k_change_norm_he<<<g, kBlock, 0, s>>>(P, A, H);
    return g;
}
