// Discrete adjoint of one implicit step (FP64).
//
// The step maps the carried state X = (E^n, n_HI^n, e_h^n) to the root U = (e_c, n_HI, E) of
// f(U; X, p) = 0 and hands (E, n_HI, e_h^n + e_c) to the next step.  Given lambda, the adjoint
// of that hand-over state, the transposed Newton system J_U^T mu = lambda_U is reduced exactly
// like the forward one: with J_Eu = (0, A_En) and the cell-local 2x2 block A_uu,
//     (J_EE - J_Eu A_uu^-1 J_uE)^T mu_E = lambda_E - J_uE^T A_uu^-T lambda_u,
//     mu_u = A_uu^-T (lambda_u - J_Eu^T mu_E),
// and the reduced operator is the forward Schur operator S (symmetric with the lagged limiter),
// so the same multigrid-preconditioned CG solves it.  Then
//     lambda^n = -J_X^T mu (+ lambda_eh passed on to e_h^n),
//     dJ/dNdot_s = dt src_scale mu_E[cell_s],   dJ/dC = mu_n dS_n/dC,
// with J_X taken in gather form: each cell collects the contributions of its own rows and of the
// six face terms it shares with its neighbours (the face coefficient D is differentiated with
// respect to the starting state it is evaluated from).
#include "cellgrid.cuh"
#include "kernels.cuh"

namespace {

constexpr int kBlock = 256;

int grid_for(long long n) {
    long long b = (n + kBlock - 1) / kBlock;
    const long long cap = 152LL * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

using cellgrid::cell_coords;
using cellgrid::dn;
using cellgrid::up;

__device__ __forceinline__ CellIn cell_in(const AdjointArgs& A, long long i) {
    CellIn c;
    c.rho = A.rho[i];
    c.nHI0 = A.n0[i];
    c.E0 = A.E0[i];
    double v2 = 0.0;
    if (A.vx) v2 += A.vx[i] * A.vx[i];
    if (A.vy) v2 += A.vy[i] * A.vy[i];
    if (A.vz) v2 += A.vz[i] * A.vz[i];
    c.eh_kin = A.e_h[i] - 0.5 * v2;
    c.clump = A.clump ? (double)A.clump[i] : 1.0;
    return c;
}

// derivative slots: 0 e_c, 1 n_HI, 2 E, 3 E^n, 4 n_HI^n, 5 C
using D6 = Dual<6>;

struct LocalJac {
    double a11, a12, a21, a22;   // A_uu = d(f_e, f_n)/d(e_c, n_HI)
    double be, bn;               // A_uE = d(f_e, f_n)/dE
    double eE0, nE0;             // d(f_e, f_n)/dE^n
    double en0, nn0;             // d(f_e, f_n)/dn_HI^n
    double eC, nC;               // d(f_e, f_n)/dC
    double eeh, neh;             // d(f_e, f_n)/de_h
};

__device__ __forceinline__ LocalJac local_jacobian(const PhysParams& P, const CellIn& c, double ec, double n,
                                                  double E) {
    D6 Se, Sn;
    local_solutions_full<D6>(P, c, dvar<6>(ec, 0), dvar<6>(n, 1), dvar<6>(E, 2), dvar<6>(c.E0, 3),
                             dvar<6>(c.nHI0, 4), dvar<6>(c.clump, 5), Se, Sn);
    LocalJac J;
    // f_e = e_c - S_e (isothermal: f_e = e_c, S_e = 0), f_n = n_HI - S_n
    J.a11 = 1.0 - Se.d[0];
    J.a12 = -Se.d[1];
    J.a21 = -Sn.d[0];
    J.a22 = 1.0 - Sn.d[1];
    J.be = -Se.d[2];
    J.bn = -Sn.d[2];
    J.eE0 = -Se.d[3];
    J.nE0 = -Sn.d[3];
    J.en0 = -Se.d[4];
    J.nn0 = -Sn.d[4];
    J.eC = -Se.d[5];
    J.nC = -Sn.d[5];
    // e_h enters only through T(e_h + e_c), like e_c does inside S
    J.eeh = -Se.d[0];
    J.neh = -Sn.d[0];
    return J;
}

// right side of the reduced adjoint system: lambda_E - J_uE^T A_uu^-T lambda_u
__global__ void __launch_bounds__(kBlock) k_adj_rhs(PhysParams P, AdjointArgs A) {
    const long long n = (long long)P.nx * P.ny * P.nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const CellIn c = cell_in(A, i);
        const LocalJac J = local_jacobian(P, c, A.ec[i], A.nHI[i], A.E[i]);
        const double le = A.lam_eh_in[i], ln = A.lam_n_in[i];
        const double det = J.a11 * J.a22 - J.a12 * J.a21;
        // v = A_uu^-T (le, ln)
        const double ve = (J.a22 * le - J.a21 * ln) / det;
        const double vn = (-J.a12 * le + J.a11 * ln) / det;
        A.rhs[i] = A.lam_E_in[i] - (J.be * ve + J.bn * vn);
    }
}

// back-substitution and the transposed start-state and parameter Jacobians
__global__ void __launch_bounds__(kBlock) k_adj_back(PhysParams P, AdjointArgs A) {
    const long long n = (long long)P.nx * P.ny * P.nz;
    const double rho_e = (1.0 - P.theta) / P.theta;
    const double dtt = P.dt * P.theta;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        cell_coords(k, P.nx, P.ny, x, y, z);
        const CellIn c = cell_in(A, k);
        const double Ek = A.E[k];
        const LocalJac J = local_jacobian(P, c, A.ec[k], A.nHI[k], Ek);
        const double muE = A.muE[k];
        const double AEn = dtt * P.c * P.kE * Ek / P.a3;
        // mu_u = A_uu^-T (lambda_u - J_Eu^T mu_E),  J_Eu^T mu_E = (0, A_En mu_E)
        const double le = A.lam_eh_in[k], ln = A.lam_n_in[k] - AEn * muE;
        const double det = J.a11 * J.a22 - J.a12 * J.a21;
        const double mue = (J.a22 * le - J.a21 * ln) / det;
        const double mun = (-J.a12 * le + J.a11 * ln) / det;

        // own rows: local equations and the non-face terms of f_E
        const double kap0 = P.kE * c.nHI0 / P.a3;
        double lE0 = -(mue * J.eE0 + mun * J.nE0) + muE * (1.0 - P.dt * (1.0 - P.theta) * (P.H + P.c * kap0));
        double ln0 = -(mue * J.en0 + mun * J.nn0) - muE * P.dt * (1.0 - P.theta) * P.c * P.kE * c.E0 / P.a3;
        const double leh = A.lam_eh_in[k] - (mue * J.eeh + mun * J.neh);

        // face terms Q_f = w_f [(E_b - E_a) + rho (E0_b - E0_a)] with f_E,a -= Q_f, f_E,b += Q_f;
        // cell k collects (mu_E,a - mu_E,b) dQ_f/d(E0_k, n0_k) from each of its six faces
        const long long sy = P.nx, sz = (long long)P.nx * P.ny;
        const long long b0 = k - x - (long long)y * sy - (long long)z * sz;
        const int coords[3] = {x, y, z};
        const int dims[3] = {P.nx, P.ny, P.nz};
        for (int d = 0; d < 3; ++d) {
            for (int side = 0; side < 2; ++side) {
                // side 0: the face to the + neighbour (k = a); side 1: to the - neighbour (k = b)
                const int cc = coords[d];
                if (side == 0 && !P.per[d] && cc == dims[d] - 1) continue;   // wall face
                if (side == 1 && !P.per[d] && cc == 0) continue;
                const int nb = side == 0 ? up(cc, dims[d], P.per[d]) : dn(cc, dims[d], P.per[d]);
                int q[3] = {x, y, z};
                q[d] = nb;
                const long long j = b0 + q[0] + (long long)q[1] * sy + (long long)q[2] * sz;
                const long long a = side == 0 ? k : j, b = side == 0 ? j : k;
                // D at this face as a function of cell k's start values (slots 0: E0_k, 1: n0_k)
                Dual<2> Ea = side == 0 ? dvar<2>(c.E0, 0) : dconst<2>(A.E0[a]);
                Dual<2> Eb = side == 0 ? dconst<2>(A.E0[b]) : dvar<2>(c.E0, 0);
                Dual<2> ka = side == 0 ? dvar<2>(c.nHI0, 1) * (P.kE / P.a3) : dconst<2>(P.kE * A.n0[a] / P.a3);
                Dual<2> kb = side == 0 ? dconst<2>(P.kE * A.n0[b] / P.a3) : dvar<2>(c.nHI0, 1) * (P.kE / P.a3);
                const Dual<2> w = limiter_face_t<Dual<2>>(P, Ea, Eb, ka, kb) * P.wscale;
                const double bracket = (A.E[b] - A.E[a]) + rho_e * (A.E0[b] - A.E0[a]);
                const double sgn = side == 0 ? -1.0 : 1.0;   // d(E0_b - E0_a)/dE0_k
                const double dQdE0 = w.d[0] * bracket + w.v * rho_e * sgn;
                const double dQdn0 = w.d[1] * bracket;
                const double dmu = A.muE[a] - A.muE[b];
                lE0 += dmu * dQdE0;
                ln0 += dmu * dQdn0;
            }
        }
        A.lam_E_out[k] = lE0;
        A.lam_n_out[k] = ln0;
        A.lam_eh_out[k] = leh;
        if (A.g_clump) A.g_clump[k] += (float)(-(mun * J.nC + mue * J.eC));
    }
}

__global__ void k_adj_sources(const AdjointArgs A, int nsrc, double scale, long long ncell) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsrc) return;
    const long long c = A.src_cell[s];
    if (c < 0 || c >= ncell) return;
    A.g_ndot[s] += scale * A.muE[c];
}

}  // namespace

void launch_adj_rhs(const PhysParams& P, const AdjointArgs& A, cudaStream_t s) {
    const long long n = (long long)P.nx * P.ny * P.nz;
    k_adj_rhs<<<grid_for(n), kBlock, 0, s>>>(P, A);
}

void launch_adj_back(const PhysParams& P, const AdjointArgs& A, int nsrc, cudaStream_t s) {
    const long long n = (long long)P.nx * P.ny * P.nz;
    k_adj_back<<<grid_for(n), kBlock, 0, s>>>(P, A);
    if (nsrc > 0 && A.g_ndot) k_adj_sources<<<(nsrc + 255) / 256, 256, 0, s>>>(A, nsrc, P.dt * P.src_scale, n);
}
