// Advection pre-step: step (iv) of the operator split moves the species and radiation densities
// with the baryon velocity (Eqs. enzo-chemical_ionization and enzo-cons_radiation,
// d_t q + (1/a) div(q v_b) = 0), here by the first-order donor-cell finite-volume scheme.
//
// Face f between cell i and its '+' neighbour j on an axis: c_f = (v_i + v_j)/2 * dt/(a dx),
// zero on a wall face.  The flux c_f q_donor (donor i if c_f > 0, else j) leaves i and enters
// j.  One thread per cell gathers its six faces; each face is evaluated by both of its cells.
// The baryon density rho_b (Eq. enzo-cons_mass) can be moved with the same fluxes, which keeps
// n_HI*/n_H* a convex combination of the neighbours' fractions; on helium grids n_HeI and
// n_HeII move with them too.  Per cell the forward map reads
// E, n_HI, rho_b and three velocity components and writes E*, n_HI*, rho_b* (72 bytes) for
// about 50 FP64 operations, so on GB300's FP64 pipe it is ALU-bound, not HBM-bound.
//
//  k_advect_courant  per-cell sum of outflow Courant numbers, block maxima (stability check)
//  k_advect          q* = q - sum of net outward face fluxes, for E, n_HI (and rho_b) together
//  k_advect_adj      the transpose: lam_i + sum over i's outflow faces c (lam_j - lam_i)
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

// the two faces of cell i along axis d: Courant numbers (0 on a wall) and neighbour indices
struct AxisFaces {
    double cp, cm;      // '+' face (i -> j) and '-' face (m -> i), positive along +axis
    long long j, m;
};

__device__ __forceinline__ AxisFaces axis_faces(const AdvectArgs& A, int d, long long i, int coord, int n,
                                                long long stride) {
    AxisFaces f;
    const bool per = A.per[d] != 0;
    const bool has_up = per || coord + 1 < n, has_dn = per || coord > 0;
    f.j = coord + 1 < n ? i + stride : i - (long long)(n - 1) * stride;
    f.m = coord > 0 ? i - stride : i + (long long)(n - 1) * stride;
    const double* v = A.v[d];
    const double vi = v[i];
    f.cp = has_up ? 0.5 * (vi + v[f.j]) * A.k : 0.0;
    f.cm = has_dn ? 0.5 * (v[f.m] + vi) * A.k : 0.0;
    return f;
}

__device__ __forceinline__ void coords(long long i, int nx, int ny, int& x, int& y, int& z) {
    long long q = i / nx;
    x = (int)(i - q * nx);
    z = (int)(q / ny);
    y = (int)(q - (long long)z * ny);
}

__global__ void __launch_bounds__(kBlock) k_advect_courant(AdvectArgs A) {
    const long long n = (long long)A.nx * A.ny * A.nz;
    const int dims[3] = {A.nx, A.ny, A.nz};
    const long long strides[3] = {1, A.nx, (long long)A.nx * A.ny};
    double cmax = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int c[3];
        coords(i, A.nx, A.ny, c[0], c[1], c[2]);
        double out = 0.0;
        for (int d = 0; d < 3; ++d) {
            if (!A.v[d]) continue;
            const AxisFaces f = axis_faces(A, d, i, c[d], dims[d], strides[d]);
            out += fmax(f.cp, 0.0) + fmax(-f.cm, 0.0);
        }
        cmax = fmax(cmax, out);
    }
    __shared__ double sh[kBlock / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cmax = fmax(cmax, __shfl_down_sync(0xffffffffu, cmax, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = cmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) m = fmax(m, sh[w]);
        A.partials[blockIdx.x] = m;
    }
}

__global__ void __launch_bounds__(kBlock) k_advect(AdvectArgs A) {
    const long long n = (long long)A.nx * A.ny * A.nz;
    const int dims[3] = {A.nx, A.ny, A.nz};
    const long long strides[3] = {1, A.nx, (long long)A.nx * A.ny};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int c[3];
        coords(i, A.nx, A.ny, c[0], c[1], c[2]);
        const double Ei = A.qE[i], ni = A.qn[i], ri = A.qr ? A.qr[i] : 0.0;
        double oE = Ei, on = ni, orh = ri;
        double o1 = A.qh1 ? A.qh1[i] : 0.0, o2 = A.qh2 ? A.qh2[i] : 0.0;
        for (int d = 0; d < 3; ++d) {
            if (!A.v[d]) continue;
            const AxisFaces f = axis_faces(A, d, i, c[d], dims[d], strides[d]);
            // donors of the '+' and '-' faces (the cell the flow leaves)
            const long long dp = f.cp > 0.0 ? i : f.j, dm = f.cm > 0.0 ? f.m : i;
            oE = oE - (f.cp * A.qE[dp] - f.cm * A.qE[dm]);
            on = on - (f.cp * A.qn[dp] - f.cm * A.qn[dm]);
            if (A.qr) orh = orh - (f.cp * A.qr[dp] - f.cm * A.qr[dm]);
            if (A.qh1) {
                o1 = o1 - (f.cp * A.qh1[dp] - f.cm * A.qh1[dm]);
                o2 = o2 - (f.cp * A.qh2[dp] - f.cm * A.qh2[dm]);
            }
        }
        A.oE[i] = oE;
        A.on[i] = on;
        if (A.qr) A.orh[i] = orh;
        if (A.qh1) {
            A.oh1[i] = o1;
            A.oh2[i] = o2;
        }
    }
}

__global__ void __launch_bounds__(kBlock) k_advect_adj(AdvectArgs A) {
    const long long n = (long long)A.nx * A.ny * A.nz;
    const int dims[3] = {A.nx, A.ny, A.nz};
    const long long strides[3] = {1, A.nx, (long long)A.nx * A.ny};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int c[3];
        coords(i, A.nx, A.ny, c[0], c[1], c[2]);
        const double Ei = A.qE[i], ni = A.qn[i];
        double oE = Ei, on = ni;
        for (int d = 0; d < 3; ++d) {
            if (!A.v[d]) continue;
            const AxisFaces f = axis_faces(A, d, i, c[d], dims[d], strides[d]);
            if (f.cp > 0.0) {            // flow leaves i through its '+' face into j
                oE += f.cp * (A.qE[f.j] - Ei);
                on += f.cp * (A.qn[f.j] - ni);
            }
            if (f.cm < 0.0) {            // flow leaves i through its '-' face into m
                oE -= f.cm * (A.qE[f.m] - Ei);
                on -= f.cm * (A.qn[f.m] - ni);
            }
        }
        A.oE[i] = oE;
        A.on[i] = on;
    }
}

}  // namespace

int launch_advect_courant(const AdvectArgs& A, cudaStream_t s) {
    const int g = grid_for((long long)A.nx * A.ny * A.nz);
    k_advect_courant<<<g, kBlock, 0, s>>>(A);
    return g;
}

void launch_advect(const AdvectArgs& A, bool transpose, cudaStream_t s) {
    const int g = grid_for((long long)A.nx * A.ny * A.nz);
    if (transpose) k_advect_adj<<<g, kBlock, 0, s>>>(A);
    else k_advect<<<g, kBlock, 0, s>>>(A);
}
