// Linear-solver kernels for the reduced (Schur) radiation system S x = b.
//
// S is the 7-point symmetric operator (S x)_i = diag_i x_i - sum_faces w_f x_nb, stored as
// the diagonal and the coupling on each cell's +x/+y/+z face (a wall face has w = 0).
//
//  * FP64 conjugate-gradient vector kernels (matrix-vector product with fused dot product,
//    fused x/r update with the residual norm, fused dot pairs) -- HBM-bound streams;
//  * geometric multigrid, templated on the working precision T (float for the mixed path):
//      - red-black Gauss-Seidel sweeps as two in-place colour passes over a colour-split
//        storage of each smoothed level (rbpass.cuh);
//      - fused residual + restriction (average of the 8 children) and the trilinear
//        cell-centred prolongation of the coarse correction added to the fine iterate;
//      - coarse operators by averaging: sigma_c = geometric mean of the children's
//        sigma = diag - sum w, coarse face coupling = sum of the 4 fine face couplings / 16
//        (what re-discretising the diffusion term on the doubled cell gives for constant
//        coefficients);
//      - a single-CTA solver that runs the remaining coarse levels in shared memory and finishes
//        with a dense Cholesky solve (or the exact 1-cell solve) on the coarsest one.
#include "cellgrid.cuh"
#include "kernels.cuh"
#include "rbpass.cuh"
#include "fpbits.cuh"

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

// block partials of NS sums followed by NM maxima (slot k at partials[k * gridDim.x + block])
template <int NS, int NM>
__device__ void block_sums_max(double (&v)[NS + NM], double* partials) {
    __shared__ double sh[NS + NM][kBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NS + NM; ++k) {
        double s = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double t = __shfl_down_sync(0xffffffffu, s, o);
            s = k < NS ? s + t : fmax(s, t);
        }
        if (lane == 0) sh[k][warp] = s;
    }
    __syncthreads();
    if (threadIdx.x < NS + NM) {
        double s = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) s = (int)threadIdx.x < NS ? s + sh[threadIdx.x][w] : fmax(s, sh[threadIdx.x][w]);
        partials[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
    }
}

template <int NS>
__device__ void block_sums(double (&v)[NS], double* partials) {
    __shared__ double sh[NS][kBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        double s = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) sh[k][warp] = s;
    }
    __syncthreads();
    if (threadIdx.x < NS) {
        double s = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) s += sh[threadIdx.x][w];
        partials[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
    }
}

// (S v)_i for cell i with coordinates (x, y, z)
template <class T, class V>
__device__ __forceinline__ V apply_S(long long i, int x, int y, int z, const Dims& d, const T* __restrict__ diag,
                                     const T* __restrict__ wx, const T* __restrict__ wy, const T* __restrict__ wz,
                                     const V* __restrict__ v) {
    const long long sy = d.nx, sz = (long long)d.nx * d.ny;
    const long long b = i - x - (long long)y * sy - (long long)z * sz;
    const long long xm = b + dn(x, d.nx, d.per[0]) + y * sy + z * sz;
    const long long xp = b + up(x, d.nx, d.per[0]) + y * sy + z * sz;
    const long long ym = b + x + dn(y, d.ny, d.per[1]) * sy + z * sz;
    const long long yp = b + x + up(y, d.ny, d.per[1]) * sy + z * sz;
    const long long zm = b + x + y * sy + dn(z, d.nz, d.per[2]) * sz;
    const long long zp = b + x + y * sy + up(z, d.nz, d.per[2]) * sz;
    const V wxm = (!d.per[0] && x == 0) ? V(0) : V(wx[xm]);
    const V wym = (!d.per[1] && y == 0) ? V(0) : V(wy[ym]);
    const V wzm = (!d.per[2] && z == 0) ? V(0) : V(wz[zm]);
    V off = V(wx[i]) * v[xp] + wxm * v[xm] + V(wy[i]) * v[yp] + wym * v[ym] + V(wz[i]) * v[zp] + wzm * v[zm];
    return V(diag[i]) * v[i] - off;
}

// ------------------------------------------------------------------ CG kernels (FP64)

__global__ void __launch_bounds__(kBlock) k_spmv_dot(Dims d, const double* __restrict__ diag,
                                                      const double* __restrict__ wx, const double* __restrict__ wy,
                                                      const double* __restrict__ wz, const double* __restrict__ p,
                                                      double* __restrict__ q, double* partials) {
    const long long n = d.n();
    double acc[1] = {0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        cell_coords(i, d.nx, d.ny, x, y, z);
        const double v = apply_S<double, double>(i, x, y, z, d, diag, wx, wy, wz, p);
        q[i] = v;
        acc[0] += p[i] * v;
    }
    block_sums<1>(acc, partials);
}

__global__ void __launch_bounds__(kBlock) k_residual_norm(Dims d, const double* __restrict__ diag,
                                                           const double* __restrict__ wx, const double* __restrict__ wy,
                                                           const double* __restrict__ wz, const double* __restrict__ b,
                                                           const double* __restrict__ xv, double* __restrict__ r,
                                                           const double* __restrict__ w, double* partials) {
    const long long n = d.n();
    double acc[2] = {0.0, 0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        cell_coords(i, d.nx, d.ny, x, y, z);
        const double v = b[i] - apply_S<double, double>(i, x, y, z, d, diag, wx, wy, wz, xv);
        r[i] = v;
        const double wv = w ? w[i] * v : v;
        acc[0] += wv * wv;
        acc[1] = fmax(acc[1], fabs(v));
    }
    block_sums_max<1, 1>(acc, partials);
}

__global__ void __launch_bounds__(kBlock) k_cg_update_xr(long long n, const double* __restrict__ scal,
                                                          double* __restrict__ x, double* __restrict__ r,
                                                          const double* __restrict__ p, const double* __restrict__ q,
                                                          const double* __restrict__ w, double* partials) {
    const double alpha = scal[0];
    double acc[2] = {0.0, 0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        x[i] = fma(alpha, p[i], x[i]);
        const double rv = fma(-alpha, q[i], r[i]);
        r[i] = rv;
        const double wv = w ? w[i] * rv : rv;
        acc[0] += wv * wv;
        acc[1] = fmax(acc[1], fabs(rv));
    }
    block_sums_max<1, 1>(acc, partials);
}

__global__ void __launch_bounds__(kBlock) k_dot2(long long n, const double* __restrict__ z, const double* __restrict__ r,
                                                  const double* __restrict__ q, double* partials) {
    double acc[2] = {0.0, 0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double zi = z[i];
        acc[0] += zi * r[i];
        if (q) acc[1] += zi * q[i];
    }
    block_sums<2>(acc, partials);
}

__global__ void k_p_update(long long n, const double* __restrict__ scal, const double* __restrict__ z,
                           double* __restrict__ p) {
    const double beta = scal[1];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = fma(beta, p[i], z[i]);
}

// Diagonal of the operator the multigrid preconditioner works on.  Where the local
// elimination makes sigma = diag - sum_faces w negative (a cell crossing the ionisation
// fold: more light makes it more transparent), the row is not diagonally dominant and
// Gauss-Seidel / coarse-grid correction diverge; the preconditioner uses sigma = 0 there,
// which keeps it a symmetric M-matrix.  The outer CG works on the true operator.
template <class T>
__global__ void k_mg_diag(Dims d, const double* __restrict__ diag, const double* __restrict__ wx,
                          const double* __restrict__ wy, const double* __restrict__ wz, T* __restrict__ out) {
    const long long n = d.n();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        cell_coords(i, d.nx, d.ny, x, y, z);
        const long long sy = d.nx, sz = (long long)d.nx * d.ny;
        const long long b = i - x - (long long)y * sy - (long long)z * sz;
        const double wxm = (!d.per[0] && x == 0) ? 0.0 : wx[b + dn(x, d.nx, d.per[0]) + y * sy + z * sz];
        const double wym = (!d.per[1] && y == 0) ? 0.0 : wy[b + x + dn(y, d.ny, d.per[1]) * sy + z * sz];
        const double wzm = (!d.per[2] && z == 0) ? 0.0 : wz[b + x + y * sy + dn(z, d.nz, d.per[2]) * sz];
        const double sw = wx[i] + wy[i] + wz[i] + wxm + wym + wzm;
        out[i] = (T)fmax(diag[i], sw);
    }
}

// Level-0 vectors in the multigrid's storage order, as r 2^-e on the way in and x 2^e on the way
// out (2^e >= *amax; e = 0 when amax is null).  Between FP64 and FP32 the scaled conversion works
// on the bit patterns (fpbits.cuh); FP64 to FP64 is a permutation.
__device__ __forceinline__ int scale_exponent(const double* amax) { return amax ? fpbits::pow2_exponent(*amax) : 0; }
__device__ __forceinline__ float cvt_in(double v, int e, float*) { return fpbits::to_float_scaled(v, e); }
__device__ __forceinline__ double cvt_in(double v, int, double*) { return v; }
__device__ __forceinline__ double cvt_out(float v, int e) { return fpbits::from_float_scaled(v, e); }
__device__ __forceinline__ double cvt_out(double v, int) { return v; }

// natural order: thread per cell
template <class Tin, class Tout>
__global__ void k_to_level(Dims d, const Tin* __restrict__ a, Tout* __restrict__ out, const double* __restrict__ amax) {
    const int e = scale_exponent(amax);
    const long long n = d.n();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = cvt_in(a[i], e, (Tout*)nullptr);
}
template <class Tin, class Tout>
__global__ void k_from_level(Dims d, const Tin* __restrict__ a, Tout* __restrict__ out,
                             const double* __restrict__ amax) {
    const int e = scale_exponent(amax);
    const long long n = d.n();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = cvt_out(a[i], e);
}
// Colour-split order: thread per x-pair (one 16-byte load or store of the FP64 pair, one element
// into or out of each colour half), launched in pass_grid's shape so that no index is divided
template <class Tout>
__global__ void __launch_bounds__(rbp::kPairs) k_to_split(Dims d, int rows, const double* __restrict__ a,
                                                          Tout* __restrict__ out, const double* __restrict__ amax) {
    int px, y, z;
    if (!rbp::grid_pair(d.nx, d.ny, rows, blockIdx.x, blockIdx.y, blockIdx.z, threadIdx.x, px, y, z)) return;
    const int e = scale_exponent(amax);
    const long long hx = d.nx >> 1, half = hx * d.ny * d.nz;
    const long long m = ((long long)z * d.ny + y) * hx + px;
    const int c0 = (y + z) & 1;   // colour of the pair's even-x cell
    const double2 v = reinterpret_cast<const double2*>(a)[m];
    out[c0 * half + m] = cvt_in(v.x, e, (Tout*)nullptr);
    out[(1 - c0) * half + m] = cvt_in(v.y, e, (Tout*)nullptr);
}
template <class Tin>
__global__ void __launch_bounds__(rbp::kPairs) k_from_split(Dims d, int rows, const Tin* __restrict__ a,
                                                            double* __restrict__ out, const double* __restrict__ amax) {
    int px, y, z;
    if (!rbp::grid_pair(d.nx, d.ny, rows, blockIdx.x, blockIdx.y, blockIdx.z, threadIdx.x, px, y, z)) return;
    const int e = scale_exponent(amax);
    const long long hx = d.nx >> 1, half = hx * d.ny * d.nz;
    const long long m = ((long long)z * d.ny + y) * hx + px;
    const int c0 = (y + z) & 1;
    double2 v;
    v.x = cvt_out(a[c0 * half + m], e);
    v.y = cvt_out(a[(1 - c0) * half + m], e);
    reinterpret_cast<double2*>(out)[m] = v;
}
__global__ void k_add(long long n, const double* __restrict__ a, double* __restrict__ b) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] += a[i];
}
__global__ void k_copy(long long n, const double* __restrict__ a, double* __restrict__ b) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = a[i];
}

// scal: [0] alpha, [1] beta, [2] (z, r), [3] (p, q).  dots: finalize output of the phase.
//   phase 0: dots = {(z,r)}         -> scal[2]
//   phase 1: dots = {(p,q)}         -> scal[3], alpha = scal[2] / scal[3]
//   phase 2: dots = {(z,r), (z,q)}  -> beta = -(z,q) / (p,q) (flexible Polak-Ribiere), scal[2]
__global__ void k_cg_scalars(double* scal, const double* dots, int phase) {
    if (threadIdx.x != 0) return;
    if (phase == 0) {
        scal[2] = dots[0];
    } else if (phase == 1) {
        scal[3] = dots[0];
        scal[0] = scal[2] / scal[3];
    } else {
        scal[1] = -dots[1] / scal[3];
        scal[2] = dots[0];
    }
}

// ------------------------------------------------------------------- multigrid kernels

// one colour pass (colour C) of a red-black sweep of a colour-split level in place (rbpass.cuh)
template <int C, class T>
__global__ void __launch_bounds__(rbp::kPairs, 16) k_rbgs_pass(rbp::Pass<T> A) {
    if (A.quad) {   // two pairs per thread, two-element loads and stores
        int px, y, z;
        if (!rbp::quad_pairs(A, blockIdx.x, blockIdx.y, blockIdx.z, threadIdx.x, px, y, z)) return;
        T v0, v1;
        rbp::quad_values<C>(A, px, y, z, v0, v1);
        rbp::st2(A.x + (z * A.ny + y) * (A.nx >> 1) + px, v0, v1);
        return;
    }
    int x, y, z;
    if (!rbp::pair_cell(A, blockIdx.x, blockIdx.y, blockIdx.z, threadIdx.x, x, y, z)) return;
    A.x[rbp::pair_of(A, x, y, z)] = rbp::cell_value<C>(A, x, y, z);
}

// the smoother's copy of a level's operator (colour-split diagonal, colour-0 face arrays)
template <class T>
__global__ void __launch_bounds__(kBlock) k_split_level(Level<T> L) {
    const long long half = L.d.n() / 2;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < half; m += (long long)gridDim.x * blockDim.x)
        rbp::split_pair(L.d.nx, L.d.ny, L.d.nz, L.d.per, L.diag, L.wx, L.wy, L.wz, m, L.dinv, L.w6);
}

// x += P xc: trilinear cell-centred prolongation of the coarse correction; thread per fine pair
// (both cells lie in one coarse cell, rbp::prolong_pair), launched in pass_grid's shape
template <class T>
__global__ void __launch_bounds__(rbp::kPairs) k_prolong_add(Level<T> c, Level<T> f, int rows) {
    int px, y, z;
    if (!rbp::grid_pair(f.d.nx, f.d.ny, rows, blockIdx.x, blockIdx.y, blockIdx.z, threadIdx.x, px, y, z)) return;
    const int hx = f.d.nx >> 1, half = hx * f.d.ny * f.d.nz;
    const int m = (z * f.d.ny + y) * hx + px;
    const int c0 = (y + z) & 1;   // colour of the even-x cell
    T v0, v1;
    rbp::prolong_pair(c.x, c.split, c.d.nx, c.d.ny, c.d.nz, c.d.per, px, y, z, v0, v1);
    f.x[c0 * half + m] += v0;
    f.x[(1 - c0) * half + m] += v1;
}

// c.b = average over the 8 children of f.b - S f.x: thread per coarse cell, whose children are
// fine pair X of the four fine rows (2Y + j, 2Z + k) (rbp::pair_residuals), launched in the
// passes' shape over the coarse cells
template <class T>
__global__ void __launch_bounds__(rbp::kPairs) k_resid_restrict(Level<T> f, Level<T> c, int rows) {
    int X, Y, Z;
    if (!rbp::grid_pair(2 * c.d.nx, c.d.ny, rows, blockIdx.x, blockIdx.y, blockIdx.z, threadIdx.x, X, Y, Z)) return;
    T sum = T(0);
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            T rE, rO;
            rbp::pair_residuals(f.d.nx, f.d.ny, f.d.nz, f.d.per, f.diag, f.wx, f.wy, f.wz, f.b, f.x, X, 2 * Y + j,
                                2 * Z + k, rE, rO);
            sum += rE + rO;
        }
    c.b[rbp::level_index(c.split, c.d.nx, c.d.ny, c.d.nz, X, Y, Z)] = sum * T(0.125);
}

template <class T>
__device__ __forceinline__ void coarsen_cell(const Dims& fd, const T* fdiag, const T* fwx, const T* fwy, const T* fwz,
                                             const Dims& cd, long long I, int X, int Y, int Z, T* cdiag, T* cwx,
                                             T* cwy, T* cwz) {
    const long long fsy = fd.nx, fsz = (long long)fd.nx * fd.ny;
    auto fi = [&](int x, int y, int z) { return (long long)z * fsz + (long long)y * fsy + x; };
    // coarse sigma: geometric mean of the children's sigma.  Around a small ionised bubble
    // the children mix sigma ~ 1 (transparent) with sigma ~ 1e4 (neutral, optically thick);
    // an arithmetic mean makes every coarse cell touching neutral gas look opaque and the
    // bubble's smooth error modes get no coarse correction (measured: more CG iterations)
    T sig = T(0);
    for (int k = 0; k < 2; ++k)
        for (int j = 0; j < 2; ++j)
            for (int l = 0; l < 2; ++l) {
                const int x = 2 * X + l, y = 2 * Y + j, z = 2 * Z + k;
                const long long i = fi(x, y, z);
                const T wxm = (!fd.per[0] && x == 0) ? T(0) : fwx[fi(dn(x, fd.nx, fd.per[0]), y, z)];
                const T wym = (!fd.per[1] && y == 0) ? T(0) : fwy[fi(x, dn(y, fd.ny, fd.per[1]), z)];
                const T wzm = (!fd.per[2] && z == 0) ? T(0) : fwz[fi(x, y, dn(z, fd.nz, fd.per[2]))];
                const T sc = fdiag[i] - (fwx[i] + fwy[i] + fwz[i] + wxm + wym + wzm);
                sig += log(sc > T(1e-30) ? sc : T(1e-30));
            }
    sig = exp(sig * T(0.125));
    // + faces: fine faces leaving the children on the + side
    T ax = T(0), ay = T(0), az = T(0), bx = T(0), by = T(0), bz = T(0);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            ax += fwx[fi(2 * X + 1, 2 * Y + a, 2 * Z + b)];
            ay += fwy[fi(2 * X + a, 2 * Y + 1, 2 * Z + b)];
            az += fwz[fi(2 * X + a, 2 * Y + b, 2 * Z + 1)];
            // - faces: the + faces of the fine cells just below this coarse cell
            if (fd.per[0] || X > 0) bx += fwx[fi(dn(2 * X, fd.nx, fd.per[0]), 2 * Y + a, 2 * Z + b)];
            if (fd.per[1] || Y > 0) by += fwy[fi(2 * X + a, dn(2 * Y, fd.ny, fd.per[1]), 2 * Z + b)];
            if (fd.per[2] || Z > 0) bz += fwz[fi(2 * X + a, 2 * Y + b, dn(2 * Z, fd.nz, fd.per[2]))];
        }
    const T s = T(1.0 / 16.0);
    cwx[I] = ax * s;
    cwy[I] = ay * s;
    cwz[I] = az * s;
    cdiag[I] = sig + (ax + ay + az + bx + by + bz) * s;
}

template <class T>
__global__ void __launch_bounds__(kBlock) k_coarsen(Level<T> f, Level<T> c) {
    const long long nc = c.d.n();
    for (long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x; I < nc; I += (long long)gridDim.x * blockDim.x) {
        int X, Y, Z;
        cell_coords(I, c.d.nx, c.d.ny, X, Y, Z);
        coarsen_cell<T>(f.d, f.diag, f.wx, f.wy, f.wz, c.d, I, X, Y, Z, c.diag, c.wx, c.wy, c.wz);
    }
}

// ----------------------------------------------------------- single-CTA coarse solver

constexpr int kTailThreads = 1024;
constexpr int kTailMaxLevels = 16;
constexpr int kDenseMax = 64;

struct TailPlan {
    int nlev;
    Dims d[kTailMaxLevels];
    int off[kTailMaxLevels];   // cell offset of each level in the packed arrays
    int total;                 // packed cells
    int dense;                 // coarsest level solved by dense Cholesky (cells <= kDenseMax)
};

__host__ __device__ inline void make_plan(const Dims& top, TailPlan& p) {
    p.nlev = 0;
    p.total = 0;
    Dims d = top;
    while (true) {
        p.d[p.nlev] = d;
        p.off[p.nlev] = p.total;
        p.total += (int)d.n();
        p.nlev++;
        const bool even = (d.nx % 2 == 0) && (d.ny % 2 == 0) && (d.nz % 2 == 0);
        if (!even || d.n() <= 1 || p.nlev == kTailMaxLevels) break;
        d.nx /= 2;
        d.ny /= 2;
        d.nz /= 2;
    }
    const Dims& last = p.d[p.nlev - 1];
    p.dense = (last.n() > 1 && last.n() <= kDenseMax) ? 1 : 0;
}

// colouring of a shared-memory level for its Gauss-Seidel sweeps (rbpass.cuh)
__device__ __forceinline__ bool odd_periodic(const Dims& d) {
    return rbp::odd_periodic(d.nx, d.ny, d.nz, d.per);
}
__device__ __forceinline__ int tail_colour(const Dims& d, int ncol, int x, int y, int z) {
    return rbp::multicolour(d.nx, d.ny, d.nz, d.per, ncol, x, y, z);
}

// one colour of a multicolour Gauss-Seidel sweep on a shared-memory level: the new value is
// (b + sum of the neighbours' couplings) / diag; the cell's own previous value is not read.  All
// new values of the colour are computed before any is stored.  Levels hold at most
// kTailCellsPerThread * blockDim.x cells.
constexpr int kTailCellsPerThread = 4;

template <class T>
__device__ void tail_smooth(const Dims& d, T* diag, T* wx, T* wy, T* wz, T* x, const T* b, int ncol, int color,
                            bool zero) {
    const long long n = d.n();
    const long long sy = d.nx, sz = (long long)d.nx * d.ny;
    T nv[kTailCellsPerThread];
#pragma unroll
    for (int k = 0; k < kTailCellsPerThread; ++k) {
        const long long i = threadIdx.x + (long long)k * blockDim.x;
        nv[k] = T(0);
        if (i >= n) continue;
        int cx, cy, cz;
        cell_coords(i, d.nx, d.ny, cx, cy, cz);
        if (tail_colour(d, ncol, cx, cy, cz) != color) continue;
        T num = b[i];
        if (!zero) {
            const long long b0 = i - cx - (long long)cy * sy - (long long)cz * sz;
            const long long xm = b0 + dn(cx, d.nx, d.per[0]) + cy * sy + cz * sz;
            const long long xp = b0 + up(cx, d.nx, d.per[0]) + cy * sy + cz * sz;
            const long long ym = b0 + cx + dn(cy, d.ny, d.per[1]) * sy + cz * sz;
            const long long yp = b0 + cx + up(cy, d.ny, d.per[1]) * sy + cz * sz;
            const long long zm = b0 + cx + cy * sy + dn(cz, d.nz, d.per[2]) * sz;
            const long long zp = b0 + cx + cy * sy + up(cz, d.nz, d.per[2]) * sz;
            const T wxm = (!d.per[0] && cx == 0) ? T(0) : wx[xm];
            const T wym = (!d.per[1] && cy == 0) ? T(0) : wy[ym];
            const T wzm = (!d.per[2] && cz == 0) ? T(0) : wz[zm];
            num += wx[i] * x[xp] + wxm * x[xm] + wy[i] * x[yp] + wym * x[ym] + wz[i] * x[zp] + wzm * x[zm];
        }
        nv[k] = num / diag[i];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kTailCellsPerThread; ++k) {
        const long long i = threadIdx.x + (long long)k * blockDim.x;
        if (i >= n) continue;
        int cx, cy, cz;
        cell_coords(i, d.nx, d.ny, cx, cy, cz);
        if (tail_colour(d, ncol, cx, cy, cz) == color) x[i] = nv[k];
    }
}

template <class T>
__global__ void __launch_bounds__(kTailThreads) k_tail(Level<T> L, int ncycles, int nu, TailPlan plan) {
    extern __shared__ unsigned char smem_raw[];
    T* base = reinterpret_cast<T*>(smem_raw);
    const int tot = plan.total;
    T* sdiag = base;
    T* swx = base + tot;
    T* swy = base + 2 * tot;
    T* swz = base + 3 * tot;
    T* sx = base + 4 * tot;
    T* sb = base + 5 * tot;
    T* dense = base + 6 * tot;          // kDenseMax^2 (+ kDenseMax rhs) when plan.dense
    const long long n0 = L.d.n();
    for (long long i = threadIdx.x; i < n0; i += blockDim.x) {
        sdiag[i] = L.diag[i];
        swx[i] = L.wx[i];
        swy[i] = L.wy[i];
        swz[i] = L.wz[i];
        sb[i] = L.b[i];
    }
    // every level's iterate starts at zero: shared memory holds whatever an earlier kernel left
    for (int i = threadIdx.x; i < tot; i += blockDim.x) sx[i] = T(0);
    __syncthreads();
    for (int l = 1; l < plan.nlev; ++l) {
        const Dims& cd = plan.d[l];
        const Dims& fd = plan.d[l - 1];
        const int fo = plan.off[l - 1], co = plan.off[l];
        for (long long I = threadIdx.x; I < cd.n(); I += blockDim.x) {
            int X, Y, Z;
            cell_coords(I, cd.nx, cd.ny, X, Y, Z);
            coarsen_cell<T>(fd, sdiag + fo, swx + fo, swy + fo, swz + fo, cd, I, X, Y, Z, sdiag + co, swx + co,
                            swy + co, swz + co);
        }
        __syncthreads();
    }
    const int last = plan.nlev - 1;
    const Dims& ld = plan.d[last];
    const int lo = plan.off[last];
    const int m = (int)ld.n();
    if (plan.dense) {
        // assemble the coarsest operator densely and factor it once (Cholesky, lower triangle)
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) dense[e] = T(0);
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int i = 0; i < m; ++i) {
                int cx, cy, cz;
                cell_coords(i, ld.nx, ld.ny, cx, cy, cz);
                dense[i * m + i] += sdiag[lo + i];
                const int nbx[3] = {up(cx, ld.nx, ld.per[0]), up(cy, ld.ny, ld.per[1]), up(cz, ld.nz, ld.per[2])};
                const T w[3] = {swx[lo + i], swy[lo + i], swz[lo + i]};
                for (int dd = 0; dd < 3; ++dd) {
                    if (w[dd] == T(0)) continue;
                    int jx = cx, jy = cy, jz = cz;
                    if (dd == 0) jx = nbx[0];
                    if (dd == 1) jy = nbx[1];
                    if (dd == 2) jz = nbx[2];
                    const int j = (jz * ld.ny + jy) * ld.nx + jx;
                    dense[i * m + j] -= w[dd];
                    dense[j * m + i] -= w[dd];
                }
            }
        }
        __syncthreads();
        for (int k = 0; k < m; ++k) {
            if (threadIdx.x == 0) {
                T dkk = dense[k * m + k];
                dense[k * m + k] = dkk > T(0) ? sqrt(dkk) : T(1);
            }
            __syncthreads();
            const T piv = dense[k * m + k];
            for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) dense[i * m + k] /= piv;
            __syncthreads();
            for (int e = threadIdx.x; e < (m - k - 1) * (m - k - 1); e += blockDim.x) {
                const int i = k + 1 + e / (m - k - 1), j = k + 1 + e % (m - k - 1);
                if (j <= i) dense[i * m + j] -= dense[i * m + k] * dense[j * m + k];
            }
            __syncthreads();
        }
    }
    for (int cyc = 0; cyc < ncycles; ++cyc) {
        for (int l = 0; l < last; ++l) {
            const Dims& d = plan.d[l];
            const int o = plan.off[l];
            const bool zero_start = (l > 0) || (cyc == 0);
            const int ncol = odd_periodic(d) ? 3 : 2;
            for (int s = 0; s < nu; ++s)
                for (int col = 0; col < ncol; ++col) {
                    tail_smooth<T>(d, sdiag + o, swx + o, swy + o, swz + o, sx + o, sb + o, ncol, col,
                                   zero_start && s == 0 && col == 0);
                    __syncthreads();
                }
            const Dims& cd = plan.d[l + 1];
            const int co = plan.off[l + 1];
            for (long long I = threadIdx.x; I < cd.n(); I += blockDim.x) {
                int X, Y, Z;
                cell_coords(I, cd.nx, cd.ny, X, Y, Z);
                T sum = T(0);
                for (int k = 0; k < 2; ++k)
                    for (int j = 0; j < 2; ++j)
                        for (int a = 0; a < 2; ++a) {
                            const int x = 2 * X + a, y = 2 * Y + j, z = 2 * Z + k;
                            const long long i = ((long long)z * d.ny + y) * d.nx + x;
                            sum += sb[o + i] -
                                   apply_S<T, T>(i, x, y, z, d, sdiag + o, swx + o, swy + o, swz + o, sx + o);
                        }
                sb[co + I] = sum * T(0.125);
            }
            __syncthreads();
        }
        // coarsest level
        if (m == 1) {
            if (threadIdx.x == 0) {
                const T sig = sdiag[lo] - T(2) * (swx[lo] + swy[lo] + swz[lo]);
                const T wsum = ld.per[0] || ld.per[1] || ld.per[2] ? sig : sdiag[lo];
                sx[lo] = sb[lo] / (wsum != T(0) ? wsum : T(1));
            }
            __syncthreads();
        } else if (plan.dense) {
            if (threadIdx.x == 0) {
                T* y = dense + m * m;
                for (int i = 0; i < m; ++i) {
                    T s = sb[lo + i];
                    for (int j = 0; j < i; ++j) s -= dense[i * m + j] * y[j];
                    y[i] = s / dense[i * m + i];
                }
                for (int i = m - 1; i >= 0; --i) {
                    T s = y[i];
                    for (int j = i + 1; j < m; ++j) s -= dense[j * m + i] * sx[lo + j];
                    sx[lo + i] = s / dense[i * m + i];
                }
            }
            __syncthreads();
        } else {
            const int ncol = odd_periodic(ld) ? 3 : 2;
            for (int s = 0; s < 8 * (ld.nx + ld.ny + ld.nz); ++s)
                for (int col = 0; col < ncol; ++col) {
                    tail_smooth<T>(ld, sdiag + lo, swx + lo, swy + lo, swz + lo, sx + lo, sb + lo, ncol, col,
                                   s == 0 && col == 0);
                    __syncthreads();
                }
        }
        for (int l = last - 1; l >= 0; --l) {
            const Dims& d = plan.d[l];
            const Dims& cd = plan.d[l + 1];
            const int o = plan.off[l], co = plan.off[l + 1];
            for (long long i = threadIdx.x; i < d.n(); i += blockDim.x) {
                int x, y, z;
                cell_coords(i, d.nx, d.ny, x, y, z);
                const int X = x >> 1, Y = y >> 1, Z = z >> 1;
                const int X2 = (x & 1) ? up(X, cd.nx, cd.per[0]) : dn(X, cd.nx, cd.per[0]);
                const int Y2 = (y & 1) ? up(Y, cd.ny, cd.per[1]) : dn(Y, cd.ny, cd.per[1]);
                const int Z2 = (z & 1) ? up(Z, cd.nz, cd.per[2]) : dn(Z, cd.nz, cd.per[2]);
                auto C = [&](int a, int b, int e) { return sx[co + (e * cd.ny + b) * cd.nx + a]; };
                const T w1 = T(0.75), w2 = T(0.25);
                const T v1 = w1 * (w1 * C(X, Y, Z) + w2 * C(X2, Y, Z)) + w2 * (w1 * C(X, Y2, Z) + w2 * C(X2, Y2, Z));
                const T v2 = w1 * (w1 * C(X, Y, Z2) + w2 * C(X2, Y, Z2)) + w2 * (w1 * C(X, Y2, Z2) + w2 * C(X2, Y2, Z2));
                sx[o + i] += w1 * v1 + w2 * v2;
            }
            __syncthreads();
            // post-smoothing takes the colours in reverse order
            const int ncol = odd_periodic(d) ? 3 : 2;
            for (int s = 0; s < nu; ++s)
                for (int col = ncol - 1; col >= 0; --col) {
                    tail_smooth<T>(d, sdiag + o, swx + o, swy + o, swz + o, sx + o, sb + o, ncol, col, false);
                    __syncthreads();
                }
        }
    }
    for (long long i = threadIdx.x; i < n0; i += blockDim.x) L.x[i] = sx[i];
}

}  // namespace

// ---------------------------------------------------------------------- launchers

int launch_spmv_dot(const Dims& D, const double* diag, const double* wx, const double* wy, const double* wz,
                    const double* p, double* q, double* partials, cudaStream_t s) {
    const int g = grid_for(D.n());
    k_spmv_dot<<<g, kBlock, 0, s>>>(D, diag, wx, wy, wz, p, q, partials);
    return g;
}
int launch_residual_norm(const Dims& D, const double* diag, const double* wx, const double* wy, const double* wz,
                         const double* b, const double* x, double* r, const double* w, double* partials,
                         cudaStream_t s) {
    const int g = grid_for(D.n());
    k_residual_norm<<<g, kBlock, 0, s>>>(D, diag, wx, wy, wz, b, x, r, w, partials);
    return g;
}
int launch_cg_update_xr(long long n, const double* scal, double* x, double* r, const double* p, const double* q,
                        const double* w, double* partials, cudaStream_t s) {
    const int g = grid_for(n);
    k_cg_update_xr<<<g, kBlock, 0, s>>>(n, scal, x, r, p, q, w, partials);
    return g;
}
int launch_dot2(long long n, const double* z, const double* r, const double* q, double* partials, cudaStream_t s) {
    const int g = grid_for(n);
    k_dot2<<<g, kBlock, 0, s>>>(n, z, r, q, partials);
    return g;
}
void launch_p_update(long long n, const double* scal, const double* z, double* p, cudaStream_t s) {
    k_p_update<<<grid_for(n), kBlock, 0, s>>>(n, scal, z, p);
}
template <class Tin, class Tout>
void launch_to_level(const Dims& d, int split, const Tin* a, Tout* out, const double* amax, cudaStream_t s) {
    if (split) {
        int gx, gy, gz, rows;
        rbp::pass_grid(d.nx, d.ny, d.nz, gx, gy, gz, rows);
        k_to_split<Tout><<<dim3(gx, gy, gz), rbp::kPairs, 0, s>>>(d, rows, a, out, amax);
    } else {
        k_to_level<Tin, Tout><<<grid_for(d.n()), kBlock, 0, s>>>(d, a, out, amax);
    }
}
template <class Tin, class Tout>
void launch_from_level(const Dims& d, int split, const Tin* a, Tout* out, const double* amax, cudaStream_t s) {
    if (split) {
        int gx, gy, gz, rows;
        rbp::pass_grid(d.nx, d.ny, d.nz, gx, gy, gz, rows);
        k_from_split<Tin><<<dim3(gx, gy, gz), rbp::kPairs, 0, s>>>(d, rows, a, out, amax);
    } else {
        k_from_level<Tin, Tout><<<grid_for(d.n()), kBlock, 0, s>>>(d, a, out, amax);
    }
}
template void launch_to_level<double, float>(const Dims&, int, const double*, float*, const double*, cudaStream_t);
template void launch_to_level<double, double>(const Dims&, int, const double*, double*, const double*, cudaStream_t);
template void launch_from_level<float, double>(const Dims&, int, const float*, double*, const double*, cudaStream_t);
template void launch_from_level<double, double>(const Dims&, int, const double*, double*, const double*,
                                                cudaStream_t);
void launch_copy(long long n, const double* a, double* b, cudaStream_t s) { k_copy<<<grid_for(n), kBlock, 0, s>>>(n, a, b); }
void launch_add(long long n, const double* a, double* b, cudaStream_t s) { k_add<<<grid_for(n), kBlock, 0, s>>>(n, a, b); }
void launch_cg_scalars(double* scal, const double* dots, int phase, cudaStream_t s) {
    k_cg_scalars<<<1, 32, 0, s>>>(scal, dots, phase);
}

template <class T>
void launch_mg_diag(const Dims& D, const double* diag, const double* wx, const double* wy, const double* wz, T* out,
                    cudaStream_t s) {
    k_mg_diag<T><<<grid_for(D.n()), kBlock, 0, s>>>(D, diag, wx, wy, wz, out);
}
template void launch_mg_diag<float>(const Dims&, const double*, const double*, const double*, const double*, float*,
                                    cudaStream_t);
template void launch_mg_diag<double>(const Dims&, const double*, const double*, const double*, const double*, double*,
                                     cudaStream_t);

template <class T>
void launch_coarsen(const Level<T>& f, const Level<T>& c, cudaStream_t s) {
    k_coarsen<T><<<grid_for(c.d.n()), kBlock, 0, s>>>(f, c);
}

template <class T>
void launch_split_level(const Level<T>& L, cudaStream_t s) {
    k_split_level<T><<<grid_for(L.d.n() / 2), kBlock, 0, s>>>(L);
}

template <class T>
int launch_rbgs_inplace(const Level<T>& L, int first, bool zero_guess, cudaStream_t s) {
    const Dims& d = L.d;
    for (int pass = 0; pass < 2; ++pass) {
        const int colour = pass == 0 ? first : 1 - first;
        // the second pass starts on the planes the first read last
        rbp::Pass<T> A = rbp::make_pass<T>(d.nx, d.ny, d.nz, d.per, L.w6, L.dinv, L.b, L.x, colour,
                                           pass == 0 && zero_guess, pass);
        int gx, gy, gz;
        rbp::pass_launch(A, gx, gy, gz);
        const dim3 grid(gx, gy, gz);
        if (colour == 0)
            k_rbgs_pass<0, T><<<grid, rbp::kPairs, 0, s>>>(A);
        else
            k_rbgs_pass<1, T><<<grid, rbp::kPairs, 0, s>>>(A);
    }
    return 2;
}

template <class T>
void launch_prolong_add(const Level<T>& c, const Level<T>& f, cudaStream_t s) {
    int gx, gy, gz, rows;
    rbp::pass_grid(f.d.nx, f.d.ny, f.d.nz, gx, gy, gz, rows);
    k_prolong_add<T><<<dim3(gx, gy, gz), rbp::kPairs, 0, s>>>(c, f, rows);
}

template <class T>
void launch_resid_restrict(const Level<T>& f, const Level<T>& c, cudaStream_t s) {
    int gx, gy, gz, rows;
    rbp::pass_grid(2 * c.d.nx, c.d.ny, c.d.nz, gx, gy, gz, rows);
    k_resid_restrict<T><<<dim3(gx, gy, gz), rbp::kPairs, 0, s>>>(f, c, rows);
}
template <class T>
size_t tail_smem_bytes(const Dims& d) {
    TailPlan p;
    make_plan(d, p);
    size_t cells = (size_t)p.total * 6;
    if (p.dense) cells += (size_t)kDenseMax * kDenseMax + kDenseMax;
    return cells * sizeof(T);
}
static_assert(TailMax<float>::value <= kTailCellsPerThread * kTailThreads &&
                  TailMax<double>::value <= kTailCellsPerThread * kTailThreads,
              "a tail level must fit the per-thread cells of tail_smooth");

template <class T>
int launch_tail(const Level<T>& L, int ncycles, int nu, cudaStream_t s) {
    TailPlan p;
    make_plan(L.d, p);
    const size_t bytes = tail_smem_bytes<T>(L.d);
    // the attribute is per device: set it on the first launch on each
    static bool configured[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !configured[dev]) {
        cudaFuncSetAttribute(k_tail<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (dev >= 0 && dev < 64) configured[dev] = true;
    }
    k_tail<T><<<1, kTailThreads, bytes, s>>>(L, ncycles, nu, p);
    return 1;
}

template void launch_coarsen<float>(const Level<float>&, const Level<float>&, cudaStream_t);
template void launch_coarsen<double>(const Level<double>&, const Level<double>&, cudaStream_t);
template void launch_split_level<float>(const Level<float>&, cudaStream_t);
template void launch_split_level<double>(const Level<double>&, cudaStream_t);
template int launch_rbgs_inplace<float>(const Level<float>&, int, bool, cudaStream_t);
template int launch_rbgs_inplace<double>(const Level<double>&, int, bool, cudaStream_t);
template void launch_prolong_add<float>(const Level<float>&, const Level<float>&, cudaStream_t);
template void launch_prolong_add<double>(const Level<double>&, const Level<double>&, cudaStream_t);
template void launch_resid_restrict<float>(const Level<float>&, const Level<float>&, cudaStream_t);
template void launch_resid_restrict<double>(const Level<double>&, const Level<double>&, cudaStream_t);
template int launch_tail<float>(const Level<float>&, int, int, cudaStream_t);
template int launch_tail<double>(const Level<double>&, int, int, cudaStream_t);
template size_t tail_smem_bytes<float>(const Dims&);
template size_t tail_smem_bytes<double>(const Dims&);
