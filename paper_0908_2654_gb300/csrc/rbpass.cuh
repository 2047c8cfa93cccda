// Red-black Gauss-Seidel sweeps of a multigrid level as in-place colour passes, launched slab by
// slab so that the second pass over a slab finds the slab's arrays in L2.
//
// The level's operator is (S x)_i = diag_i x_i - sum_faces w_f x_nb (w on each cell's +x/+y/+z
// face, zero on boundary faces).  A sweep sets every cell of the first colour (parity of x + y + z
// equal to `first`) from its neighbours, which all have the other colour, then every cell of the
// other colour from the new first-colour values, both in place.
//
// A pass over the planes [z0, z1) is one kernel launch with one thread per pair of x-neighbours
// (one cell of each colour), a block per row segment and plane, and no loop, barrier or
// division.  Levels larger than a slab of planes are swept in the launch order
//     R0, R1, B0, R2, B1, ..., R(K-1), B(K-2), B(K-1)        (periodic z: B0 moved to the end)
// where Rk / Bk is the first / second colour pass over slab k: the second pass over slab k runs
// after the first passes over slabs k - 1, k and k + 1 (the stream orders launches), and right
// after the first pass over slab k + 1, while the slab's arrays are still in L2.  One sweep then
// moves about 7 words per cell through HBM (b, diag, wx, wy, wz and x read, x written).
//
// The functions are host/device so that a host build can run the passes in the same order and
// compare them with a plain sweep (tests/host/smoother_host.cu).
#pragma once
#include <cuda_runtime.h>

#ifndef RT_HD
#define RT_HD __host__ __device__ __forceinline__
#endif
#ifndef RT_SWEEP_CHECK
#define RT_SWEEP_CHECK(cond) ((void)0)
#endif

namespace rbp {

constexpr int kPairs = 128;   // threads (pairs) per block

template <class T>
struct Pass {
    int nx, ny, nz;
    int per[3];
    const T* diag;
    const T* wx;
    const T* wy;
    const T* wz;
    const T* b;
    T* x;
    int colour;     // parity of the cells this pass sets
    int zero;       // the old iterate is zero (first pass of a sweep from zero)
    int z0;         // first plane of the pass
    int rows;       // rows per block: kPairs / pairs per row (at least 1)
};

// the thread of block (bx, by, bz) and lane t: pair px of row y, plane z; returns false when
// it has no cell
template <class T>
RT_HD bool pair_cell(const Pass<T>& A, int bx, int by, int bz, int t, int& x, int& y, int& z) {
    const int hp = (A.nx + 1) >> 1;
    int px, ry;
    if (A.rows == 1) {
        px = bx * kPairs + t;
        ry = 0;
    } else {
        ry = t / hp;
        px = t - ry * hp;
    }
    y = by * A.rows + ry;
    z = A.z0 + bz;
    if (px >= hp || y >= A.ny || ry >= A.rows) return false;
    x = 2 * px + ((y + z + A.colour) & 1);   // the pair's cell of this colour
    return x < A.nx;
}

// new value of cell (x, y, z) from its neighbours
template <class T>
RT_HD T cell_value(const Pass<T>& A, int x, int y, int z) {
    const long long sy = A.nx, sz = (long long)A.nx * A.ny;
    const long long i = (long long)z * sz + (long long)y * sy + x;
    RT_SWEEP_CHECK(i >= 0 && i < sz * A.nz);
    T num = A.b[i];
    if (!A.zero) {
        if (x + 1 < A.nx) num += A.wx[i] * A.x[i + 1];
        else if (A.per[0]) num += A.wx[i] * A.x[i + 1 - A.nx];
        if (x > 0) num += A.wx[i - 1] * A.x[i - 1];
        else if (A.per[0]) num += A.wx[i - 1 + A.nx] * A.x[i - 1 + A.nx];
        if (y + 1 < A.ny) num += A.wy[i] * A.x[i + sy];
        else if (A.per[1]) num += A.wy[i] * A.x[i + sy - sz];
        if (y > 0) num += A.wy[i - sy] * A.x[i - sy];
        else if (A.per[1]) num += A.wy[i - sy + sz] * A.x[i - sy + sz];
        const long long sv = sz * A.nz;
        if (z + 1 < A.nz) num += A.wz[i] * A.x[i + sz];
        else if (A.per[2]) num += A.wz[i] * A.x[i + sz - sv];
        if (z > 0) num += A.wz[i - sz] * A.x[i - sz];
        else if (A.per[2]) num += A.wz[i - sz + sv] * A.x[i - sz + sv];
    }
    return num / A.diag[i];
}

// launch geometry of a pass over `planes` planes: (blocks per row, row blocks, planes)
inline void pass_grid(int nx, int ny, int planes, int& gx, int& gy, int& gz, int& rows) {
    const int hp = (nx + 1) / 2;
    if (hp >= kPairs) {
        rows = 1;
        gx = (hp + kPairs - 1) / kPairs;
    } else {
        rows = kPairs / hp;
        gx = 1;
    }
    gy = (ny + rows - 1) / rows;
    gz = planes;
}

// slabs of a level: planes per slab so that a slab of the seven arrays stays well inside L2
// (about 40 MB); a level that fits is one slab
inline int slab_planes(int nx, int ny, int nz, int bytes_per_value, double l2_budget = 40e6) {
    const double plane = 7.0 * bytes_per_value * (double)nx * ny;
    int s = (int)(l2_budget / plane);
    if (s < 2) s = 2;
    if (s >= nz) return nz;
    return s;
}

// launch j of a sweep with K slabs -> (slab, colour pass: 0 first, 1 second); 2K launches
inline void launch_of(int K, int per_z, int j, int& slab, int& pass) {
    if (j == 0) {
        slab = 0;
        pass = 0;
        return;
    }
    if (j == 2 * K - 1) {
        slab = per_z ? 0 : K - 1;
        pass = 1;
        return;
    }
    if (!per_z) {
        const int m = j - 1;
        slab = (m % 2 == 0) ? m / 2 + 1 : (m - 1) / 2;
        pass = m % 2;
        return;
    }
    if (j == 1) {
        slab = 1;
        pass = 0;
        return;
    }
    if (j == 2 * K - 2) {
        slab = K - 1;
        pass = 1;
        return;
    }
    const int m = j - 2;
    slab = (m % 2 == 0) ? m / 2 + 2 : (m - 1) / 2 + 1;
    pass = m % 2;
}

}  // namespace rbp
