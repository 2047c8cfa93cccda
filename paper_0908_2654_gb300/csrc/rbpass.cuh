// Red-black Gauss-Seidel sweeps of a multigrid level as two in-place colour passes, and the
// trilinear prolongation of a coarse correction.
//
// The level's operator is (S x)_i = diag_i x_i - sum_faces w_f x_nb (w on each cell's +x/+y/+z
// face, zero on boundary faces).  A sweep sets every cell of the first colour (parity of x + y + z
// equal to `first`) from its neighbours, which all have the other colour, then every cell of the
// other colour from the new first-colour values, both in place.
//
// A pass is one kernel launch with one thread per pair of x-neighbours (one cell of each colour),
// a block per row segment and plane, and no loop, barrier or division: all SM resources go to
// keeping loads in flight.  The second pass takes the planes in reverse order, so that it starts
// on the planes the first pass read last (still in L2), and the next sweep's first pass starts on
// the planes this second pass read last.
//
// The functions are host/device so that a host build can run the passes and compare them with a
// plain sweep (tests/host/smoother_host.cu).
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
    int planes;     // planes of the pass
    int rev;        // blocks take the planes from the last to the first
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
    z = A.z0 + (A.rev ? A.planes - 1 - bz : bz);
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

// coarse-cell value of the trilinear cell-centred prolongation at fine cell (x, y, z): weights
// 3/4 and 1/4 along each axis from the coarse cell holding the fine cell and its neighbour on the
// fine cell's side (the cell itself at a non-periodic edge)
template <class T>
RT_HD T prolong_at(const T* xc, int cnx, int cny, int cnz, const int* per, int x, int y, int z) {
    const int X = x >> 1, Y = y >> 1, Z = z >> 1;
    auto other = [](int C, int odd, int n, int p) {
        const int c = odd ? C + 1 : C - 1;
        if (c >= 0 && c < n) return c;
        return p ? (c + n) % n : C;
    };
    const int X2 = other(X, x & 1, cnx, per[0]);
    const int Y2 = other(Y, y & 1, cny, per[1]);
    const int Z2 = other(Z, z & 1, cnz, per[2]);
    const long long sy = cnx, sz = (long long)cnx * cny;
    auto C = [&](int a, int b, int e) {
        const long long j = (long long)e * sz + (long long)b * sy + a;
        RT_SWEEP_CHECK(j >= 0 && j < sz * cnz);
        return xc[j];
    };
    const T w1 = T(0.75), w2 = T(0.25);
    const T v1 = w1 * (w1 * C(X, Y, Z) + w2 * C(X2, Y, Z)) + w2 * (w1 * C(X, Y2, Z) + w2 * C(X2, Y2, Z));
    const T v2 = w1 * (w1 * C(X, Y, Z2) + w2 * C(X2, Y, Z2)) + w2 * (w1 * C(X, Y2, Z2) + w2 * C(X2, Y2, Z2));
    return w1 * v1 + w2 * v2;
}

}  // namespace rbp
