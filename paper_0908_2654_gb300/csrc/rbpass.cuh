// Red-black Gauss-Seidel sweeps of a multigrid level as two in-place colour passes over a
// colour-split storage of the level, and the trilinear prolongation of a coarse correction.
//
// The level's operator is (S x)_i = diag_i x_i - sum_faces w_f x_nb.  A sweep sets every cell of
// the first colour (parity of x + y + z equal to `first`) from its neighbours, which all have the
// other colour, then every cell of the other colour from the new first-colour values.
//
// Storage (levels with even nx, ny, nz): each x-pair of cells (2p, 2p + 1) holds one cell of each
// colour, so pair m = (z ny + y) nx/2 + p indexes both colour halves: the cell of colour c of
// pair m sits at c * n/2 + m in x, b and the diagonal.  Every face joins a colour-0 cell to a
// colour-1 cell, so the 3n face couplings are stored once, as the six faces of the colour-0 cells
// (face arrays of n/2 each, in the order -x, +x, -y, +y, -z, +z).  A colour pass then streams
// contiguous arrays only: its own half of b and the diagonal, all six face arrays, the other
// colour's half of x (neighbours at pair offsets 0, +-1, +-nx/2, +-nx ny/2) and its own half of x
// written: 5 words per cell of the level per pass (the diagonal is stored inverted).  In natural order a pass over one colour moves
// every sector of b, diag, x, wx, wy, wz (half of each used) and rewrites half of x: about 7.
//
// A pass is one kernel launch with one thread per pair, a block per row segment and plane, and no
// loop, barrier or division.  The second pass takes the planes in reverse order, so that it starts
// on the planes the first pass read last (still in L2).
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
enum Face { FXM = 0, FXP = 1, FYM = 2, FYP = 3, FZM = 4, FZP = 5 };

// storage index of cell (x, y, z) in a colour-split level (even nx) or in natural order
RT_HD long long level_index(int split, int nx, int ny, int nz, int x, int y, int z) {
    const long long i = ((long long)z * ny + y) * nx + x;
    if (!split) return i;
    const long long half = (long long)nx * ny * nz / 2;
    return (long long)((x + y + z) & 1) * half + (i >> 1);
}

// two-element vector loads and stores (8 bytes for float, 16 for double): the address must be
// aligned to that size
template <class T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };
template <class T>
RT_HD void ld2(const T* p, T& a, T& b) {
    const typename Vec2<T>::type v = *reinterpret_cast<const typename Vec2<T>::type*>(p);
    a = v.x;
    b = v.y;
}
template <class T>
RT_HD void st2(T* p, T a, T b) {
    typename Vec2<T>::type v;
    v.x = a;
    v.y = b;
    *reinterpret_cast<typename Vec2<T>::type*>(p) = v;
}

// launch geometry of a pass: (blocks per row, row blocks, planes)
RT_HD void pass_grid(int nx, int ny, int nz, int& gx, int& gy, int& gz, int& rows) {
    const int hp = nx / 2;
    if (hp >= kPairs) {
        rows = 1;
        gx = (hp + kPairs - 1) / kPairs;
    } else {
        rows = kPairs / hp;
        gx = 1;
    }
    gy = (ny + rows - 1) / rows;
    gz = nz;
}

// One colour pass.  The host points each array at the half (or face array) the pass uses, so the
// kernel indexes with the pair number alone: a level holds at most 2^31 cells, so every pair
// number and neighbour pair number fits in an int.
template <class T>
struct Pass {
    int nx, ny, nz;
    int per[3];
    const T* w[6];  // face arrays of the colour-0 cells, -x, +x, -y, +y, -z, +z
    const T* dinv;  // 1 / diagonal over this colour's half
    const T* b;     // this colour's half of b
    const T* xo;    // the other colour's half of x (read)
    T* x;           // this colour's half of x (written)
    int colour;     // parity of the cells this pass sets
    int zero;       // the old iterate is zero (first pass of a sweep from zero)
    int rev;        // blocks take the planes from the last to the first
    int quad;       // each thread updates the cells of two pairs (nx a multiple of 4)
    int rows;       // rows per block: kPairs / threads per row (at least 1)
};

// launch geometry of pass A (threads per row: pairs, or pairs of pairs when A.quad); sets A.rows
template <class T>
RT_HD void pass_launch(Pass<T>& A, int& gx, int& gy, int& gz) {
    pass_grid(A.quad ? A.nx / 2 : A.nx, A.ny, A.nz, gx, gy, gz, A.rows);
}

// the pass over level arrays x, b (colour-split), dinv (colour-split) and w6 (six face arrays)
template <class T>
RT_HD Pass<T> make_pass(int nx, int ny, int nz, const int* per, const T* w6, const T* dinv, const T* b, T* x,
                        int colour, int zero, int rev) {
    Pass<T> A;
    const long long half = (long long)nx * ny * nz / 2;
    A.nx = nx;
    A.ny = ny;
    A.nz = nz;
    for (int k = 0; k < 3; ++k) A.per[k] = per[k];
    for (int f = 0; f < 6; ++f) A.w[f] = w6 + f * half;
    A.dinv = dinv + colour * half;
    A.b = b + colour * half;
    A.xo = x + (1 - colour) * half;
    A.x = x + colour * half;
    A.colour = colour;
    A.zero = zero;
    A.rev = rev;
    A.quad = nx % 4 == 0;
    int gx, gy, gz;
    pass_launch(A, gx, gy, gz);
    return A;
}

// the pair of the thread of block (bx, by, bz) and lane t in a launch of pass_grid's shape: pair
// px of row y, plane bz; returns false when it has none
RT_HD bool grid_pair(int nx, int ny, int rows, int bx, int by, int bz, int t, int& px, int& y, int& z) {
    const int hp = nx >> 1;
    int ry;
    if (rows == 1) {
        px = bx * kPairs + t;
        ry = 0;
    } else {
        ry = t / hp;
        px = t - ry * hp;
    }
    y = by * rows + ry;
    z = bz;
    return px < hp && y < ny && ry < rows;
}

// the cell of the pass's colour in the pair of block (bx, by, bz) and lane t (planes in reverse
// when A.rev); returns false when there is none
template <class T>
RT_HD bool pair_cell(const Pass<T>& A, int bx, int by, int bz, int t, int& x, int& y, int& z) {
    int px;
    if (!grid_pair(A.nx, A.ny, A.rows, bx, by, A.rev ? A.nz - 1 - bz : bz, t, px, y, z)) return false;
    x = 2 * px + ((y + z + A.colour) & 1);   // the pair's cell of this colour
    return true;
}

// the first of the two pairs of the thread of block (bx, by, bz) and lane t in a quad pass
// (planes in reverse when A.rev); returns false when there is none
template <class T>
RT_HD bool quad_pairs(const Pass<T>& A, int bx, int by, int bz, int t, int& px, int& y, int& z) {
    int pq;
    if (!grid_pair(A.nx >> 1, A.ny, A.rows, bx, by, A.rev ? A.nz - 1 - bz : bz, t, pq, y, z)) return false;
    px = 2 * pq;
    return true;
}

// neighbour pairs of cell (x, y, z) (pair m) in face order; -1 across a non-periodic boundary.
// The neighbour across face f has the other colour; for a colour-1 cell the coupling of face f
// is the opposite face (f ^ 1) of that colour-0 neighbour.
RT_HD void neighbour_pairs(int nx, int ny, int nz, const int* per, int x, int y, int z, int m, int* q) {
    const int hx = nx >> 1, hxy = hx * ny, half = hxy * nz;
    const int odd = x & 1;
    q[FXM] = odd ? m : (x > 0 ? m - 1 : (per[0] ? m - 1 + hx : -1));
    q[FXP] = !odd ? m : (x + 1 < nx ? m + 1 : (per[0] ? m + 1 - hx : -1));
    q[FYM] = y > 0 ? m - hx : (per[1] ? m - hx + hxy : -1);
    q[FYP] = y + 1 < ny ? m + hx : (per[1] ? m + hx - hxy : -1);
    q[FZM] = z > 0 ? m - hxy : (per[2] ? m - hxy + half : -1);
    q[FZP] = z + 1 < nz ? m + hxy : (per[2] ? m + hxy - half : -1);
}

// pair number of cell (x, y, z)
template <class T>
RT_HD int pair_of(const Pass<T>& A, int x, int y, int z) {
    return (z * A.ny + y) * (A.nx >> 1) + (x >> 1);
}

// new value of cell (x, y, z) of colour C from its neighbours
template <int C, class T>
RT_HD T cell_value(const Pass<T>& A, int x, int y, int z) {
    const int m = pair_of(A, x, y, z);
    RT_SWEEP_CHECK(m >= 0 && (long long)m < (long long)A.nx * A.ny * A.nz / 2);
    T num = A.b[m];
    if (!A.zero) {
        int q[6];
        neighbour_pairs(A.nx, A.ny, A.nz, A.per, x, y, z, m, q);
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            if (q[f] < 0) continue;
            RT_SWEEP_CHECK((long long)q[f] < (long long)A.nx * A.ny * A.nz / 2);
            const T w = C == 0 ? A.w[f][m] : A.w[f ^ 1][q[f]];
            num += w * A.xo[q[f]];
        }
    }
    return num * A.dinv[m];
}

// New values of the cells of colour C in pairs m and m + 1, m the pair of (2 px, y, z) with px
// even; nx a multiple of 4, so that every pair number used in a two-element access is even and
// all but the x-neighbour beyond the two pairs come in aligned pairs.  The same sums as
// cell_value for each of the two cells, with half the loads.
template <int C, class T>
RT_HD void quad_values(const Pass<T>& A, int px, int y, int z, T& v0, T& v1) {
    const int hx = A.nx >> 1, hxy = hx * A.ny, half = hxy * A.nz;
    const int m = (z * A.ny + y) * hx + px;
    RT_SWEEP_CHECK(m >= 0 && m + 1 < half && (m & 1) == 0);
    T n0, n1;
    ld2(A.b + m, n0, n1);
    if (!A.zero) {
        // y and z neighbours: pairs q, q + 1 for the two cells
        auto yz = [&](int f, int q) {
            RT_SWEEP_CHECK(q >= 0 && q + 1 < half && (q & 1) == 0);
            T x0, x1, w0, w1;
            ld2(A.xo + q, x0, x1);
            if (C == 0)
                ld2(A.w[f] + m, w0, w1);
            else
                ld2(A.w[f ^ 1] + q, w0, w1);
            n0 += w0 * x0;
            n1 += w1 * x1;
        };
        if (y > 0) yz(FYM, m - hx);
        else if (A.per[1]) yz(FYM, m - hx + hxy);
        if (y + 1 < A.ny) yz(FYP, m + hx);
        else if (A.per[1]) yz(FYP, m + hx - hxy);
        if (z > 0) yz(FZM, m - hxy);
        else if (A.per[2]) yz(FZM, m - hxy + half);
        if (z + 1 < A.nz) yz(FZP, m + hxy);
        else if (A.per[2]) yz(FZP, m + hxy - half);
        // x neighbours: the other colour at pairs m and m + 1, and at m - 1 (this colour's cells
        // at even x) or m + 2 (at odd x), which wrap on a periodic axis
        T xa, xb;
        ld2(A.xo + m, xa, xb);
        T wm0, wm1, wp0, wp1;   // face arrays -x and +x at pairs m, m + 1
        ld2(A.w[FXM] + m, wm0, wm1);
        ld2(A.w[FXP] + m, wp0, wp1);
        if (((y + z + C) & 1) == 0) {
            const int qw = px > 0 ? m - 1 : (A.per[0] ? m - 1 + hx : -1);
            if (C == 0) {
                if (qw >= 0) n0 += wm0 * A.xo[qw];
                n0 += wp0 * xa;
                n1 += wm1 * xa + wp1 * xb;
            } else {
                if (qw >= 0) n0 += A.w[FXP][qw] * A.xo[qw];
                n0 += wm0 * xa;
                n1 += wp0 * xa + wm1 * xb;
            }
        } else {
            const int qe = px + 2 < hx ? m + 2 : (A.per[0] ? m + 2 - hx : -1);
            if (C == 0) {
                n0 += wm0 * xa + wp0 * xb;
                n1 += wm1 * xb;
                if (qe >= 0) n1 += wp1 * A.xo[qe];
            } else {
                n0 += wp0 * xa + wm1 * xb;
                n1 += wp1 * xb;
                if (qe >= 0) n1 += A.w[FXM][qe] * A.xo[qe];
            }
        }
    }
    T d0, d1;
    ld2(A.dinv + m, d0, d1);
    v0 = n0 * d0;
    v1 = n1 * d1;
}

// colour-split inverse diagonal and colour-0 face arrays of pair m from the natural diagonal and
// the couplings on each cell's +x/+y/+z face (zero on a non-periodic boundary face)
template <class T>
RT_HD void split_pair(int nx, int ny, int nz, const int* per, const T* diag, const T* wx, const T* wy, const T* wz,
                      long long m, T* dinv, T* w6) {
    const long long hx = nx >> 1, half = hx * ny * nz;
    const long long r = m / hx;
    const int px = (int)(m - r * hx), y = (int)(r % ny), z = (int)(r / ny);
    const long long sy = nx, sz = (long long)nx * ny, sv = sz * nz;
    for (int o = 0; o < 2; ++o) {
        const int x = 2 * px + o;
        const long long i = 2 * m + o;
        RT_SWEEP_CHECK(i >= 0 && i < sv);
        const int c = (x + y + z) & 1;
        dinv[c * half + m] = T(1) / diag[i];
        if (c) continue;
        w6[FXM * half + m] = x > 0 ? wx[i - 1] : (per[0] ? wx[i - 1 + nx] : T(0));
        w6[FXP * half + m] = x + 1 < nx || per[0] ? wx[i] : T(0);
        w6[FYM * half + m] = y > 0 ? wy[i - sy] : (per[1] ? wy[i - sy + sz] : T(0));
        w6[FYP * half + m] = y + 1 < ny || per[1] ? wy[i] : T(0);
        w6[FZM * half + m] = z > 0 ? wz[i - sz] : (per[2] ? wz[i - sz + sv] : T(0));
        w6[FZP * half + m] = z + 1 < nz || per[2] ? wz[i] : T(0);
    }
}

// Colouring of the levels the single-CTA coarse solver sweeps, which may have odd dimensions.
// With no periodic axis of odd length it is the red-black one, (x + y + z) mod 2 (ncol = 2).  A
// periodic axis of odd length n puts cells 0 and n-1, which are neighbours, on the same parity;
// then (ncol = 3) each coordinate maps to c(v) = v mod 2, except c(n-1) = 2 on such an axis, and
// the colour is (c(x) + c(y) + c(z)) mod 3: neighbours differ in one coordinate, whose c differs
// by 1 or 2, so no two neighbours share a colour.
RT_HD bool odd_periodic(int nx, int ny, int nz, const int* per) {
    return (per[0] && (nx & 1)) || (per[1] && (ny & 1)) || (per[2] && (nz & 1));
}
RT_HD int multicolour(int nx, int ny, int nz, const int* per, int ncol, int x, int y, int z) {
    if (ncol == 2) return (x + y + z) & 1;
    auto c = [](int v, int n, int p) { return (p && (n & 1) && v == n - 1) ? 2 : (v & 1); };
    return (c(x, nx, per[0]) + c(y, ny, per[1]) + c(z, nz, per[2])) % 3;
}

// coarse-cell value of the trilinear cell-centred prolongation at fine cell (x, y, z): weights
// 3/4 and 1/4 along each axis from the coarse cell holding the fine cell and its neighbour on the
// fine cell's side (the cell itself at a non-periodic edge); xc colour-split when csplit
template <class T>
RT_HD T prolong_at(const T* xc, int csplit, int cnx, int cny, int cnz, const int* per, int x, int y, int z) {
    const int X = x >> 1, Y = y >> 1, Z = z >> 1;
    auto other = [](int C, int odd, int n, int p) {
        const int c = odd ? C + 1 : C - 1;
        if (c >= 0 && c < n) return c;
        return p ? (c + n) % n : C;
    };
    const int X2 = other(X, x & 1, cnx, per[0]);
    const int Y2 = other(Y, y & 1, cny, per[1]);
    const int Z2 = other(Z, z & 1, cnz, per[2]);
    auto C = [&](int a, int b, int e) {
        const long long j = level_index(csplit, cnx, cny, cnz, a, b, e);
        RT_SWEEP_CHECK(j >= 0 && j < (long long)cnx * cny * cnz);
        return xc[j];
    };
    const T w1 = T(0.75), w2 = T(0.25);
    const T v1 = w1 * (w1 * C(X, Y, Z) + w2 * C(X2, Y, Z)) + w2 * (w1 * C(X, Y2, Z) + w2 * C(X2, Y2, Z));
    const T v2 = w1 * (w1 * C(X, Y, Z2) + w2 * C(X2, Y, Z2)) + w2 * (w1 * C(X, Y2, Z2) + w2 * C(X2, Y2, Z2));
    return w1 * v1 + w2 * v2;
}

// prolong_at for both cells of fine pair (2 px, 2 px + 1), which lie in coarse cell px and take
// their x-neighbour from coarse cells px - 1 and px + 1: twelve coarse values instead of sixteen
template <class T>
RT_HD void prolong_pair(const T* xc, int csplit, int cnx, int cny, int cnz, const int* per, int px, int y, int z,
                        T& v0, T& v1) {
    const int Y = y >> 1, Z = z >> 1;
    auto other = [](int C, int odd, int n, int p) {
        const int c = odd ? C + 1 : C - 1;
        if (c >= 0 && c < n) return c;
        return p ? (c < 0 ? c + n : c - n) : C;
    };
    const int Xm = other(px, 0, cnx, per[0]), Xp = other(px, 1, cnx, per[0]);
    const int Y2 = other(Y, y & 1, cny, per[1]);
    const int Z2 = other(Z, z & 1, cnz, per[2]);
    // the four coarse rows (Y or Y2, Z or Z2): row start and the parity of Y + Z; a coarse level
    // holds at most 2^30 cells, so the indices are 32-bit
    const int halfc = csplit ? cnx * cny * cnz / 2 : 0;
    const int r00 = (Z * cny + Y) * cnx, r10 = (Z * cny + Y2) * cnx;
    const int r01 = (Z2 * cny + Y) * cnx, r11 = (Z2 * cny + Y2) * cnx;
    const int p00 = (Y + Z) & 1, p10 = (Y2 + Z) & 1, p01 = (Y + Z2) & 1, p11 = (Y2 + Z2) & 1;
    auto C = [&](int row, int par, int a) {
        const int j = csplit ? ((a + par) & 1) * halfc + ((row + a) >> 1) : row + a;
        RT_SWEEP_CHECK(j >= 0 && (long long)j < (long long)cnx * cny * cnz);
        return xc[j];
    };
    const T w1 = T(0.75), w2 = T(0.25);
    // y-z weighted columns at coarse x = px - 1, px, px + 1
    auto col = [&](int a) {
        return w1 * (w1 * C(r00, p00, a) + w2 * C(r10, p10, a)) + w2 * (w1 * C(r01, p01, a) + w2 * C(r11, p11, a));
    };
    const T cm = col(Xm), c0 = col(px), cp = col(Xp);
    v0 = w1 * c0 + w2 * cm;
    v1 = w1 * c0 + w2 * cp;
}

// b - S x at the two cells of fine pair m = (z ny + y) nx/2 + px of a colour-split level (x, b
// colour-split; the operator in natural order: diag and the +x/+y/+z face couplings, zero on a
// non-periodic boundary face): rE for the even-x cell, rO for the odd one.  The even cell has
// colour (y + z) mod 2; the neighbours of each cell are in the other colour's half.
template <class T>
RT_HD void pair_residuals(int nx, int ny, int nz, const int* per, const T* diag, const T* wx, const T* wy,
                          const T* wz, const T* b, const T* x, int px, int y, int z, T& rE, T& rO) {
    const int hx = nx >> 1, hxy = hx * ny, half = hxy * nz, plane = nx * ny;
    const int m = (z * ny + y) * hx + px;
    const int ce = (y + z) & 1;
    const T* xe = x + ce * half;         // this row's even cells and the odd cells of the rows above/below
    const T* xo = x + (1 - ce) * half;   // this row's odd cells and the even cells of the rows above/below
    const int i = 2 * m;                 // natural index of the even cell
    RT_SWEEP_CHECK(m >= 0 && m < half);
    T dE, dO, wE, wO;
    ld2(diag + i, dE, dO);
    ld2(wx + i, wE, wO);                 // the face between the two cells, and the odd cell's +x face
    const T vE = xe[m], vO = xo[m];
    T sE = wE * vO, sO = wE * vE;
    if (px > 0) sE += wx[i - 1] * xo[m - 1];
    else if (per[0]) sE += wx[i - 1 + nx] * xo[m - 1 + hx];
    if (px + 1 < hx) sO += wO * xe[m + 1];
    else if (per[0]) sO += wO * xe[m + 1 - hx];
    // y and z faces: the neighbour pair q, the couplings of the two cells at natural index j, j + 1
    auto face = [&](const T* w, int j, int q) {
        RT_SWEEP_CHECK(q >= 0 && q < half && j >= 0 && j + 1 < 2 * half);
        T w0, w1;
        ld2(w + j, w0, w1);
        sE += w0 * xo[q];
        sO += w1 * xe[q];
    };
    if (y + 1 < ny) face(wy, i, m + hx);
    else if (per[1]) face(wy, i, m + hx - hxy);
    if (y > 0) face(wy, i - nx, m - hx);
    else if (per[1]) face(wy, i - nx + plane, m - hx + hxy);
    if (z + 1 < nz) face(wz, i, m + hxy);
    else if (per[2]) face(wz, i, m + hxy - half);
    if (z > 0) face(wz, i - plane, m - hxy);
    else if (per[2]) face(wz, i - plane + 2 * half, m - hxy + half);
    rE = b[ce * half + m] - (dE * vE - sE);
    rO = b[(1 - ce) * half + m] - (dO * vO - sO);
}

}  // namespace rbp
