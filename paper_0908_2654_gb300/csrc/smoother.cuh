// One red-black Gauss-Seidel sweep of a multigrid level in a single pass over HBM.
//
// The level's operator is (S x)_i = diag_i x_i - sum_faces w_f x_nb (w on each cell's +x/+y/+z
// face, zero on boundary faces).  A sweep updates the cells of the first colour (parity of
// x + y + z equal to `first`) from the old values of the other colour, then the other colour
// from the new values of the first.  The first colour's old values are never read, so the sweep
// is a function of the old second-colour values alone.
//
// Layout of the work: a CTA owns a TX x TY column of cells and marches through a chunk of z
// planes.  Per plane it stages, in shared memory, the old iterate and the five coefficient
// arrays over the column plus a two-cell halo in x and y, computes the first colour on the
// column plus a one-cell halo (the halo values are recomputed locally instead of being read from
// the neighbouring CTA), and one plane behind that the second colour on the column.  The old
// iterate is read from one buffer and the result written to another, so the sweep is exactly
// the red-black Gauss-Seidel sweep and does not depend on the order in which CTAs run.  Every
// array is read once per sweep (plus the halo, mostly from L2) and x is written once: the
// 7 words per cell of a sweep.
//
// Optionally the old iterate is the fine level's x plus the trilinear prolongation of a coarse
// correction (the V-cycle's coarse-grid correction fused into the first post-smoothing sweep).
//
// The phases are host/device functions over an explicit (thread, thread count) pair, so that a
// host build can run a CTA's phases one after another and compare the sweep with a plain
// Gauss-Seidel sweep (tests/host/smoother_host.cu).
#pragma once
#include <cuda_runtime.h>

#ifndef RT_HD
#define RT_HD __host__ __device__ __forceinline__
#endif

#ifndef RT_SWEEP_CHECK
#define RT_SWEEP_CHECK(cond) ((void)0)
#endif

namespace sweep {

constexpr int TX = 32, TY = 16, HALO = 2;
constexpr int PX = TX + 2 * HALO, PY = TY + 2 * HALO;   // staged plane: column plus halo
constexpr int PLANE = PX * PY;
constexpr int XR = 3, RR = 3, CR = 4;                   // ring depths: old x, first colour, coefficients
constexpr int kThreads = 256;

struct Geo {
    int nx, ny, nz;
    int per[3];
};

template <class T>
struct Args {
    Geo d;
    const T* diag;
    const T* wx;
    const T* wy;
    const T* wz;
    const T* b;
    const T* xin;      // old iterate (unused when zero_guess)
    T* xout;           // new iterate (must not alias xin)
    int first;         // colour updated first
    int zero_guess;    // old iterate = 0
    int zc;            // z planes per CTA chunk
    // fused coarse-grid correction: old iterate = xin + P xc (xc null: none)
    const T* xc;
    Geo cd;
};

template <class T>
struct Tile {
    T xo[XR][PLANE];   // old iterate
    T rd[RR][PLANE];   // first-colour values
    T cb[CR][PLANE];   // b
    T cg[CR][PLANE];   // diag
    T cx[CR][PLANE];   // wx
    T cy[CR][PLANE];   // wy
    T cz[CR][PLANE];   // wz
};

RT_HD int ring(int p, int n) { return ((p % n) + n) % n; }

// global coordinate along an axis for local coordinate c of a tile starting at c0: the wrapped
// index, or -1 outside a non-periodic axis
RT_HD int gcoord(int c, int n, int per) {
    if (c >= 0 && c < n) return c;
    if (!per) return -1;
    return ((c % n) + n) % n;
}

// coarse cell value of the trilinear cell-centred prolongation at fine cell (x, y, z)
template <class T>
RT_HD T prolong_at(const Args<T>& A, int x, int y, int z) {
    const Geo& cd = A.cd;
    const int X = x >> 1, Y = y >> 1, Z = z >> 1;
    // the other coarse cell of the stencil along each axis; at a non-periodic edge the cell itself
    auto other = [](int C, int odd, int n, int per) {
        const int c = odd ? C + 1 : C - 1;
        if (c >= 0 && c < n) return c;
        return per ? (c + n) % n : C;
    };
    const int X2 = other(X, x & 1, cd.nx, cd.per[0]);
    const int Y2 = other(Y, y & 1, cd.ny, cd.per[1]);
    const int Z2 = other(Z, z & 1, cd.nz, cd.per[2]);
    const long long sy = cd.nx, sz = (long long)cd.nx * cd.ny;
    auto C = [&](int a, int b, int e) {
        const long long j = (long long)e * sz + (long long)b * sy + a;
        RT_SWEEP_CHECK(j >= 0 && j < sz * cd.nz);
        return A.xc[j];
    };
    const T w1 = T(0.75), w2 = T(0.25);
    const T v1 = w1 * (w1 * C(X, Y, Z) + w2 * C(X2, Y, Z)) + w2 * (w1 * C(X, Y2, Z) + w2 * C(X2, Y2, Z));
    const T v2 = w1 * (w1 * C(X, Y, Z2) + w2 * C(X2, Y, Z2)) + w2 * (w1 * C(X, Y2, Z2) + w2 * C(X2, Y2, Z2));
    return w1 * v1 + w2 * v2;
}

// stage plane p (old iterate and coefficients over the column plus halo)
template <class T>
RT_HD void load(const Args<T>& A, Tile<T>& S, int X0, int Y0, int p, int tid, int nth) {
    const Geo& d = A.d;
    const int gz = gcoord(p, d.nz, d.per[2]);
    const int xs = ring(p, XR), cs = ring(p, CR);
    const long long sy = d.nx, sz = (long long)d.nx * d.ny;
    for (int k = tid; k < PLANE; k += nth) {
        const int lx = k % PX - HALO, ly = k / PX - HALO;
        const int gx = gcoord(X0 + lx, d.nx, d.per[0]);
        const int gy = gcoord(Y0 + ly, d.ny, d.per[1]);
        T xo = T(0), b = T(0), dg = T(0), wx = T(0), wy = T(0), wz = T(0);
        if (gx >= 0 && gy >= 0 && gz >= 0) {
            const long long i = (long long)gz * sz + (long long)gy * sy + gx;
            RT_SWEEP_CHECK(i >= 0 && i < sz * d.nz);
            b = A.b[i];
            dg = A.diag[i];
            wx = A.wx[i];
            wy = A.wy[i];
            wz = A.wz[i];
            if (!A.zero_guess) {
                xo = A.xin[i];
                if (A.xc) xo += prolong_at(A, gx, gy, gz);
            }
        }
        S.xo[xs][k] = xo;
        S.cb[cs][k] = b;
        S.cg[cs][k] = dg;
        S.cx[cs][k] = wx;
        S.cy[cs][k] = wy;
        S.cz[cs][k] = wz;
    }
}

// colour of the cell at local (lx, ly) on plane p, or -1 when it lies outside the grid
RT_HD int colour(const Geo& d, int X0, int Y0, int lx, int ly, int p) {
    const int gx = gcoord(X0 + lx, d.nx, d.per[0]);
    const int gy = gcoord(Y0 + ly, d.ny, d.per[1]);
    const int gz = gcoord(p, d.nz, d.per[2]);
    if (gx < 0 || gy < 0 || gz < 0) return -1;
    return (gx + gy + gz) & 1;
}

// first colour on plane q over the column plus a one-cell halo; its column cells of planes
// z0 <= q < z1 are written out
template <class T>
RT_HD void first_colour(const Args<T>& A, Tile<T>& S, int X0, int Y0, int q, int z0, int z1, int tid, int nth) {
    const Geo& d = A.d;
    const int rs = ring(q, RR), cs = ring(q, CR), cm = ring(q - 1, CR);
    const int xs = ring(q, XR), xm = ring(q - 1, XR), xp = ring(q + 1, XR);
    const long long sy = d.nx, sz = (long long)d.nx * d.ny;
    constexpr int W1 = TX + 2, H1 = TY + 2;
    for (int k = tid; k < W1 * H1; k += nth) {
        const int lx = k % W1 - 1, ly = k / W1 - 1;
        const int c = (ly + HALO) * PX + (lx + HALO);
        T v = T(0);
        if (colour(d, X0, Y0, lx, ly, q) == A.first) {
            T num = S.cb[cs][c];
            if (!A.zero_guess) {
                num += S.cx[cs][c] * S.xo[xs][c + 1] + S.cx[cs][c - 1] * S.xo[xs][c - 1] +
                       S.cy[cs][c] * S.xo[xs][c + PX] + S.cy[cs][c - PX] * S.xo[xs][c - PX] +
                       S.cz[cs][c] * S.xo[xp][c] + S.cz[cm][c] * S.xo[xm][c];
            }
            v = num / S.cg[cs][c];
            if (q >= z0 && q < z1 && lx >= 0 && lx < TX && ly >= 0 && ly < TY && X0 + lx < d.nx &&
                Y0 + ly < d.ny) {
                const long long i = (long long)q * sz + (long long)(Y0 + ly) * sy + (X0 + lx);
                RT_SWEEP_CHECK(i >= 0 && i < sz * d.nz);
                A.xout[i] = v;
            }
        }
        S.rd[rs][c] = v;
    }
}

// second colour on plane q (z0 <= q < z1) over the column, from the first colour's new values
template <class T>
RT_HD void second_colour(const Args<T>& A, Tile<T>& S, int X0, int Y0, int q, int tid, int nth) {
    const Geo& d = A.d;
    const int rs = ring(q, RR), rm = ring(q - 1, RR), rp = ring(q + 1, RR);
    const int cs = ring(q, CR), cm = ring(q - 1, CR);
    const long long sy = d.nx, sz = (long long)d.nx * d.ny;
    for (int k = tid; k < TX * TY; k += nth) {
        const int lx = k % TX, ly = k / TX;
        if (X0 + lx >= d.nx || Y0 + ly >= d.ny) continue;
        if (colour(d, X0, Y0, lx, ly, q) != 1 - A.first) continue;
        const int c = (ly + HALO) * PX + (lx + HALO);
        const T num = S.cb[cs][c] + S.cx[cs][c] * S.rd[rs][c + 1] + S.cx[cs][c - 1] * S.rd[rs][c - 1] +
                      S.cy[cs][c] * S.rd[rs][c + PX] + S.cy[cs][c - PX] * S.rd[rs][c - PX] +
                      S.cz[cs][c] * S.rd[rp][c] + S.cz[cm][c] * S.rd[rm][c];
        const long long i = (long long)q * sz + (long long)(Y0 + ly) * sy + (X0 + lx);
        RT_SWEEP_CHECK(i >= 0 && i < sz * d.nz);
        A.xout[i] = num / S.cg[cs][c];
    }
}

// z planes per chunk for a level: enough CTAs to cover the SMs about four times over, chunks of
// at least four planes
inline int chunk_planes(const Geo& d, int nsm) {
    const long long cols = (long long)((d.nx + TX - 1) / TX) * ((d.ny + TY - 1) / TY);
    long long chunks = (4LL * nsm + cols - 1) / cols;
    if (chunks < 1) chunks = 1;
    int zc = (int)((d.nz + chunks - 1) / chunks);
    if (zc < 4) zc = 4;
    if (zc > d.nz) zc = d.nz;
    return zc;
}

}  // namespace sweep
