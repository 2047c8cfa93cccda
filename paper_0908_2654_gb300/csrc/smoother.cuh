// One red-black Gauss-Seidel sweep of a multigrid level in a single pass over HBM.
//
// The level's operator is (S x)_i = diag_i x_i - sum_faces w_f x_nb (w on each cell's +x/+y/+z
// face, zero on boundary faces).  A sweep updates the cells of the first colour (parity of
// x + y + z equal to `first`) from the old values of the other colour, then the other colour
// from the new values of the first.  The first colour's old values are never read, so the sweep
// is a function of the old second-colour values alone.
//
// Layout of the work: a work item is a TX x TY column of cells over a chunk of z planes; a CTA
// takes items in turn and marches through the chunk plane by plane.  Per plane it stages, in
// shared memory, the old iterate and the five coefficient arrays over the column plus a two-cell
// halo in x and y, computes the first colour on the column plus a one-cell halo (the halo values
// are recomputed locally instead of being read from the neighbouring CTA) and stores it in place
// of the old values of those cells, and one plane behind that computes the second colour on the
// column.  The loads of the next plane are issued into registers before the compute phases of
// the current one, so their latency overlaps the arithmetic.  The old iterate is read from one
// buffer and the result written to another, so the sweep is exactly the red-black Gauss-Seidel
// sweep and does not depend on the order in which CTAs run.  Every array is read once per sweep
// (plus the halo, mostly from L2) and x is written once: the 7 words per cell of a sweep.
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

constexpr int TX = 32, TY = 8, HALO = 2;
constexpr int PX = TX + 2 * HALO, PY = TY + 2 * HALO;   // staged plane: column plus halo
constexpr int PLANE = PX * PY;
constexpr int kThreads = 256;
constexpr int PER_THREAD = (PLANE + kThreads - 1) / kThreads;   // staged positions per thread
// ring depths, in planes: x holds p-3..p (the second colour of p-2 reads the first colour of
// p-3..p-1), b/diag/wx/wy hold p-2..p, wz holds p-3..p (the -z face of plane p-2)
constexpr int XR = 4, CR = 3, ZR = 4;

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
    int zc;            // z planes per work item
    // fused coarse-grid correction: old iterate = xin + P xc (xc null: none)
    const T* xc;
    Geo cd;
};

template <class T>
struct Tile {
    T x[XR][PLANE];    // old iterate; first-colour cells overwritten with their new values
    T b[CR][PLANE];
    T dg[CR][PLANE];
    T wx[CR][PLANE];
    T wy[CR][PLANE];
    T wz[ZR][PLANE];
};

// one thread's share of a staged plane, held in registers between its load and its store
template <class T>
struct Fetch {
    T x[PER_THREAD], b[PER_THREAD], dg[PER_THREAD], wx[PER_THREAD], wy[PER_THREAD], wz[PER_THREAD];
};

RT_HD int ring(int p, int n) { return ((p % n) + n) % n; }

// global coordinate along an axis: the wrapped index, or -1 outside a non-periodic axis
RT_HD int gcoord(int c, int n, int per) {
    if (c >= 0 && c < n) return c;
    if (!per) return -1;
    return ((c % n) + n) % n;
}

// number of work items and their layout: columns of TX x TY cells times chunks of zc planes
RT_HD int columns_x(const Geo& d) { return (d.nx + TX - 1) / TX; }
RT_HD int columns_y(const Geo& d) { return (d.ny + TY - 1) / TY; }
RT_HD int chunks(const Geo& d, int zc) { return (d.nz + zc - 1) / zc; }
RT_HD long long items(const Geo& d, int zc) { return (long long)columns_x(d) * columns_y(d) * chunks(d, zc); }

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

// Per-thread addressing of a work item, fixed for all its planes: the in-plane offsets of the
// thread's staged positions (-1 outside a non-periodic edge) and of its first- and second-colour
// pairs.  A pair is two x-neighbours starting at an odd (first colour, column plus halo) or even
// (second colour, column) local x; exactly one of them has each colour, so every thread of a
// colour phase updates one cell and no lane waits on a colour test.
constexpr int P1 = (TX + 2) / 2 * (TY + 2);   // first-colour pairs: 17 x 10 for 32 x 8
constexpr int P2 = TX / 2 * TY;               // second-colour pairs: 16 x 8
static_assert(P1 <= kThreads && P2 <= kThreads, "one pair per thread");

struct Item {
    int X0, Y0, z0, z1;
    int off[PER_THREAD];         // staged position: gy * nx + gx, or -1 (a plane holds < 2^31 cells)
    // first-colour pair: shared-memory index of its left cell, whether each cell lies in the grid,
    // the left cell's parity (gx + gy) & 1, whether each is a column cell to write out, and the
    // left cell's in-plane offset
    int c1;
    bool in1[2];
    int par1;
    bool w1[2];
    int o1;
    // second-colour pair (always column cells)
    int c2;
    bool in2[2];
    int par2;
    int o2;
};

template <class T>
RT_HD void item_setup(const Args<T>& A, long long it, int tid, Item& I) {
    const Geo& d = A.d;
    const int cx = columns_x(d), cy = columns_y(d);
    const long long col = it % ((long long)cx * cy);
    const int ch = (int)(it / ((long long)cx * cy));
    I.X0 = (int)(col % cx) * TX;
    I.Y0 = (int)(col / cx) * TY;
    I.z0 = ch * A.zc;
    I.z1 = I.z0 + A.zc < d.nz ? I.z0 + A.zc : d.nz;
#pragma unroll
    for (int j = 0; j < PER_THREAD; ++j) {
        const int k = tid + j * kThreads;
        I.off[j] = -1;
        if (k < PLANE) {
            const int gx = gcoord(I.X0 + k % PX - HALO, d.nx, d.per[0]);
            const int gy = gcoord(I.Y0 + k / PX - HALO, d.ny, d.per[1]);
            if (gx >= 0 && gy >= 0) I.off[j] = gy * d.nx + gx;
        }
    }
    I.c1 = -1;
    if (tid < P1) {
        const int lx = -1 + 2 * (tid % ((TX + 2) / 2)), ly = -1 + tid / ((TX + 2) / 2);
        const int gy = gcoord(I.Y0 + ly, d.ny, d.per[1]);
        const int g0 = gcoord(I.X0 + lx, d.nx, d.per[0]), g1 = gcoord(I.X0 + lx + 1, d.nx, d.per[0]);
        I.c1 = (ly + HALO) * PX + (lx + HALO);
        I.in1[0] = gy >= 0 && g0 >= 0;
        I.in1[1] = gy >= 0 && g1 >= 0;
        // parity of the left cell; the right one has the other parity (even dimensions)
        I.par1 = I.in1[0] ? (g0 + gy) & 1 : (I.in1[1] ? (g1 + gy + 1) & 1 : 0);
        const bool row = ly >= 0 && ly < TY && I.Y0 + ly < d.ny;
        I.w1[0] = row && lx >= 0 && I.X0 + lx < d.nx;
        I.w1[1] = row && lx + 1 < TX && I.X0 + lx + 1 < d.nx;
        I.o1 = (I.Y0 + ly) * d.nx + (I.X0 + lx);
    }
    I.c2 = -1;
    if (tid < P2) {
        const int lx = 2 * (tid % (TX / 2)), ly = tid / (TX / 2);
        I.c2 = (ly + HALO) * PX + (lx + HALO);
        const bool row = I.Y0 + ly < d.ny;
        I.in2[0] = row && I.X0 + lx < d.nx;
        I.in2[1] = row && I.X0 + lx + 1 < d.nx;
        I.par2 = (I.X0 + lx + I.Y0 + ly) & 1;
        I.o2 = (I.Y0 + ly) * d.nx + (I.X0 + lx);
    }
}

// load this thread's share of plane p (old iterate and coefficients over the column plus halo)
template <class T>
RT_HD void fetch(const Args<T>& A, const Item& I, int p, Fetch<T>& F) {
    const Geo& d = A.d;
    const int gz = gcoord(p, d.nz, d.per[2]);
    const long long plane = (long long)gz * d.nx * d.ny;
#pragma unroll
    for (int j = 0; j < PER_THREAD; ++j) {
        T xo = T(0), b = T(0), dg = T(0), wx = T(0), wy = T(0), wz = T(0);
        if (I.off[j] >= 0 && gz >= 0) {
            const long long i = plane + I.off[j];
            RT_SWEEP_CHECK(i >= 0 && i < (long long)d.nx * d.ny * d.nz);
            b = A.b[i];
            dg = A.diag[i];
            wx = A.wx[i];
            wy = A.wy[i];
            wz = A.wz[i];
            if (!A.zero_guess) {
                xo = A.xin[i];
                if (A.xc) {
                    const int r = I.off[j] / d.nx;
                    xo += prolong_at(A, I.off[j] - r * d.nx, r, gz);
                }
            }
        }
        F.x[j] = xo;
        F.b[j] = b;
        F.dg[j] = dg;
        F.wx[j] = wx;
        F.wy[j] = wy;
        F.wz[j] = wz;
    }
}

// store this thread's share of plane p into the rings
template <class T>
RT_HD void stage(Tile<T>& S, int p, int tid, const Fetch<T>& F) {
    const int xs = ring(p, XR), cs = ring(p, CR), zs = ring(p, ZR);
#pragma unroll
    for (int j = 0; j < PER_THREAD; ++j) {
        const int k = tid + j * kThreads;
        if (k < PLANE) {
            S.x[xs][k] = F.x[j];
            S.b[cs][k] = F.b[j];
            S.dg[cs][k] = F.dg[j];
            S.wx[cs][k] = F.wx[j];
            S.wy[cs][k] = F.wy[j];
            S.wz[zs][k] = F.wz[j];
        }
    }
}

// (b + sum_faces w x_nb) / diag at shared-memory index c of a plane: coefficients from slots
// (cs, zs; zm for the -z face), x from slots (xs; xm, xp for the z neighbours)
template <class T>
RT_HD T update(const Tile<T>& S, int c, int cs, int zs, int zm, int xs, int xm, int xp, bool zero) {
    T num = S.b[cs][c];
    if (!zero) {
        num += S.wx[cs][c] * S.x[xs][c + 1] + S.wx[cs][c - 1] * S.x[xs][c - 1] + S.wy[cs][c] * S.x[xs][c + PX] +
               S.wy[cs][c - PX] * S.x[xs][c - PX] + S.wz[zs][c] * S.x[xp][c] + S.wz[zm][c] * S.x[xm][c];
    }
    return num / S.dg[cs][c];
}

// first colour on plane q over the column plus a one-cell halo, stored in place of the old
// values of those cells (their old values are never read); the column cells of planes
// z0 <= q < z1 are also written out
template <class T>
RT_HD void first_colour(const Args<T>& A, Tile<T>& S, const Item& I, int q) {
    if (I.c1 < 0) return;
    const Geo& d = A.d;
    const int gz = gcoord(q, d.nz, d.per[2]);
    if (gz < 0) return;
    // the pair's cell of the first colour: the left one when its parity matches
    const int o = ((I.par1 + gz) & 1) == A.first ? 0 : 1;
    if (!I.in1[o]) return;
    const int c = I.c1 + o;
    const T v = update(S, c, ring(q, CR), ring(q, ZR), ring(q - 1, ZR), ring(q, XR), ring(q - 1, XR), ring(q + 1, XR),
                       A.zero_guess != 0);
    S.x[ring(q, XR)][c] = v;
    if (I.w1[o] && q >= I.z0 && q < I.z1) {
        const long long i = (long long)q * d.nx * d.ny + I.o1 + o;
        RT_SWEEP_CHECK(i >= 0 && i < (long long)d.nx * d.ny * d.nz);
        A.xout[i] = v;
    }
}

// second colour on plane q (z0 <= q < z1) over the column, from the first colour's new values
template <class T>
RT_HD void second_colour(const Args<T>& A, const Tile<T>& S, const Item& I, int q) {
    if (I.c2 < 0) return;
    const Geo& d = A.d;
    const int o = ((I.par2 + q) & 1) == 1 - A.first ? 0 : 1;
    if (!I.in2[o]) return;
    const int c = I.c2 + o;
    const T v = update(S, c, ring(q, CR), ring(q, ZR), ring(q - 1, ZR), ring(q, XR), ring(q - 1, XR), ring(q + 1, XR),
                       false);
    const long long i = (long long)q * d.nx * d.ny + I.o2 + o;
    RT_SWEEP_CHECK(i >= 0 && i < (long long)d.nx * d.ny * d.nz);
    A.xout[i] = v;
}

// z planes per work item: 16, halved (to no fewer than 4) while the items would not fill
// `slots` resident CTAs
inline int chunk_planes(const Geo& d, long long slots) {
    int zc = 16;
    while (zc > 4 && items(d, zc) < slots) zc /= 2;
    if (zc > d.nz) zc = d.nz;
    return zc;
}

}  // namespace sweep
