// The red-black Gauss-Seidel sweep of smoother.cuh with its planes staged by the Tensor Memory
// Accelerator: one thread issues, per plane, six bulk tensor copies (b, diag, wx, wy, wz and the
// old iterate) of the column plus halo into a ring of shared-memory slots, a few planes ahead of
// the plane being computed, and an mbarrier per slot signals their arrival.  The threads then
// only compute: no load or staging instructions, and the copies' latency is hidden behind the
// arithmetic of the planes in between.
//
// The copied box starts XOFF cells to the left of the column so that its first element lies on
// a 16-byte boundary (XOFF = 4 for FP32, 2 for FP64), spans the column plus that margin on both
// sides in x and a two-cell halo in y, and is one plane deep.  Cells of the box outside the grid
// arrive as zeros, which is what a reflecting or outflow face needs (its coupling is zero); on a
// periodic axis the cells beyond the edge are then overwritten with their wrapped values by
// ordinary loads (only CTAs whose box crosses such an edge do this).  Planes outside a
// non-periodic grid are not copied: their slot is zeroed.  A zero old iterate (the first
// pre-smoothing sweep) is not copied either: its tile is zeroed.
//
// Every wait on an mbarrier is bounded: a CTA that runs out of tries records the failure in an
// error word, waits (again bounded) for its own copies still in flight and returns.
//
// The compute phases are host/device functions (a host build emulates the copies and runs them,
// tests/host/smoother_host.cu); the copies and barriers are device code.
#pragma once
#include <cuda_runtime.h>

#include "smoother.cuh"

namespace tsweep {

using sweep::Geo;
using sweep::gcoord;
constexpr int TX = sweep::TX, TY = sweep::TY, HALO = sweep::HALO;
constexpr int kThreads = sweep::kThreads;
enum { AB = 0, AD, AWX, AWY, AWZ, AX, NARR };   // the copied arrays of a plane

template <class T>
struct Geom {
    static constexpr int XOFF = sizeof(T) == 4 ? 4 : 2;   // cells between the box's start and the column
    static constexpr int BX = TX + 2 * XOFF;              // box width: 40 (FP32) or 36 (FP64)
    static constexpr int BY = TY + 2 * HALO;              // box height: 12
    static constexpr int TILE = BX * BY;                  // elements of one array's plane
    static constexpr int D = sizeof(T) == 4 ? 2 : 1;      // planes copied ahead of the computed one
    // slots: the second colour of plane p - 2 still reads the first colour of p - 3 while the
    // copies of planes up to p + D are in flight
    static constexpr int NR = D + 4;
};

template <class T>
struct Tile {
    T t[Geom<T>::NR][NARR][Geom<T>::TILE];   // each tile 128-byte aligned: TILE * sizeof(T) % 128 == 0
    unsigned long long bar[Geom<T>::NR];
};
static_assert(Geom<float>::TILE * sizeof(float) % 128 == 0 && Geom<double>::TILE * sizeof(double) % 128 == 0,
              "tiles stay 128-byte aligned");

template <class T>
struct Args {
    Geo d;
    const T* b;        // the same arrays the tensor maps describe, for the periodic edge cells
    const T* diag;
    const T* wx;
    const T* wy;
    const T* wz;
    const T* xin;
    T* xout;
    int first;
    int zero_guess;
    int zc;
    int* err;          // bit 4 (value 16) set when a CTA gave up waiting for its copies
};

// per-thread addressing of a work item (as sweep::Item, for the box layout)
struct Item {
    int X0, Y0, z0, z1;
    int patch;         // the box crosses an edge of a periodic x or y axis
    int c1;            // first-colour pair (column plus halo): box index of the left cell
    bool in1[2];
    int par1;
    bool w1[2];
    int o1;
    int c2;            // second-colour pair (column)
    bool in2[2];
    int par2;
    int o2;
};

template <class T>
RT_HD int box_index(int lx, int ly) {
    return (ly + HALO) * Geom<T>::BX + (lx + Geom<T>::XOFF);
}

template <class T>
RT_HD void item_setup(const Args<T>& A, long long it, int tid, Item& I) {
    const Geo& d = A.d;
    const int cx = sweep::columns_x(d), cy = sweep::columns_y(d);
    const long long col = it % ((long long)cx * cy);
    const int ch = (int)(it / ((long long)cx * cy));
    I.X0 = (int)(col % cx) * TX;
    I.Y0 = (int)(col / cx) * TY;
    I.z0 = ch * A.zc;
    I.z1 = I.z0 + A.zc < d.nz ? I.z0 + A.zc : d.nz;
    const int xo = Geom<T>::XOFF;
    I.patch = (d.per[0] && (I.X0 - xo < 0 || I.X0 + TX + xo > d.nx)) ||
              (d.per[1] && (I.Y0 - HALO < 0 || I.Y0 + TY + HALO > d.ny));
    I.c1 = -1;
    if (tid < sweep::P1) {
        const int lx = -1 + 2 * (tid % ((TX + 2) / 2)), ly = -1 + tid / ((TX + 2) / 2);
        const int gy = gcoord(I.Y0 + ly, d.ny, d.per[1]);
        const int g0 = gcoord(I.X0 + lx, d.nx, d.per[0]), g1 = gcoord(I.X0 + lx + 1, d.nx, d.per[0]);
        I.c1 = box_index<T>(lx, ly);
        I.in1[0] = gy >= 0 && g0 >= 0;
        I.in1[1] = gy >= 0 && g1 >= 0;
        I.par1 = I.in1[0] ? (g0 + gy) & 1 : (I.in1[1] ? (g1 + gy + 1) & 1 : 0);
        const bool row = ly >= 0 && ly < TY && I.Y0 + ly < d.ny;
        I.w1[0] = row && lx >= 0 && I.X0 + lx < d.nx;
        I.w1[1] = row && lx + 1 < TX && I.X0 + lx + 1 < d.nx;
        I.o1 = (I.Y0 + ly) * d.nx + (I.X0 + lx);
    }
    I.c2 = -1;
    if (tid < sweep::P2) {
        const int lx = 2 * (tid % (TX / 2)), ly = tid / (TX / 2);
        I.c2 = box_index<T>(lx, ly);
        const bool row = I.Y0 + ly < d.ny;
        I.in2[0] = row && I.X0 + lx < d.nx;
        I.in2[1] = row && I.X0 + lx + 1 < d.nx;
        I.par2 = (I.X0 + lx + I.Y0 + ly) & 1;
        I.o2 = (I.Y0 + ly) * d.nx + (I.X0 + lx);
    }
}

RT_HD int slot_of(long long seq, int nr) { return (int)(seq % nr); }

// after the copies of plane p landed in slot s: zero the old iterate (zero start), zero the whole
// slot (a plane outside a non-periodic grid), or overwrite the box cells beyond a periodic edge
// with their wrapped values
template <class T>
RT_HD void fix_plane(const Args<T>& A, Tile<T>& S, const Item& I, int p, int s, int tid, int nth) {
    const Geo& d = A.d;
    const int gz = gcoord(p, d.nz, d.per[2]);
    constexpr int TILE = Geom<T>::TILE, BX = Geom<T>::BX, XOFF = Geom<T>::XOFF;
    if (gz < 0) {
        for (int k = tid; k < NARR * TILE; k += nth) S.t[s][k / TILE][k % TILE] = T(0);
        return;
    }
    if (A.zero_guess)
        for (int k = tid; k < TILE; k += nth) S.t[s][AX][k] = T(0);
    if (!I.patch) return;
    const long long plane = (long long)gz * d.nx * d.ny;
    for (int k = tid; k < TILE; k += nth) {
        const int ux = I.X0 + k % BX - XOFF, uy = I.Y0 + k / BX - HALO;   // unwrapped coordinates
        const bool outx = ux < 0 || ux >= d.nx, outy = uy < 0 || uy >= d.ny;
        if (!outx && !outy) continue;
        const int gx = gcoord(ux, d.nx, d.per[0]), gy = gcoord(uy, d.ny, d.per[1]);
        if (gx < 0 || gy < 0) continue;          // beyond a non-periodic edge: the copy's zero stays
        const long long i = plane + (long long)gy * d.nx + gx;
        RT_SWEEP_CHECK(i >= 0 && i < (long long)d.nx * d.ny * d.nz);
        S.t[s][AB][k] = A.b[i];
        S.t[s][AD][k] = A.diag[i];
        S.t[s][AWX][k] = A.wx[i];
        S.t[s][AWY][k] = A.wy[i];
        S.t[s][AWZ][k] = A.wz[i];
        if (!A.zero_guess) S.t[s][AX][k] = A.xin[i];
    }
}

// (b + sum_faces w x_nb) / diag at box index c: coefficients of slot cs (wz of slot zm for the -z
// face), x from slot cs and the z neighbours' slots xm, xp
template <class T>
RT_HD T update(const Tile<T>& S, int c, int cs, int zm, int xm, int xp, bool zero) {
    constexpr int BX = Geom<T>::BX;
    const T(&sl)[NARR][Geom<T>::TILE] = S.t[cs];
    T num = sl[AB][c];
    if (!zero) {
        num += sl[AWX][c] * sl[AX][c + 1] + sl[AWX][c - 1] * sl[AX][c - 1] + sl[AWY][c] * sl[AX][c + BX] +
               sl[AWY][c - BX] * sl[AX][c - BX] + sl[AWZ][c] * S.t[xp][AX][c] + S.t[zm][AWZ][c] * S.t[xm][AX][c];
    }
    return num / sl[AD][c];
}

// first colour of plane q (sequence number seq_q, slots of q - 1 and q + 1 at seq_q -+ 1),
// stored in place of the old values and, for column cells of planes z0 <= q < z1, written out
template <class T>
RT_HD void first_colour(const Args<T>& A, Tile<T>& S, const Item& I, int q, long long seq_q) {
    if (I.c1 < 0) return;
    const Geo& d = A.d;
    const int gz = gcoord(q, d.nz, d.per[2]);
    if (gz < 0) return;
    const int o = ((I.par1 + gz) & 1) == A.first ? 0 : 1;
    if (!I.in1[o]) return;
    constexpr int NR = Geom<T>::NR;
    const int cs = slot_of(seq_q, NR), sm = slot_of(seq_q - 1, NR), sp = slot_of(seq_q + 1, NR);
    const int c = I.c1 + o;
    const T v = update(S, c, cs, sm, sm, sp, A.zero_guess != 0);
    S.t[cs][AX][c] = v;
    if (I.w1[o] && q >= I.z0 && q < I.z1) {
        const long long i = (long long)q * d.nx * d.ny + I.o1 + o;
        RT_SWEEP_CHECK(i >= 0 && i < (long long)d.nx * d.ny * d.nz);
        A.xout[i] = v;
    }
}

// second colour of plane q (z0 <= q < z1) from the first colour's new values
template <class T>
RT_HD void second_colour(const Args<T>& A, const Tile<T>& S, const Item& I, int q, long long seq_q) {
    if (I.c2 < 0) return;
    const Geo& d = A.d;
    const int o = ((I.par2 + q) & 1) == 1 - A.first ? 0 : 1;
    if (!I.in2[o]) return;
    constexpr int NR = Geom<T>::NR;
    const int cs = slot_of(seq_q, NR), sm = slot_of(seq_q - 1, NR), sp = slot_of(seq_q + 1, NR);
    const int c = I.c2 + o;
    const T v = update(S, c, cs, sm, sm, sp, false);
    const long long i = (long long)q * d.nx * d.ny + I.o2 + o;
    RT_SWEEP_CHECK(i >= 0 && i < (long long)d.nx * d.ny * d.nz);
    A.xout[i] = v;
}

// the copy of plane p as a host build performs it (the box with zeros outside the grid), for the
// emulation of the kernel
template <class T>
inline void emulate_copy(const Args<T>& A, Tile<T>& S, const Item& I, int p, int s) {
    const Geo& d = A.d;
    constexpr int TILE = Geom<T>::TILE, BX = Geom<T>::BX, XOFF = Geom<T>::XOFF;
    const T* src[NARR] = {A.b, A.diag, A.wx, A.wy, A.wz, A.xin};
    const int gz = gcoord(p, d.nz, d.per[2]);     // the kernel copies the wrapped plane
    if (gz < 0) return;                           // and no plane outside a non-periodic grid
    for (int a = 0; a < NARR; ++a) {
        if (a == AX && A.zero_guess) continue;
        for (int k = 0; k < TILE; ++k) {
            const int x = I.X0 + k % BX - XOFF, y = I.Y0 + k / BX - HALO;
            const bool in = x >= 0 && x < d.nx && y >= 0 && y < d.ny;
            S.t[s][a][k] = in ? src[a][((long long)gz * d.ny + y) * d.nx + x] : T(0);
        }
    }
}

}  // namespace tsweep
