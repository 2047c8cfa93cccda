// One red-black Gauss-Seidel sweep of a multigrid level as two in-place colour passes in one
// kernel, ordered so that the second pass finds its data in L2.
//
// The level's operator is (S x)_i = diag_i x_i - sum_faces w_f x_nb (w on each cell's +x/+y/+z
// face, zero on boundary faces).  The first pass sets every cell of the first colour (parity of
// x + y + z equal to `first`) from its neighbours, which all have the other colour; the second
// pass then sets the cells of the other colour from the new first-colour values.  Both passes
// update x in place.
//
// The grid is cut into slabs of `slab` z planes and each colour pass over a slab into chunks (a
// plane and a block of rows, about 8192 cells).  Work items are taken from a counter in a fixed
// queue order in which the second pass over slab k comes right after the first pass over slab
// k + 1:  R0, R1, B0, R2, B1, ..., R(K-1), B(K-2), B(K-1)  (periodic z: B0 moves to the end, as
// it needs R(K-1)).  So the slab's arrays, read from HBM by its first pass, are still in L2 when
// its second pass reads them again: one sweep moves about 7 words per cell through HBM (b, diag,
// wx, wy, wz and x read, x written).
//
// The second pass over slab k reads first-colour values of slabs k - 1 and k + 1 (one plane
// each) and must not overwrite second-colour values that the first pass over slab k + 1 (or
// k - 1) still reads: its chunks wait until the first passes over slabs k - 1, k and k + 1 are
// complete (a per-slab counter of finished chunks).  Every such pass comes earlier in the queue,
// so it has been taken by a running CTA and the wait ends; it is still bounded, and a CTA that
// gives up records it in the error word.  The sweep is exactly the red-black Gauss-Seidel sweep
// whatever the order in which CTAs run.
//
// Chunks map one thread to a pair of x-neighbours (one of each colour), so that every thread of
// a pass updates one cell per pair.  The host functions below give the queue order, the chunk
// layout and the cell updates to a host build too (tests/host/smoother_host.cu).
#pragma once
#include <cuda_runtime.h>

#ifndef RT_HD
#define RT_HD __host__ __device__ __forceinline__
#endif
#ifndef RT_SWEEP_CHECK
#define RT_SWEEP_CHECK(cond) ((void)0)
#endif

namespace rbq {

constexpr int kThreads = 256;
constexpr int kMaxPasses = 1024;   // 2 passes per slab: slabs <= 512

struct Plan {
    int nx, ny, nz;
    int per[3];
    int slab;         // z planes per slab
    int nslab;        // slabs
    int rows;         // rows of a chunk
    int row_blocks;   // chunks per plane
    int chunks;       // chunks per slab pass: slab planes (the last slab may have fewer) x row_blocks
};

// queue position j -> (slab, colour pass: 0 first, 1 second).  With K slabs the queue is
//   non-periodic z: R0, R1, B0, R2, B1, ..., R(K-1), B(K-2), B(K-1)
//   periodic z:     R0, R1, R2, B1, R3, B2, ..., R(K-1), B(K-2), B(K-1), B0
// so every second pass comes after the first passes over its own and both neighbouring slabs
RT_HD void pass_of(const Plan& P, int j, int& slab, int& pass) {
    const int K = P.nslab;
    if (j == 0) {
        slab = 0;
        pass = 0;
        return;
    }
    if (j == 2 * K - 1) {
        slab = P.per[2] ? 0 : K - 1;
        pass = 1;
        return;
    }
    if (!P.per[2]) {
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

// The cells of chunk c of a slab: plane z (>= nz: an empty chunk of the last slab), rows [y0, y1)
RT_HD void chunk_of(const Plan& P, int k, int c, int& z, int& y0, int& y1) {
    z = k * P.slab + c / P.row_blocks;
    y0 = (c % P.row_blocks) * P.rows;
    y1 = y0 + P.rows < P.ny ? y0 + P.rows : P.ny;
}

template <class T>
struct Args {
    Plan P;
    const T* diag;
    const T* wx;
    const T* wy;
    const T* wz;
    const T* b;
    T* x;
    int first;
    int zero_guess;
    unsigned* next;   // work-item counter (zero at launch)
    unsigned* done;   // finished first-pass chunk-warps per slab (zero at launch): a pass over a
                      // slab is complete at chunks x warps per CTA
    int* err;         // bit 5 (value 32) when a CTA gave up waiting
};

RT_HD int up_i(int c, int n, int per) { return c + 1 < n ? c + 1 : (per ? 0 : -1); }
RT_HD int dn_i(int c, int n, int per) { return c > 0 ? c - 1 : (per ? n - 1 : -1); }

// cell (x, y, z) of `colour`-pass: its new value from the current x (neighbours of the other
// colour); `zero` starts from x = 0.  LD reads x (uncached in L1 on the device).
template <class T, class LD>
RT_HD T cell_update(const Args<T>& A, int x, int y, int z, bool zero, LD ld) {
    const Plan& P = A.P;
    const int sy = P.nx;
    const long long sz = (long long)P.nx * P.ny;
    const long long i = (long long)z * sz + (long long)y * sy + x;
    RT_SWEEP_CHECK(i >= 0 && i < sz * P.nz);
    T num = A.b[i];
    if (!zero) {
        const int xm = dn_i(x, P.nx, P.per[0]), xp = up_i(x, P.nx, P.per[0]);
        const int ym = dn_i(y, P.ny, P.per[1]), yp = up_i(y, P.ny, P.per[1]);
        const int zm = dn_i(z, P.nz, P.per[2]), zp = up_i(z, P.nz, P.per[2]);
        const long long row = (long long)z * sz + (long long)y * sy;
        if (xp >= 0) num += A.wx[i] * ld(row + xp);
        if (xm >= 0) num += A.wx[row + xm] * ld(row + xm);
        if (yp >= 0) num += A.wy[i] * ld((long long)z * sz + (long long)yp * sy + x);
        if (ym >= 0) {
            const long long j = (long long)z * sz + (long long)ym * sy + x;
            num += A.wy[j] * ld(j);
        }
        if (zp >= 0) num += A.wz[i] * ld((long long)zp * sz + (long long)y * sy + x);
        if (zm >= 0) {
            const long long j = (long long)zm * sz + (long long)y * sy + x;
            num += A.wz[j] * ld(j);
        }
    }
    return num / A.diag[i];
}

// one thread's part of chunk (slab k, chunk c) of a colour pass: pairs p = tid, tid + nth, ...
// of the chunk's rows, the pair's cell of this pass's colour.  The pairs are taken four at a
// time, their new values all computed before any is stored (a store could otherwise keep the
// next pair's loads from being issued early)
template <class T, class LD>
RT_HD void chunk_pass(const Args<T>& A, int k, int c, int pass, int tid, int nth, LD ld) {
    const Plan& P = A.P;
    int z, y0, y1;
    chunk_of(P, k, c, z, y0, y1);
    if (z >= P.nz) return;
    const int colour = pass == 0 ? A.first : 1 - A.first;
    const bool zero = pass == 0 && A.zero_guess;
    const int hp = (P.nx + 1) / 2;            // pairs per row
    const int npairs = hp * (y1 - y0);
    constexpr int U = 4;
    for (int base = 0; base < npairs; base += U * nth) {
        T v[U];
        int xs[U], ys[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int p = base + u * nth + tid;
            xs[u] = -1;
            if (p >= npairs) continue;
            const int ry = p / hp, px = p - ry * hp;
            const int y = y0 + ry;
            const int x = 2 * px + ((2 * px + y + z + colour) & 1);   // the pair's cell of this colour
            if (x >= P.nx) continue;
            xs[u] = x;
            ys[u] = y;
            v[u] = cell_update(A, x, y, z, zero, ld);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (xs[u] >= 0) A.x[(long long)z * P.nx * P.ny + (long long)ys[u] * P.nx + xs[u]] = v[u];
    }
}

// the plan of a level: slabs of 8 planes (all planes of a thinner grid), chunks of about 8192
// cells
inline Plan make_plan(int nx, int ny, int nz, const int* per) {
    Plan P;
    P.nx = nx;
    P.ny = ny;
    P.nz = nz;
    for (int k = 0; k < 3; ++k) P.per[k] = per[k];
    int rows = 8192 / (nx > 0 ? nx : 1);
    if (rows < 1) rows = 1;
    if (rows > ny) rows = ny;
    P.rows = rows;
    P.row_blocks = (ny + rows - 1) / rows;
    P.slab = nz < 8 ? nz : 8;
    while ((nz + P.slab - 1) / P.slab > kMaxPasses / 2) P.slab *= 2;
    P.nslab = (nz + P.slab - 1) / P.slab;
    // every pass has the same number of chunks; chunks past the last plane are empty
    P.chunks = P.slab * P.row_blocks;
    return P;
}

}  // namespace rbq
