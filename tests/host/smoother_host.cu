// Host build of the fused red-black sweep (smoother.cuh): runs every CTA's phases one after
// another, thread by thread, exactly in the order the kernel's barriers impose, with a check on
// every global index the sweep forms.  Shared memory is filled with NaN before each CTA so that
// a read of a value the CTA never staged shows up in the result.
#include <cmath>
#include <limits>
#include <vector>

static long long g_bad_index = 0;
#ifdef __CUDA_ARCH__
#define RT_SWEEP_CHECK(cond) ((void)0)
#else
#define RT_SWEEP_CHECK(cond) \
    do {                     \
        if (!(cond)) ++g_bad_index; \
    } while (0)
#endif

#include "../../paper_0908_2654_gb300/csrc/smoother.cuh"
#include "../../paper_0908_2654_gb300/csrc/smoother_tma.cuh"
#include "../../paper_0908_2654_gb300/csrc/rbqueue.cuh"
#include "../../paper_0908_2654_gb300/csrc/rbpass.cuh"

template <class T>
static long long run_sweep(int nx, int ny, int nz, const int* per, const T* diag, const T* wx, const T* wy, const T* wz,
                           const T* b, const T* xin, T* xout, int first, int zero, int zc, const T* xc, int cnx,
                           int cny, int cnz, int nth, int grid) {
    g_bad_index = 0;
    sweep::Args<T> A;
    A.d.nx = nx;
    A.d.ny = ny;
    A.d.nz = nz;
    for (int k = 0; k < 3; ++k) A.d.per[k] = per[k];
    A.diag = diag;
    A.wx = wx;
    A.wy = wy;
    A.wz = wz;
    A.b = b;
    A.xin = xin;
    A.xout = xout;
    A.first = first;
    A.zero_guess = zero;
    A.zc = zc > 0 ? zc : sweep::chunk_planes(A.d, 152 * 6);
    if (grid <= 0) grid = 1;
    A.xc = xc;
    A.cd.nx = cnx;
    A.cd.ny = cny;
    A.cd.nz = cnz;
    for (int k = 0; k < 3; ++k) A.cd.per[k] = per[k];
    std::vector<sweep::Tile<T>> tile(1);
    sweep::Tile<T>& S = tile[0];
    T* raw = reinterpret_cast<T*>(&S);
    const size_t nraw = sizeof(S) / sizeof(T);
    std::vector<sweep::Fetch<T>> F(sweep::kThreads);
    std::vector<sweep::Item> I(sweep::kThreads);
    const long long nit = sweep::items(A.d, A.zc);
    // the CTAs of a launch with `grid` blocks, each taking items blockIdx, blockIdx + grid, ...
    for (int blk = 0; blk < grid; ++blk)
        for (long long it = blk; it < nit; it += grid) {
            for (size_t k = 0; k < nraw; ++k) raw[k] = std::numeric_limits<T>::quiet_NaN();
            for (int t = 0; t < sweep::kThreads; ++t) sweep::item_setup(A, it, t, I[t]);
            const int z0 = I[0].z0, z1 = I[0].z1;
            for (int t = 0; t < sweep::kThreads; ++t) sweep::fetch(A, I[t], z0 - 2, F[t]);
            for (int p = z0 - 2; p <= z1 + 1; ++p) {
                for (int t = 0; t < sweep::kThreads; ++t) sweep::stage(S, p, t, F[t]);
                if (p < z1 + 1)
                    for (int t = 0; t < sweep::kThreads; ++t) sweep::fetch(A, I[t], p + 1, F[t]);
                if (p - 1 >= z0 - 1)
                    for (int t = 0; t < sweep::kThreads; ++t) sweep::first_colour(A, S, I[t], p - 1);
                if (p - 2 >= z0)
                    for (int t = 0; t < sweep::kThreads; ++t) sweep::second_colour(A, S, I[t], p - 2);
            }
        }
    return g_bad_index;
}

extern "C" {
long long sweep_host_f64(int nx, int ny, int nz, const int* per, const double* diag, const double* wx,
                         const double* wy, const double* wz, const double* b, const double* xin, double* xout,
                         int first, int zero, int zc, const double* xc, int cnx, int cny, int cnz, int nth,
                         int grid) {
    return run_sweep<double>(nx, ny, nz, per, diag, wx, wy, wz, b, xin, xout, first, zero, zc, xc, cnx, cny, cnz, nth,
                             grid);
}
long long sweep_host_f32(int nx, int ny, int nz, const int* per, const float* diag, const float* wx, const float* wy,
                         const float* wz, const float* b, const float* xin, float* xout, int first, int zero, int zc,
                         const float* xc, int cnx, int cny, int cnz, int nth, int grid) {
    return run_sweep<float>(nx, ny, nz, per, diag, wx, wy, wz, b, xin, xout, first, zero, zc, xc, cnx, cny, cnz, nth,
                            grid);
}
int sweep_chunk_planes(int nx, int ny, int nz, long long slots) {
    sweep::Geo d;
    d.nx = nx;
    d.ny = ny;
    d.nz = nz;
    d.per[0] = d.per[1] = d.per[2] = 0;
    return sweep::chunk_planes(d, slots);
}
}

// the TMA-fed sweep, its copies emulated in the kernel's order: the copy of plane p + D lands at
// the start of step p, in the slot plane p + D - NR held
template <class T>
static long long run_sweep_tma(int nx, int ny, int nz, const int* per, const T* diag, const T* wx, const T* wy,
                               const T* wz, const T* b, const T* xin, T* xout, int first, int zero, int zc,
                               int grid) {
    using G = tsweep::Geom<T>;
    g_bad_index = 0;
    tsweep::Args<T> A;
    A.d.nx = nx;
    A.d.ny = ny;
    A.d.nz = nz;
    for (int k = 0; k < 3; ++k) A.d.per[k] = per[k];
    A.b = b;
    A.diag = diag;
    A.wx = wx;
    A.wy = wy;
    A.wz = wz;
    A.xin = xin;
    A.xout = xout;
    A.first = first;
    A.zero_guess = zero;
    A.zc = zc > 0 ? zc : sweep::chunk_planes(A.d, 152 * 3);
    A.err = nullptr;
    if (grid <= 0) grid = 1;
    std::vector<tsweep::Tile<T>> tile(1);
    tsweep::Tile<T>& S = tile[0];
    T* raw = reinterpret_cast<T*>(&S.t[0][0][0]);
    const size_t nraw = sizeof(S.t) / sizeof(T);
    std::vector<tsweep::Item> I(tsweep::kThreads);
    const long long nit = sweep::items(A.d, A.zc);
    for (int blk = 0; blk < grid; ++blk) {
        for (size_t k = 0; k < nraw; ++k) raw[k] = std::numeric_limits<T>::quiet_NaN();
        long long seq = 0;
        for (long long it = blk; it < nit; it += grid) {
            for (int t = 0; t < tsweep::kThreads; ++t) tsweep::item_setup(A, it, t, I[t]);
            const int p0 = I[0].z0 - 2, p1 = I[0].z1 + 1;
            for (int p = p0; p < p0 + G::D && p <= p1; ++p)
                tsweep::emulate_copy(A, S, I[0], p, tsweep::slot_of(seq + (p - p0), G::NR));
            for (int p = p0; p <= p1; ++p) {
                const long long sq = seq + (p - p0);
                if (p + G::D <= p1) tsweep::emulate_copy(A, S, I[0], p + G::D, tsweep::slot_of(sq + G::D, G::NR));
                const int s = tsweep::slot_of(sq, G::NR);
                for (int t = 0; t < tsweep::kThreads; ++t) tsweep::fix_plane(A, S, I[t], p, s, t, tsweep::kThreads);
                if (p - 1 >= p0 + 1)
                    for (int t = 0; t < tsweep::kThreads; ++t) tsweep::first_colour(A, S, I[t], p - 1, sq - 1);
                if (p - 2 >= I[0].z0)
                    for (int t = 0; t < tsweep::kThreads; ++t) tsweep::second_colour(A, S, I[t], p - 2, sq - 2);
            }
            seq += p1 - p0 + 1;
        }
    }
    return g_bad_index;
}

extern "C" {
long long sweep_tma_host_f64(int nx, int ny, int nz, const int* per, const double* diag, const double* wx,
                             const double* wy, const double* wz, const double* b, const double* xin, double* xout,
                             int first, int zero, int zc, int grid) {
    return run_sweep_tma<double>(nx, ny, nz, per, diag, wx, wy, wz, b, xin, xout, first, zero, zc, grid);
}
long long sweep_tma_host_f32(int nx, int ny, int nz, const int* per, const float* diag, const float* wx,
                             const float* wy, const float* wz, const float* b, const float* xin, float* xout,
                             int first, int zero, int zc, int grid) {
    return run_sweep_tma<float>(nx, ny, nz, per, diag, wx, wy, wz, b, xin, xout, first, zero, zc, grid);
}
}

// the in-place sweep of rbqueue.cuh: its work items in queue order, each chunk's threads one
// after another (the order a single CTA would take them; the dependencies hold by construction)
template <class T>
static long long run_sweep_queue(int nx, int ny, int nz, const int* per, const T* diag, const T* wx, const T* wy,
                                 const T* wz, const T* b, T* x, int first, int zero) {
    g_bad_index = 0;
    rbq::Args<T> A;
    A.P = rbq::make_plan(nx, ny, nz, per);
    A.diag = diag;
    A.wx = wx;
    A.wy = wy;
    A.wz = wz;
    A.b = b;
    A.x = x;
    A.first = first;
    A.zero_guess = zero;
    const long long n = (long long)nx * ny * nz;
    auto ld = [&](long long j) {
        if (!(j >= 0 && j < n)) ++g_bad_index;
        return x[j];
    };
    const unsigned nitems = 2u * (unsigned)A.P.nslab * (unsigned)A.P.chunks;
    std::vector<int> done(A.P.nslab, 0);
    for (unsigned s = 0; s < nitems; ++s) {
        int k, pass;
        rbq::pass_of(A.P, (int)(s / (unsigned)A.P.chunks), k, pass);
        const int c = (int)(s % (unsigned)A.P.chunks);
        if (pass == 1)
            for (int dk = -1; dk <= 1; ++dk) {
                int kk = k + dk;
                if (kk < 0 || kk >= A.P.nslab) {
                    if (!per[2]) continue;
                    kk = (kk + A.P.nslab) % A.P.nslab;
                }
                if (done[kk] < A.P.chunks) ++g_bad_index;   // a second pass before its first passes
            }
        for (int t = 0; t < rbq::kThreads; ++t) rbq::chunk_pass(A, k, c, pass, t, rbq::kThreads, ld);
        if (pass == 0) ++done[k];
    }
    return g_bad_index;
}

extern "C" {
long long sweep_queue_host_f64(int nx, int ny, int nz, const int* per, const double* diag, const double* wx,
                               const double* wy, const double* wz, const double* b, double* x, int first, int zero) {
    return run_sweep_queue<double>(nx, ny, nz, per, diag, wx, wy, wz, b, x, first, zero);
}
long long sweep_queue_host_f32(int nx, int ny, int nz, const int* per, const float* diag, const float* wx,
                               const float* wy, const float* wz, const float* b, float* x, int first, int zero) {
    return run_sweep_queue<float>(nx, ny, nz, per, diag, wx, wy, wz, b, x, first, zero);
}
int queue_plan(int nx, int ny, int nz, int pz, int* out) {
    const int per[3] = {0, 0, pz};
    const rbq::Plan P = rbq::make_plan(nx, ny, nz, per);
    out[0] = P.slab;
    out[1] = P.nslab;
    out[2] = P.rows;
    out[3] = P.row_blocks;
    out[4] = P.chunks;
    return 0;
}
}

// the slab-ordered colour passes of rbpass.cuh, every block and thread of each launch in turn
template <class T>
static long long run_sweep_pass(int nx, int ny, int nz, const int* per, const T* diag, const T* wx, const T* wy,
                                const T* wz, const T* b, T* x, int first, int zero, int slab) {
    g_bad_index = 0;
    const int S = slab > 0 ? slab : rbp::slab_planes(nx, ny, nz, (int)sizeof(T));
    const int K = (nz + S - 1) / S;
    std::vector<int> done(K, 0);
    for (int j = 0; j < 2 * K; ++j) {
        int k, pass;
        rbp::launch_of(K, per[2], j, k, pass);
        if (pass == 1)
            for (int dk = -1; dk <= 1; ++dk) {
                int kk = k + dk;
                if (kk < 0 || kk >= K) {
                    if (!per[2]) continue;
                    kk = (kk + K) % K;
                }
                if (!done[kk]) ++g_bad_index;       // a second pass before a neighbouring first pass
            }
        if (pass == 0) done[k] = 1;
        rbp::Pass<T> A;
        A.nx = nx;
        A.ny = ny;
        A.nz = nz;
        for (int q = 0; q < 3; ++q) A.per[q] = per[q];
        A.diag = diag;
        A.wx = wx;
        A.wy = wy;
        A.wz = wz;
        A.b = b;
        A.x = x;
        A.colour = pass == 0 ? first : 1 - first;
        A.zero = pass == 0 && zero;
        A.z0 = k * S;
        const int planes = A.z0 + S <= nz ? S : nz - A.z0;
        int gx, gy, gz;
        rbp::pass_grid(nx, ny, planes, gx, gy, gz, A.rows);
        // all threads of a launch read before any writes: the cells a pass sets are never read by it
        for (int bz = 0; bz < gz; ++bz)
            for (int by = 0; by < gy; ++by)
                for (int bx = 0; bx < gx; ++bx)
                    for (int t = 0; t < rbp::kPairs; ++t) {
                        int cx, cy, cz;
                        if (!rbp::pair_cell(A, bx, by, bz, t, cx, cy, cz)) continue;
                        const long long i = ((long long)cz * ny + cy) * nx + cx;
                        if (!(i >= 0 && i < (long long)nx * ny * nz)) ++g_bad_index;
                        x[i] = rbp::cell_value(A, cx, cy, cz);
                    }
    }
    return g_bad_index;
}

extern "C" {
long long sweep_pass_host_f64(int nx, int ny, int nz, const int* per, const double* diag, const double* wx,
                              const double* wy, const double* wz, const double* b, double* x, int first, int zero,
                              int slab) {
    return run_sweep_pass<double>(nx, ny, nz, per, diag, wx, wy, wz, b, x, first, zero, slab);
}
long long sweep_pass_host_f32(int nx, int ny, int nz, const int* per, const float* diag, const float* wx,
                              const float* wy, const float* wz, const float* b, float* x, int first, int zero, int slab) {
    return run_sweep_pass<float>(nx, ny, nz, per, diag, wx, wy, wz, b, x, first, zero, slab);
}
}
