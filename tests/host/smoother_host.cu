// Host build of the multigrid level functions (rbpass.cuh): the colour-split storage of a level
// (its operator and vectors), the two in-place colour passes of a red-black sweep on it, every
// block and thread of each launch in turn, and the trilinear prolongation from a natural or
// colour-split coarse vector, with a check on every index they form.
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

#include "../../paper_0908_2654_gb300/csrc/rbpass.cuh"

template <class T>
static long long run_sweep(int nx, int ny, int nz, const int* per, const T* diag, const T* wx, const T* wy,
                           const T* wz, const T* b, T* x, int first, int zero, int quad) {
    g_bad_index = 0;
    const long long n = (long long)nx * ny * nz, half = n / 2;
    // the level in colour-split storage
    std::vector<T> dinv(n, T(-1)), w6(3 * n, T(-1)), bs(n), xs(n);
    for (long long m = 0; m < half; ++m) rbp::split_pair(nx, ny, nz, per, diag, wx, wy, wz, m, dinv.data(), w6.data());
    std::vector<int> seen(n, 0);
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int xx = 0; xx < nx; ++xx) {
                const long long i = ((long long)z * ny + y) * nx + xx;
                const long long s = rbp::level_index(1, nx, ny, nz, xx, y, z);
                if (s < 0 || s >= n) {
                    ++g_bad_index;
                    continue;
                }
                ++seen[s];
                bs[s] = b[i];
                xs[s] = x[i];
            }
    for (long long s = 0; s < n; ++s)
        if (seen[s] != 1) ++g_bad_index;   // level_index is a bijection
    for (long long k = 0; k < n; ++k)
        if (dinv[k] == T(-1)) ++g_bad_index;   // every diagonal entry written
    for (long long k = 0; k < 3 * n; ++k)
        if (w6[k] == T(-1)) ++g_bad_index;   // every face entry written
    for (int pass = 0; pass < 2; ++pass) {
        const int colour = pass == 0 ? first : 1 - first;
        rbp::Pass<T> A = rbp::make_pass<T>(nx, ny, nz, per, w6.data(), dinv.data(), bs.data(), xs.data(), colour,
                                           pass == 0 && zero, pass);
        if (A.quad != (nx % 4 == 0)) ++g_bad_index;
        A.quad = quad && A.quad;   // the single-pair form on request
        int gx, gy, gz;
        rbp::pass_launch(A, gx, gy, gz);
        std::vector<int> hits(n, 0);
        // a pass never reads the cells it sets, so the order of its threads does not matter
        for (int bz = 0; bz < gz; ++bz)
            for (int by = 0; by < gy; ++by)
                for (int bx = 0; bx < gx; ++bx)
                    for (int t = 0; t < rbp::kPairs; ++t) {
                        if (A.quad) {
                            int px, cy, cz;
                            if (!rbp::quad_pairs(A, bx, by, bz, t, px, cy, cz)) continue;
                            if (px < 0 || px + 1 >= nx / 2 || cy < 0 || cy >= ny || cz < 0 || cz >= nz) {
                                ++g_bad_index;
                                continue;
                            }
                            T v0, v1;
                            if (A.colour)
                                rbp::quad_values<1>(A, px, cy, cz, v0, v1);
                            else
                                rbp::quad_values<0>(A, px, cy, cz, v0, v1);
                            const long long m = ((long long)cz * ny + cy) * (nx / 2) + px;
                            if ((m & 1) != 0) ++g_bad_index;   // two-element accesses stay aligned
                            rbp::st2(A.x + m, v0, v1);
                            for (int k = 0; k < 2; ++k) {
                                const int cx = 2 * (px + k) + ((cy + cz + A.colour) & 1);
                                ++hits[((long long)cz * ny + cy) * nx + cx];
                                if (rbp::level_index(1, nx, ny, nz, cx, cy, cz) != A.colour * half + m + k)
                                    ++g_bad_index;
                            }
                            continue;
                        }
                        int cx, cy, cz;
                        if (!rbp::pair_cell(A, bx, by, bz, t, cx, cy, cz)) continue;
                        if (cx < 0 || cx >= nx || cy < 0 || cy >= ny || cz < 0 || cz >= nz) {
                            ++g_bad_index;
                            continue;
                        }
                        const long long s = rbp::level_index(1, nx, ny, nz, cx, cy, cz);
                        if (s != A.colour * half + rbp::pair_of(A, cx, cy, cz)) ++g_bad_index;
                        ++hits[((long long)cz * ny + cy) * nx + cx];
                        A.x[rbp::pair_of(A, cx, cy, cz)] =
                            A.colour ? rbp::cell_value<1>(A, cx, cy, cz) : rbp::cell_value<0>(A, cx, cy, cz);
                    }
        // every cell of the pass's colour set exactly once, no other cell touched
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int xx = 0; xx < nx; ++xx) {
                    const int want = ((xx + y + z) & 1) == A.colour ? 1 : 0;
                    if (hits[((long long)z * ny + y) * nx + xx] != want) ++g_bad_index;
                }
    }
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int xx = 0; xx < nx; ++xx)
                x[((long long)z * ny + y) * nx + xx] = xs[rbp::level_index(1, nx, ny, nz, xx, y, z)];
    return g_bad_index;
}

extern "C" {
long long sweep_host_f64(int nx, int ny, int nz, const int* per, const double* diag, const double* wx,
                         const double* wy, const double* wz, const double* b, double* x, int first, int zero,
                         int quad) {
    return run_sweep<double>(nx, ny, nz, per, diag, wx, wy, wz, b, x, first, zero, quad);
}
long long sweep_host_f32(int nx, int ny, int nz, const int* per, const float* diag, const float* wx,
                         const float* wy, const float* wz, const float* b, float* x, int first, int zero, int quad) {
    return run_sweep<float>(nx, ny, nz, per, diag, wx, wy, wz, b, x, first, zero, quad);
}
// out[z][y][x] = trilinear prolongation at every fine cell of the coarse vector xc (cnx x cny x
// cnz, natural order), read from a colour-split copy when csplit
long long prolong_host(int nx, int ny, int nz, const int* per, const double* xc, int cnx, int cny, int cnz,
                       int csplit, double* out) {
    g_bad_index = 0;
    const long long nc = (long long)cnx * cny * cnz;
    std::vector<double> c(nc);
    for (int Z = 0; Z < cnz; ++Z)
        for (int Y = 0; Y < cny; ++Y)
            for (int X = 0; X < cnx; ++X)
                c[rbp::level_index(csplit, cnx, cny, cnz, X, Y, Z)] = xc[((long long)Z * cny + Y) * cnx + X];
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                out[((long long)z * ny + y) * nx + x] = rbp::prolong_at(c.data(), csplit, cnx, cny, cnz, per, x, y, z);
    return g_bad_index;
}
// the same from prolong_pair, one fine x-pair at a time (nx even)
long long prolong_pair_host(int nx, int ny, int nz, const int* per, const double* xc, int cnx, int cny, int cnz,
                            int csplit, double* out) {
    g_bad_index = 0;
    const long long nc = (long long)cnx * cny * cnz;
    std::vector<double> c(nc);
    for (int Z = 0; Z < cnz; ++Z)
        for (int Y = 0; Y < cny; ++Y)
            for (int X = 0; X < cnx; ++X)
                c[rbp::level_index(csplit, cnx, cny, cnz, X, Y, Z)] = xc[((long long)Z * cny + Y) * cnx + X];
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int px = 0; px < nx / 2; ++px) {
                double v0, v1;
                rbp::prolong_pair(c.data(), csplit, cnx, cny, cnz, per, px, y, z, v0, v1);
                out[((long long)z * ny + y) * nx + 2 * px] = v0;
                out[((long long)z * ny + y) * nx + 2 * px + 1] = v1;
            }
    return g_bad_index;
}

// out[z][y][x] = b - S x for a colour-split level (x, b given in natural order, permuted here),
// every fine pair through pair_residuals
long long resid_host(int nx, int ny, int nz, const int* per, const double* diag, const double* wx, const double* wy,
                     const double* wz, const double* b, const double* x, double* out) {
    g_bad_index = 0;
    const long long n = (long long)nx * ny * nz;
    std::vector<double> bs(n), xs(n);
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int xx = 0; xx < nx; ++xx) {
                const long long i = ((long long)z * ny + y) * nx + xx;
                const long long s = rbp::level_index(1, nx, ny, nz, xx, y, z);
                bs[s] = b[i];
                xs[s] = x[i];
            }
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int px = 0; px < nx / 2; ++px) {
                double rE, rO;
                rbp::pair_residuals(nx, ny, nz, per, diag, wx, wy, wz, bs.data(), xs.data(), px, y, z, rE, rO);
                out[((long long)z * ny + y) * nx + 2 * px] = rE;
                out[((long long)z * ny + y) * nx + 2 * px + 1] = rO;
            }
    return g_bad_index;
}

// pairs of neighbours (periodic wraps included, a cell that is its own neighbour skipped) that
// share a colour of the coarse solver's colouring, and the number of colours it uses
long long colour_conflicts(int nx, int ny, int nz, const int* per, int* ncol_out) {
    const int ncol = rbp::odd_periodic(nx, ny, nz, per) ? 3 : 2;
    *ncol_out = ncol;
    long long bad = 0;
    const int n[3] = {nx, ny, nz};
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const int c = rbp::multicolour(nx, ny, nz, per, ncol, x, y, z);
                if (c < 0 || c >= ncol) ++bad;
                for (int a = 0; a < 3; ++a) {
                    int v[3] = {x, y, z};
                    if (v[a] + 1 < n[a]) v[a] += 1;
                    else if (per[a]) v[a] = 0;
                    else continue;
                    if (v[0] == x && v[1] == y && v[2] == z) continue;
                    if (rbp::multicolour(nx, ny, nz, per, ncol, v[0], v[1], v[2]) == c) ++bad;
                }
            }
    return bad;
}
}
