// Host build of the multigrid level kernels' cell functions (rbpass.cuh): the two in-place
// colour passes of a red-black sweep, every block and thread of each launch in turn, and the
// trilinear prolongation, with a check on every global index they form.
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
                           const T* wz, const T* b, T* x, int first, int zero) {
    g_bad_index = 0;
    for (int pass = 0; pass < 2; ++pass) {
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
        A.z0 = 0;
        A.planes = nz;
        A.rev = pass;
        int gx, gy, gz;
        rbp::pass_grid(nx, ny, nz, gx, gy, gz, A.rows);
        std::vector<int> hits((size_t)nx * ny * nz, 0);
        // a pass never reads the cells it sets, so the order of its threads does not matter
        for (int bz = 0; bz < gz; ++bz)
            for (int by = 0; by < gy; ++by)
                for (int bx = 0; bx < gx; ++bx)
                    for (int t = 0; t < rbp::kPairs; ++t) {
                        int cx, cy, cz;
                        if (!rbp::pair_cell(A, bx, by, bz, t, cx, cy, cz)) continue;
                        const long long i = ((long long)cz * ny + cy) * nx + cx;
                        if (!(i >= 0 && i < (long long)nx * ny * nz)) {
                            ++g_bad_index;
                            continue;
                        }
                        ++hits[i];
                        x[i] = rbp::cell_value(A, cx, cy, cz);
                    }
        // every cell of the pass's colour set exactly once, no other cell touched
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int xx = 0; xx < nx; ++xx) {
                    const int want = ((xx + y + z) & 1) == A.colour ? 1 : 0;
                    if (hits[((size_t)z * ny + y) * nx + xx] != want) ++g_bad_index;
                }
    }
    return g_bad_index;
}

extern "C" {
long long sweep_host_f64(int nx, int ny, int nz, const int* per, const double* diag, const double* wx,
                         const double* wy, const double* wz, const double* b, double* x, int first, int zero) {
    return run_sweep<double>(nx, ny, nz, per, diag, wx, wy, wz, b, x, first, zero);
}
long long sweep_host_f32(int nx, int ny, int nz, const int* per, const float* diag, const float* wx,
                         const float* wy, const float* wz, const float* b, float* x, int first, int zero) {
    return run_sweep<float>(nx, ny, nz, per, diag, wx, wy, wz, b, x, first, zero);
}
// out[z][y][x] = trilinear prolongation of the coarse vector xc (cnx x cny x cnz) at every fine cell
long long prolong_host(int nx, int ny, int nz, const int* per, const double* xc, int cnx, int cny, int cnz,
                       double* out) {
    g_bad_index = 0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                out[((long long)z * ny + y) * nx + x] = rbp::prolong_at(xc, cnx, cny, cnz, per, x, y, z);
    return g_bad_index;
}
}
