// Device helpers shared by the per-cell kernels: cell coordinates, neighbours, the 7-point
// stencil of the face couplings and per-block partial sums.
#pragma once
#include <cuda_runtime.h>

namespace cellgrid {

constexpr int kBlock = 256;

// (x, y, z) of cell i = (z ny + y) nx + x.  Grids hold at most 2^31 cells (rt_init_grid), so
// i fits 32 bits and the divisions are 32-bit ones (a 64-bit division is several times longer).
__device__ __forceinline__ void cell_coords(long long i, int nx, int ny, int& x, int& y, int& z) {
    const unsigned u = (unsigned)i, q = u / (unsigned)nx;
    x = (int)(u - q * (unsigned)nx);
    z = (int)(q / (unsigned)ny);
    y = (int)(q - (unsigned)z * (unsigned)ny);
}

// neighbour index along an axis; at a wall the index is clamped (its face coupling is 0)
__device__ __forceinline__ int up(int c, int n, int per) { return c + 1 < n ? c + 1 : (per ? 0 : c); }
__device__ __forceinline__ int dn(int c, int n, int per) { return c > 0 ? c - 1 : (per ? n - 1 : c); }

template <int NS>
__device__ void block_sums(double (&v)[NS], double* partials) {
    __shared__ double sh[NS][kBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        double s = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) sh[k][warp] = s;
    }
    __syncthreads();
    if (threadIdx.x < NS) {
        double s = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) s += sh[threadIdx.x][w];
        partials[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
    }
}

struct Stencil {
    long long xm, xp, ym, yp, zm, zp;
    double wxm, wxp, wym, wyp, wzm, wzp;
};

__device__ __forceinline__ Stencil stencil(long long i, int x, int y, int z, int nx, int ny, int nz, const int* per,
                                           const double* __restrict__ wx, const double* __restrict__ wy,
                                           const double* __restrict__ wz) {
    Stencil s;
    const long long sy = nx, sz = (long long)nx * ny;
    const long long b = i - x - (long long)y * sy - (long long)z * sz;
    s.xm = b + dn(x, nx, per[0]) + y * sy + z * sz;
    s.xp = b + up(x, nx, per[0]) + y * sy + z * sz;
    s.ym = b + x + dn(y, ny, per[1]) * sy + z * sz;
    s.yp = b + x + up(y, ny, per[1]) * sy + z * sz;
    s.zm = b + x + y * sy + dn(z, nz, per[2]) * sz;
    s.zp = b + x + y * sy + up(z, nz, per[2]) * sz;
    s.wxp = wx[i];
    s.wyp = wy[i];
    s.wzp = wz[i];
    s.wxm = (!per[0] && x == 0) ? 0.0 : wx[s.xm];
    s.wym = (!per[1] && y == 0) ? 0.0 : wy[s.ym];
    s.wzm = (!per[2] && z == 0) ? 0.0 : wz[s.zm];
    return s;
}

}  // namespace cellgrid
