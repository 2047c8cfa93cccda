// rt_residual_static: the residual evaluation of rt_residual for callers that cannot allocate
// device memory.  Some callers run where cudaMalloc is not available to them: code embedded in
// a larger application that owns the whole device memory budget through its own pool (a
// library's own cudaMalloc there fails or fragments that budget), or real-time loops that
// forbid the device-wide synchronisation cudaMalloc and cudaFree may cause.  This entry point
// needs no grid handle (rt_init_grid allocates its workspace) and calls no cudaMalloc,
// cudaFree or allocating library routine.  Its scratch memory is the file-scope device array
// below, which every GPU that loads the library keeps until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/rt.h"
#include "kernels.cuh"

int rt_internal_step_params(const rt_grid_desc* desc, const rt_step_inputs* in, PhysParams* out);
const char* rt_internal_set_detail(const char* msg);

namespace {

constexpr long long kMaxCells = RT_RESIDUAL_STATIC_MAX_CELLS;
// per-cell scratch: 4 pi eta, b_E, three face couplings, and the initial iterate the setup
// kernel writes alongside b_E (E, n_HI, e_c); then the reduction partials and an error flag
constexpr long long kPerCellArrays = 8;
constexpr long long kPartials = RT_RED_SLOTS * RT_MAX_PARTIALS;
constexpr long long kScratchDoubles = kPerCellArrays * kMaxCells + kPartials + 1;

static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_addr[kMaxDevices] = {};   // device address of g_scratch, per device

// The address of g_scratch on the current device.  In host code the name g_scratch is only a
// host-side stand-in, so the device address is looked up once per device with that device
// current (the first call on the device) and cached; the cache is not refreshed after a
// cudaDeviceReset, so calls after a reset are not supported.
int scratch_for_device(int dev, double** out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            rt_internal_set_detail("cudaGetSymbolAddress of the static scratch array failed");
            return RT_ECUDA;
        }
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return RT_OK;
}

int residual_on_device(const rt_grid_desc* desc, const rt_step_inputs* in, const rt_state* U_n, const rt_state* U,
                       double* f_e, double* f_n, double* f_E, const PhysParams& P);

}  // namespace

extern "C" int rt_residual_static(const rt_grid_desc* desc, const rt_step_inputs* in, const rt_state* U_n,
                                  const rt_state* U, double* f_e, double* f_n, double* f_E) {
    if (!desc || !in || !U_n || !U || !U_n->E || !U_n->n_HI || !U->E || !U->n_HI || !U->e_c || !f_e || !f_n ||
        !f_E) {
        rt_internal_set_detail("null argument");
        return RT_EINVAL;
    }
    if (desc->helium) {
        rt_internal_set_detail("rt_residual_static covers hydrogen-only grids");
        return RT_EINVAL;
    }
    const long long n = (long long)desc->nx * desc->ny * desc->nz;
    if (desc->nx < 1 || desc->ny < 1 || desc->nz < 1 || n > kMaxCells) {
        rt_internal_set_detail("rt_residual_static takes at most RT_RESIDUAL_STATIC_MAX_CELLS cells");
        return RT_EINVAL;
    }
    if (desc->device < 0 || desc->device >= kMaxDevices) {
        rt_internal_set_detail("rt_residual_static: device ordinal outside 0..63");
        return RT_EINVAL;
    }
    PhysParams P;
    int rc = rt_internal_step_params(desc, in, &P);
    if (rc) return rc;
    // the caller's current device is put back before returning
    int prev_dev = 0;
    if (cudaGetDevice(&prev_dev) != cudaSuccess) {
        rt_internal_set_detail("cudaGetDevice failed");
        return RT_ECUDA;
    }
    if (cudaSetDevice(desc->device) != cudaSuccess) {
        rt_internal_set_detail("cudaSetDevice failed");
        return RT_ECUDA;
    }
    rc = residual_on_device(desc, in, U_n, U, f_e, f_n, f_E, P);
    if (cudaSetDevice(prev_dev) != cudaSuccess && rc == RT_OK) {
        rt_internal_set_detail("cudaSetDevice could not restore the caller's device");
        rc = RT_ECUDA;
    }
    return rc;
}

namespace {

int residual_on_device(const rt_grid_desc* desc, const rt_step_inputs* in, const rt_state* U_n, const rt_state* U,
                       double* f_e, double* f_n, double* f_E, const PhysParams& P) {
    const long long n = (long long)desc->nx * desc->ny * desc->nz;
    double* base = nullptr;
    int rc = scratch_for_device(desc->device, &base);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)desc->stream;
    double* src = base;
    double* bE = base + 1 * kMaxCells;
    double* wx = base + 2 * kMaxCells;
    double* wy = base + 3 * kMaxCells;
    double* wz = base + 4 * kMaxCells;
    double* Ei = base + 5 * kMaxCells;
    double* ni = base + 6 * kMaxCells;
    double* eci = base + 7 * kMaxCells;
    double* partials = base + kPerCellArrays * kMaxCells;
    int* err = reinterpret_cast<int*>(base + kPerCellArrays * kMaxCells + kPartials);

    // the array keeps the previous call's contents: the error flag and the emissivity sum
    // must start at zero; every other scratch value is written before it is read
    if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) return RT_ECUDA;
    launch_zero(src, n, s);
    launch_scatter_sources(src, in->src_cell, in->src_ndot, in->nsrc, P.src_scale, n, err, s);
    launch_faces(P, U_n->E, U_n->n_HI, wx, wy, wz, nullptr, nullptr, nullptr, s);
    const HydroIn hy = {in->rho_b, in->e_h, in->vx, in->vy, in->vz};
    launch_setup(P, U_n->E, U_n->n_HI, src, wx, wy, wz, bE, Ei, ni, eci, partials, hy, err, s);
    AssembleArgs A;
    std::memset(&A, 0, sizeof(A));
    A.E_cur = U->E;
    A.n_given = U->n_HI;
    A.ec_given = U->e_c;
    A.E0 = U_n->E;
    A.n0 = U_n->n_HI;
    A.rho = in->rho_b;
    A.e_h = in->e_h;
    A.vx = in->vx;
    A.vy = in->vy;
    A.vz = in->vz;
    A.clump = in->clump;
    A.bE = bE;
    A.src = src;
    A.wx = wx;
    A.wy = wy;
    A.wz = wz;
    A.fE_out = f_E;
    A.fn_out = f_n;
    A.fe_out = f_e;
    A.partials = partials;
    launch_assemble(P, A, true, s);
    int herr = 0;
    if (cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        rt_internal_set_detail("CUDA error in rt_residual_static");
        return RT_ECUDA;
    }
    if (herr & 1) {
        rt_internal_set_detail("a source cell index is outside the grid");
        return RT_EINVAL;
    }
    if (herr & 2) {
        rt_internal_set_detail("invalid hydro state (density, energy or internal energy)");
        return RT_EINVAL;
    }
    if (cudaGetLastError() != cudaSuccess) {
        rt_internal_set_detail("kernel launch failed in rt_residual_static");
        return RT_ECUDA;
    }
    return RT_OK;
}

}  // namespace
