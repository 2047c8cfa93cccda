// C ABI and host driver of the implicit step (see include/rt.h).
//
// Per call of rt_implicit_step:
//   setup   : sources -> 4 pi eta, lagged face couplings (Eq. limiter at the step start),
//             explicit part b_E of Eq. radiation_residual, initial iterate;
//   Newton  : k_assemble evaluates the trial E_k + lam s with the exact local solution
//             (nonlinear elimination of (e_c, n_HI)), the residual norm (Eq. rmsnorm) and
//             the Schur system; backtracking (Armijo, halving) on the norm; the reduced
//             system S s = -f_E is solved by flexible CG (FP64) preconditioned with one
//             multigrid V-cycle in FP32 (RT_MIXED) or FP64 (RT_FP64).
//   The host reads one norm per Newton evaluation and one residual norm per CG iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/rt.h"
#include "kernels.cuh"

namespace {

// CGS constants used by the library's unit factors and spectral averages
constexpr double kC = 2.99792458e10;
constexpr double kKB = 1.380649e-16;
constexpr double kEV = 1.602176634e-12;
constexpr double kMH = 1.6735575e-24;
constexpr double kGamma = 5.0 / 3.0;
constexpr double kHnu0 = 13.6 * kEV;
constexpr double kSigma0 = 6.3e-18;
constexpr double kAlphaB = 2.59e-13;
// helium: thresholds, threshold cross sections (HeI: Osterbrock's two-term power law)
constexpr double kHnuHeI = 24.59 * kEV, kHnuHeII = 54.42 * kEV;
constexpr double kSigmaHeI = 7.83e-18, kBetaHeI = 1.66, kSHeI = 2.05, kSigmaHeII = 1.58e-18;

thread_local char g_detail[512] = "";

void set_detail(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_detail, sizeof(g_detail), fmt, ap);
    va_end(ap);
}

// ---------------------------------------------------------------- spectral averages
// int_{x0}^{inf} f(x) / (e^x - 1) dx by composite 16-point Gauss-Legendre on panels of
// width 0.25 out to x0 + 80 (the integrand falls as e^-x).
template <class F>
double bose_integral(F f, double x0) {
    static const double gx[8] = {0.0950125098376374, 0.2816035507792589, 0.4580167776572274, 0.6178762444026438,
                                 0.7554044083550030, 0.8656312023878318, 0.9445750230732326, 0.9894009349916499};
    static const double gw[8] = {0.1894506104550685, 0.1826034150449236, 0.1691565193950025, 0.1495959888165767,
                                 0.1246289712555339, 0.0951585116824928, 0.0622535239386479, 0.0271524594117541};
    const double h = 0.25;
    double total = 0.0;
    for (int p = 0; p < 320; ++p) {
        const double a = x0 + p * h, mid = a + 0.5 * h, half = 0.5 * h;
        double s = 0.0;
        for (int k = 0; k < 8; ++k) {
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                const double x = mid + sgn * half * gx[k];
                s += gw[k] * f(x) * std::exp(-x) / (-std::expm1(-x));
            }
        }
        total += s * half;
    }
    return total;
}
double w_x3(double x) { return x * x * x; }
double w_x2(double x) { return x * x; }
double w_1(double) { return 1.0; }
double w_xm1(double x) { return 1.0 / x; }

struct Grey {
    double sigma_E, sigma_G, eps_src;
};

Grey grey_constants(int spectrum, double T_B) {
    Grey g;
    if (spectrum == RT_SPECTRUM_MONO) {
        g.sigma_E = kSigma0;
        g.sigma_G = kSigma0 / kHnu0;
        g.eps_src = kHnu0;
        return g;
    }
    const double kT = kKB * T_B, x0 = kHnu0 / kT;
    const double e3 = bose_integral(w_x3, x0), e2 = bose_integral(w_x2, x0);
    const double s0 = bose_integral(w_1, x0), sm1 = bose_integral(w_xm1, x0);
    g.sigma_E = kSigma0 * x0 * x0 * x0 * s0 / e3;
    g.sigma_G = kSigma0 * x0 * x0 * x0 * sm1 / (kT * e3);
    g.eps_src = kT * e3 / e2;
    return g;
}

// grey constants of HeI and HeII over the same spectrum (normalised by the energy above the
// hydrogen edge): sigma_E,i and sigma_G,i; zero for the 13.6 eV line
struct GreyHe {
    double sE1, sG1, sE2, sG2;
};

GreyHe helium_grey_constants(int spectrum, double T_B) {
    GreyHe h = {0.0, 0.0, 0.0, 0.0};
    if (spectrum == RT_SPECTRUM_MONO) return h;
    const double kT = kKB * T_B, x0 = kHnu0 / kT, x1 = kHnuHeI / kT, x2 = kHnuHeII / kT;
    const double e3 = bose_integral(w_x3, x0);
    auto s1 = [x1](double x) {
        return kSigmaHeI * (kBetaHeI * std::pow(x1 / x, kSHeI) + (1.0 - kBetaHeI) * std::pow(x1 / x, kSHeI + 1.0));
    };
    h.sE1 = bose_integral([&](double x) { return s1(x) * x * x * x; }, x1) / e3;
    h.sG1 = bose_integral([&](double x) { return s1(x) * x * x; }, x1) / (kT * e3);
    h.sE2 = kSigmaHeII * x2 * x2 * x2 * bose_integral(w_1, x2) / e3;
    h.sG2 = kSigmaHeII * x2 * x2 * x2 * bose_integral(w_xm1, x2) / (kT * e3);
    return h;
}

// ------------------------------------------------------------------ device buffers

template <class T>
T* dalloc(size_t n, bool& ok) {
    void* p = nullptr;
    if (n == 0) n = 1;
    if (cudaMalloc(&p, n * sizeof(T)) != cudaSuccess) {
        ok = false;
        return nullptr;
    }
    // workspace starts at zero so that no run depends on what earlier allocations left behind
    if (cudaMemset(p, 0, n * sizeof(T)) != cudaSuccess) ok = false;
    return static_cast<T*>(p);
}

template <class T>
struct Hierarchy {
    std::vector<Level<T>> lv;   // lv[0] is the fine level; the last one goes to the tail solver
    std::vector<void*> owned;
};

}  // namespace

struct rt_grid {
    rt_grid_desc desc;
    Dims dims;
    long long n;
    cudaStream_t stream;
    Grey grey;
    PhysParams base;          // step-independent constants
    double u_x, u_t, u_g, u_d, u_v, u_E, u_n;
    // per-step inputs and state copies
    double *E0, *n0, *src, *bE;
    double *wx, *wy, *wz;     // FP64 face couplings
    float *wxf, *wyf, *wzf;   // FP32 copies for the mixed multigrid
    // Newton iterates (current / trial) and the reduced system
    double *Ec, *nc, *ecc, *Et, *nt, *ect;
    double *step, *diag, *rhs, *wE;
    double *Xec, *Xnc, *Xet, *Xnt;   // local-elimination sensitivities (current / trial)
    double *He10, *He20, *He1c, *He2c, *He1t, *He2t;   // helium: start, current, trial (n_HeI, n_HeII)
    // CG vectors
    double *x, *r, *z, *p, *q;
    // multigrid
    Hierarchy<float> mgf;
    Hierarchy<double> mgd;
    float *bf, *xf;           // FP32 level-0 right side / solution (mixed), multigrid order
    double *bs, *xs;          // FP64 level-0 right side / solution in colour-split order
    // reductions
    double *partials, *dots, *scal;
    int* d_err;
    double* h_pinned;
    int launches;
    bool schur_ready;
    // per-kernel profiling (rt_set_profiling)
    bool prof_on;
    std::vector<cudaEvent_t> ev;      // pool: pairs (start, stop)
    size_t ev_used;
    std::vector<int> ev_cls;
    std::vector<double> ev_bytes;
    double prof_ms[32], prof_bytes[32];
    int prof_cnt[32];
};

namespace {

#define RT_CUDA(call)                                                                             \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            set_detail("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
            return RT_ECUDA;                                                                      \
        }                                                                                         \
    } while (0)

int check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_detail("%s: %s", what, cudaGetErrorString(e));
        return RT_ECUDA;
    }
    return RT_OK;
}

enum KClass {
    K_ZERO, K_SOURCES, K_FACES, K_SETUP, K_ASSEMBLE, K_FINALIZE, K_SPMV, K_RESNORM, K_CG_UPDATE, K_DOT2, K_P_UPDATE,
    K_SCALARS, K_COPY, K_CAST, K_MG_DIAG, K_COARSEN, K_RBGS, K_RESTRICT, K_PROLONG, K_TAIL, K_ADD, K_ADVECT,
    K_ADVECT_CHECK, K_RBGS_FINE, K_NCLASS
};
const char* kClassName[K_NCLASS] = {"zero", "scatter_sources", "faces", "setup", "newton_assemble", "finalize",
                                    "cg_spmv_dot", "cg_residual", "cg_update_xr", "cg_dot2", "cg_p_update",
                                    "cg_scalars", "copy", "cast", "mg_diag", "mg_coarsen", "mg_rbgs",
                                    "mg_resid_restrict", "mg_prolong_add", "mg_coarse_cta", "add", "advect",
                                    "advect_courant", "mg_rbgs_fine"};

// Launch f() as kernel class cls moving `bytes` algorithmic bytes; brackets it with events
// when profiling is on.
template <class F>
void run(rt_grid* g, int cls, double bytes, F&& f) {
    size_t k = 0;
    if (g->prof_on) {
        k = g->ev_used++;
        if (2 * g->ev_used > g->ev.size()) {
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            g->ev.push_back(a);
            g->ev.push_back(b);
            g->ev_cls.push_back(0);
            g->ev_bytes.push_back(0.0);
        }
        g->ev_cls[k] = cls;
        g->ev_bytes[k] = bytes;
        cudaEventRecord(g->ev[2 * k], g->stream);
    }
    f();
    g->launches++;
    if (g->prof_on) cudaEventRecord(g->ev[2 * k + 1], g->stream);
}

// fold recorded launches into the totals; the stream must have been synchronised
void harvest(rt_grid* g) {
    for (size_t k = 0; k < g->ev_used; ++k) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, g->ev[2 * k], g->ev[2 * k + 1]);
        g->prof_ms[g->ev_cls[k]] += ms;
        g->prof_bytes[g->ev_cls[k]] += g->ev_bytes[k];
        g->prof_cnt[g->ev_cls[k]] += 1;
    }
    g->ev_used = 0;
}

enum HierarchyStatus { HIER_OK = 0, HIER_ODD, HIER_NOMEM };

// lv[0] takes diag0 (freed with the grid) whatever the outcome.  Every level but the last is
// smoothed and gets the colour-split copy of its operator (dinv, w6).
template <class T>
HierarchyStatus build_hierarchy(rt_grid* g, Hierarchy<T>& H, T* diag0, T* wx0, T* wy0, T* wz0) {
    bool ok = true;
    Dims d = g->dims;
    Level<T> L{};
    L.d = d;
    L.diag = diag0;
    L.wx = wx0;
    L.wy = wy0;
    L.wz = wz0;
    L.x = nullptr;   // level 0 vectors are bound per solve
    L.b = nullptr;
    H.lv.push_back(L);
    while (d.n() > TailMax<T>::value) {
        if (d.nx % 2 || d.ny % 2 || d.nz % 2) return HIER_ODD;
        d.nx /= 2;
        d.ny /= 2;
        d.nz /= 2;
        Level<T> c{};
        c.d = d;
        const size_t n = (size_t)d.n();
        c.diag = dalloc<T>(n, ok);
        c.wx = dalloc<T>(n, ok);
        c.wy = dalloc<T>(n, ok);
        c.wz = dalloc<T>(n, ok);
        c.x = dalloc<T>(n, ok);
        c.b = dalloc<T>(n, ok);
        for (void* p : {(void*)c.diag, (void*)c.wx, (void*)c.wy, (void*)c.wz, (void*)c.x, (void*)c.b}) H.owned.push_back(p);
        if (!ok) return HIER_NOMEM;
        H.lv.push_back(c);
    }
    for (size_t l = 0; l + 1 < H.lv.size(); ++l) {
        Level<T>& s = H.lv[l];
        const size_t n = (size_t)s.d.n();
        s.split = 1;
        s.dinv = dalloc<T>(n, ok);
        s.w6 = dalloc<T>(3 * n, ok);
        H.owned.push_back(s.dinv);
        H.owned.push_back(s.w6);
        if (!ok) return HIER_NOMEM;
    }
    return HIER_OK;
}

template <class T>
void free_hierarchy(Hierarchy<T>& H) {
    for (void* p : H.owned) cudaFree(p);
    H.owned.clear();
    H.lv.clear();
}

template <class T>
void mg_setup(rt_grid* g, Hierarchy<T>& H) {
    for (size_t l = 1; l < H.lv.size(); ++l) {
        const double fine = (double)H.lv[l - 1].d.n();
        run(g, K_COARSEN, fine * 4.5 * sizeof(T), [&] { launch_coarsen<T>(H.lv[l - 1], H.lv[l], g->stream); });
    }
    for (size_t l = 0; l + 1 < H.lv.size(); ++l) {
        const double n = (double)H.lv[l].d.n();
        run(g, K_COARSEN, n * 8 * sizeof(T), [&] { launch_split_level<T>(H.lv[l], g->stream); });
    }
}

// nu red-black Gauss-Seidel sweeps of level L in place (first colour `first`); the first from a
// zero iterate when `zero`
template <class T>
void smooth_inplace(rt_grid* g, Level<T>& L, int nu, int first, bool zero, int cls) {
    const double n = (double)L.d.n(), t = sizeof(T);
    for (int k = 0; k < nu; ++k) {
        const bool z0 = zero && k == 0;
        // algorithmic words per cell of a sweep: b, diag, wx, wy, wz and x read once, x written
        // once (no read of x from a zero iterate)
        const double words = z0 ? 6.0 : 7.0;
        int nl = 1;
        run(g, cls, n * words * t, [&] { nl = launch_rbgs_inplace<T>(L, first, z0, g->stream); });
        g->launches += nl - 1;
    }
}

// one V-cycle on the hierarchy: level-0 b and x must be bound; the result is left in level 0's x
template <class T>
void vcycle(rt_grid* g, Hierarchy<T>& H) {
    const int nu1 = g->desc.mg_nu1, nu2 = g->desc.mg_nu2;
    const int last = (int)H.lv.size() - 1;
    cudaStream_t s = g->stream;
    const double t = sizeof(T);
    for (int l = 0; l < last; ++l) {
        const double n = (double)H.lv[l].d.n();
        const int cls = l == 0 ? K_RBGS_FINE : K_RBGS;   // the fine level timed on its own
        smooth_inplace<T>(g, H.lv[l], nu1, 0, true, cls);
        run(g, K_RESTRICT, n * 6.125 * t, [&] { launch_resid_restrict<T>(H.lv[l], H.lv[l + 1], s); });
    }
    run(g, K_TAIL, (double)H.lv[last].d.n() * 6 * t, [&] { launch_tail<T>(H.lv[last], 1, std::max(nu1, 1), s); });
    for (int l = last - 1; l >= 0; --l) {
        const double n = (double)H.lv[l].d.n();
        const int cls = l == 0 ? K_RBGS_FINE : K_RBGS;
        // fine x read and written, the coarse correction read (1/8 word per fine cell)
        run(g, K_PROLONG, n * 2.125 * t, [&] { launch_prolong_add<T>(H.lv[l + 1], H.lv[l], s); });
        smooth_inplace<T>(g, H.lv[l], nu2, 1, false, cls);
    }
}

// z = M^{-1} r into g->z
void precondition(rt_grid* g, const double* r) {
    cudaStream_t s = g->stream;
    const double n = (double)g->n;
    if (g->desc.precision == RT_MIXED) {
        // r is scaled by a power of two (from max|r| in dots[1], left there by the residual
        // update) so that the FP32 copy neither overflows nor underflows; z is scaled back
        const double* amax = g->dots + 1;
        Level<float>& L0 = g->mgf.lv[0];
        run(g, K_CAST, n * 12, [&] { launch_to_level<double, float>(g->dims, L0.split, r, g->bf, amax, s); });
        L0.b = g->bf;
        L0.x = g->xf;
        vcycle<float>(g, g->mgf);
        run(g, K_CAST, n * 12, [&] { launch_from_level<float, double>(g->dims, L0.split, g->xf, g->z, amax, s); });
    } else {
        Level<double>& L0 = g->mgd.lv[0];
        if (L0.split) {
            run(g, K_CAST, n * 16, [&] { launch_to_level<double, double>(g->dims, 1, r, g->bs, nullptr, s); });
            L0.b = g->bs;
            L0.x = g->xs;
        } else {
            L0.b = const_cast<double*>(r);
            L0.x = g->z;
        }
        vcycle<double>(g, g->mgd);
        if (L0.split)
            run(g, K_CAST, n * 16, [&] { launch_from_level<double, double>(g->dims, 1, g->xs, g->z, nullptr, s); });
    }
}

int read_scalars(rt_grid* g, int nb, int nslots, double* out, int nmax = 0) {
    run(g, K_FINALIZE, 0.0, [&] { launch_finalize_ext(g->partials, nb, nslots, nmax, g->dots, g->stream); });
    nslots += nmax;
    RT_CUDA(cudaMemcpyAsync(g->h_pinned, g->dots, sizeof(double) * nslots, cudaMemcpyDeviceToHost, g->stream));
    RT_CUDA(cudaStreamSynchronize(g->stream));
    for (int k = 0; k < nslots; ++k) out[k] = g->h_pinned[k];
    return check_launch("reduction");
}

// Flexible preconditioned CG on the operator in (diag, wx, wy, wz) (FP64): solves S x = b from
// the guess in x; stops when ||w r|| <= rtol ||w r0|| (w = weights or 1).
int pcg(rt_grid* g, const double* b, double* x, const double* w, double rtol, int maxit, int* iters) {
    cudaStream_t s = g->stream;
    const long long n = g->n;
    const double N = (double)n;
    const double wb = w ? 8.0 : 0.0;
    *iters = 0;
    int nb = 0;
    run(g, K_RESNORM, N * (56 + wb),
        [&] { nb = launch_residual_norm(g->dims, g->diag, g->wx, g->wy, g->wz, b, x, g->r, w, g->partials, s); });
    double v[2];
    int rc = read_scalars(g, nb, 1, v, 1);
    if (rc) return rc;
    const double rn0 = std::sqrt(v[0]);
    if (!std::isfinite(rn0)) {
        set_detail("non-finite right side in the linear solve");
        return RT_ENONFINITE;
    }
    if (rn0 == 0.0) return RT_OK;
    precondition(g, g->r);
    run(g, K_DOT2, N * 16, [&] { nb = launch_dot2(n, g->z, g->r, nullptr, g->partials, s); });
    run(g, K_FINALIZE, 0.0, [&] { launch_finalize(g->partials, nb, 2, g->dots, s); });
    run(g, K_SCALARS, 0.0, [&] { launch_cg_scalars(g->scal, g->dots, 0, s); });
    run(g, K_COPY, N * 16, [&] { launch_copy(n, g->z, g->p, s); });
    run(g, K_SPMV, N * 48, [&] { nb = launch_spmv_dot(g->dims, g->diag, g->wx, g->wy, g->wz, g->p, g->q, g->partials, s); });
    run(g, K_FINALIZE, 0.0, [&] { launch_finalize(g->partials, nb, 1, g->dots, s); });
    run(g, K_SCALARS, 0.0, [&] { launch_cg_scalars(g->scal, g->dots, 1, s); });
    for (int k = 1; k <= maxit; ++k) {
        run(g, K_CG_UPDATE, N * (48 + wb),
            [&] { nb = launch_cg_update_xr(n, g->scal, x, g->r, g->p, g->q, w, g->partials, s); });
        rc = read_scalars(g, nb, 1, v, 1);
        if (rc) return rc;
        *iters = k;
        const double rn = std::sqrt(v[0]);
        if (!std::isfinite(rn)) {
            double sc[4] = {0, 0, 0, 0};
            cudaMemcpy(sc, g->scal, sizeof(sc), cudaMemcpyDeviceToHost);
            set_detail("non-finite residual in CG iteration %d (alpha %g, beta %g, (z,r) %g, (p,q) %g, |r0| %g)", k,
                       sc[0], sc[1], sc[2], sc[3], rn0);
            return RT_ENONFINITE;
        }
        if (rn <= rtol * rn0) return RT_OK;
        if (k == maxit) break;
        precondition(g, g->r);
        run(g, K_DOT2, N * 24, [&] { nb = launch_dot2(n, g->z, g->r, g->q, g->partials, s); });
        run(g, K_FINALIZE, 0.0, [&] { launch_finalize(g->partials, nb, 2, g->dots, s); });
        run(g, K_SCALARS, 0.0, [&] { launch_cg_scalars(g->scal, g->dots, 2, s); });
        run(g, K_P_UPDATE, N * 24, [&] { launch_p_update(n, g->scal, g->z, g->p, s); });
        run(g, K_SPMV, N * 48,
            [&] { nb = launch_spmv_dot(g->dims, g->diag, g->wx, g->wy, g->wz, g->p, g->q, g->partials, s); });
        run(g, K_FINALIZE, 0.0, [&] { launch_finalize(g->partials, nb, 1, g->dots, s); });
        run(g, K_SCALARS, 0.0, [&] { launch_cg_scalars(g->scal, g->dots, 1, s); });
    }
    set_detail("CG reached %d iterations without the requested reduction", maxit);
    return RT_ELINEAR;
}

void bind_operator_levels(rt_grid* g) {
    // level 0 of the multigrid hierarchy: the FP64 face couplings (FP64 path) or their FP32
    // copies written by k_faces (mixed path), and the diagonal max(diag, sum w)
    const double n = (double)g->n;
    if (g->desc.precision == RT_MIXED) {
        run(g, K_MG_DIAG, n * 36,
            [&] { launch_mg_diag<float>(g->dims, g->diag, g->wx, g->wy, g->wz, g->mgf.lv[0].diag, g->stream); });
        mg_setup<float>(g, g->mgf);
    } else {
        run(g, K_MG_DIAG, n * 40,
            [&] { launch_mg_diag<double>(g->dims, g->diag, g->wx, g->wy, g->wz, g->mgd.lv[0].diag, g->stream); });
        mg_setup<double>(g, g->mgd);
    }
}

int validate_inputs(const rt_grid* g, const rt_step_inputs* in) {
    if (!in || !in->rho_b || !in->e_h) {
        set_detail("rho_b and e_h are required");
        return RT_EINVAL;
    }
    if (!(in->a > 0.0) || !(in->dt > 0.0) || !std::isfinite(in->adot)) {
        set_detail("need a > 0, dt > 0 and finite adot (a=%g dt=%g adot=%g)", in->a, in->dt, in->adot);
        return RT_EINVAL;
    }
    if (in->nsrc < 0 || (in->nsrc > 0 && (!in->src_cell || !in->src_ndot))) {
        set_detail("invalid source list");
        return RT_EINVAL;
    }
    return RT_OK;
}

// per-step values of PhysParams: expansion, step length, face-coupling scale
void apply_step(PhysParams& P, const rt_grid_desc& d, const rt_step_inputs* in) {
    P.a = in->a;
    P.a3 = in->a * in->a * in->a;
    P.H = in->adot / in->a;
    P.dt = in->dt;
    P.adx = in->a * d.dx;
    P.wscale = in->dt * d.theta / (P.adx * P.adx);
    const double x = 2.0 * P.H * in->dt;
    P.phi_e = in->dt * (std::fabs(x) < 1e-8 ? 1.0 - 0.5 * x + x * x / 6.0 : -std::expm1(-x) / x);
    // the local equations are solved three orders of magnitude below the Newton tolerance
    P.local_tol = std::max(1e-14, 1e-3 * d.newton_tol);
}

PhysParams step_params(const rt_grid* g, const rt_step_inputs* in) {
    PhysParams P = g->base;
    apply_step(P, g->desc, in);
    return P;
}

// Checks of the descriptor's geometry, units, theta and boundaries (every entry point that
// takes a descriptor); sets the detail text and returns RT_EINVAL on the first failure.
int check_geometry(const rt_grid_desc& d) {
    if (d.nx < 1 || d.ny < 1 || d.nz < 1 || !(d.dx > 0) || !(d.u_x > 0) || !(d.u_t > 0) || !(d.u_g > 0)) {
        set_detail("grid dims, dx and unit factors must be positive");
        return RT_EINVAL;
    }
    if (!(d.theta > 0.0 && d.theta <= 1.0)) {
        set_detail("theta must lie in (0, 1]");
        return RT_EINVAL;
    }
    for (int f = 0; f < 6; ++f)
        if (d.bc[f] != RT_BC_PERIODIC && d.bc[f] != RT_BC_REFLECT && d.bc[f] != RT_BC_OUTFLOW) {
            set_detail("unknown boundary type on face %d", f);
            return RT_EINVAL;
        }
    for (int k = 0; k < 3; ++k)
        if ((d.bc[2 * k] == RT_BC_PERIODIC) != (d.bc[2 * k + 1] == RT_BC_PERIODIC)) {
            set_detail("axis %d: periodic on one face only", k);
            return RT_EINVAL;
        }
    return RT_OK;
}

// Step-independent PhysParams of a descriptor: unit factors (Eqs. units, scalings), the grey
// constants of Eq. grey_definition in normalised units, boundaries and physics switches.
PhysParams base_params(const rt_grid_desc& d, const Grey& grey) {
    const double u_d = d.u_g / (d.u_x * d.u_x * d.u_x), u_v = d.u_x / d.u_t;
    const double u_E = u_d * u_v * u_v, u_n = u_d / kMH;
    PhysParams P;
    std::memset(&P, 0, sizeof(P));
    P.nx = d.nx;
    P.ny = d.ny;
    P.nz = d.nz;
    for (int k = 0; k < 3; ++k) P.per[k] = d.bc[2 * k] == RT_BC_PERIODIC;
    for (int f = 0; f < 6; ++f) P.outflow[f] = d.bc[f] == RT_BC_OUTFLOW;
    P.dx = d.dx;
    P.theta = d.theta;
    P.c = kC * d.u_t / d.u_x;
    P.kE = grey.sigma_E * u_n * d.u_x;
    P.kG = kC * grey.sigma_G * u_E * d.u_t;
    P.kA = d.u_t * u_n;
    P.kH = kC * u_n * (grey.sigma_E - kHnu0 * grey.sigma_G) * d.u_t;
    P.kC = d.u_t / u_E;
    P.kT = (kGamma - 1.0) * u_v * u_v * kMH / kKB;
    P.un = u_n;
    P.E_min = (d.E_min > 0 ? d.E_min : 1e-35) / u_E;
    P.E_floor = P.E_min;
    P.e_floor = kKB * 1.0 / ((kGamma - 1.0) * kMH) / (u_v * u_v);
    P.T_iso = d.T_iso;
    P.D_const = d.D_const * d.u_t / (d.u_x * d.u_x);
    P.src_scale = grey.eps_src * d.u_t / (d.u_x * d.u_x * d.u_x * u_E * d.dx * d.dx * d.dx);
    P.alpha_const = kAlphaB;
    P.isothermal = d.isothermal;
    P.helium = d.helium;
    P.Y = d.helium ? d.Y : 0.0;
    if (d.helium) {
        const GreyHe h = helium_grey_constants(d.spectrum, d.T_B);
        P.kE1 = h.sE1 * u_n * d.u_x;
        P.kE2 = h.sE2 * u_n * d.u_x;
        P.kG1 = kC * h.sG1 * u_E * d.u_t;
        P.kG2 = kC * h.sG2 * u_E * d.u_t;
        P.kH1 = kC * u_n * (h.sE1 - kHnuHeI * h.sG1) * d.u_t;
        P.kH2 = kC * u_n * (h.sE2 - kHnuHeII * h.sG2) * d.u_t;
    }
    P.recomb = d.recomb;
    P.cooling = d.cooling;
    P.limiter = d.limiter;
    return P;
}

bool has_outflow(const rt_grid_desc& d) {
    for (int f = 0; f < 6; ++f)
        if (d.bc[f] == RT_BC_OUTFLOW) return true;
    return false;
}

// sources, faces, explicit part, initial iterate into (Ec, nc, ecc); sets P.E_floor
int step_setup(rt_grid* g, const rt_step_inputs* in, PhysParams& P, const double* E_start,
               const double* n_start, const double* he1_start = nullptr, const double* he2_start = nullptr) {
    cudaStream_t s = g->stream;
    const long long n = g->n;
    RT_CUDA(cudaMemcpyAsync(g->E0, E_start, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    RT_CUDA(cudaMemcpyAsync(g->n0, n_start, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (g->desc.helium) {
        // start copies (their opacity enters D^n and b_E) and the initial iterate's helium
        RT_CUDA(cudaMemcpyAsync(g->He10, he1_start, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        RT_CUDA(cudaMemcpyAsync(g->He20, he2_start, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        RT_CUDA(cudaMemcpyAsync(g->He1c, he1_start, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        RT_CUDA(cudaMemcpyAsync(g->He2c, he2_start, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        P.nHeI0 = g->He10;
        P.nHeII0 = g->He20;
    }
    RT_CUDA(cudaMemsetAsync(g->d_err, 0, sizeof(int), s));
    const double N = (double)n;
    run(g, K_ZERO, N * 8, [&] { launch_zero(g->src, n, s); });
    if (in->nsrc > 0)
        run(g, K_SOURCES, in->nsrc * 24.0, [&] {
            launch_scatter_sources(g->src, in->src_cell, in->src_ndot, in->nsrc, P.src_scale, n, g->d_err, s);
        });
    run(g, K_FACES, N * (g->wxf ? 52 : 40),
        [&] { launch_faces(P, g->E0, g->n0, g->wx, g->wy, g->wz, g->wxf, g->wyf, g->wzf, s); });
    int nb = 0;
    const HydroIn hy = {in->rho_b, in->e_h, in->vx, in->vy, in->vz};
    run(g, K_SETUP, N * (96 + (in->vx ? 24 : 0)), [&] {
        nb = launch_setup(P, g->E0, g->n0, g->src, g->wx, g->wy, g->wz, g->bE, g->Ec, g->nc, g->ecc, g->partials, hy,
                          g->d_err, s);
    });
    run(g, K_FINALIZE, 0.0, [&] { launch_finalize_ext(g->partials, nb, 0, 1, g->dots, s); });
    int herr = 0;
    RT_CUDA(cudaMemcpyAsync(&g->h_pinned[0], g->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    RT_CUDA(cudaMemcpyAsync(&g->h_pinned[1], g->dots, sizeof(double), cudaMemcpyDeviceToHost, s));
    RT_CUDA(cudaStreamSynchronize(s));
    std::memcpy(&herr, &g->h_pinned[0], sizeof(int));
    P.E_floor = std::max(P.E_min, 1e-12 * g->h_pinned[1]);
    if (herr & 1) {
        set_detail("a source cell index is outside the grid");
        return RT_EINVAL;
    }
    if (herr & 2) {
        set_detail("invalid hydro state: a density that is not positive and finite, a non-finite energy, or a "
                   "non-positive internal energy of non-isothermal gas");
        return RT_EINVAL;
    }
    return check_launch("step setup");
}

AssembleArgs base_args(rt_grid* g, const rt_step_inputs* in) {
    AssembleArgs A;
    std::memset(&A, 0, sizeof(A));
    A.E0 = g->E0;
    A.n0 = g->n0;
    A.rho = in->rho_b;
    A.e_h = in->e_h;
    A.vx = in->vx;
    A.vy = in->vy;
    A.vz = in->vz;
    A.clump = in->clump;
    A.bE = g->bE;
    A.src = g->src;
    A.wx = g->wx;
    A.wy = g->wy;
    A.wz = g->wz;
    A.partials = g->partials;
    return A;
}

// Donor-cell advection of (E, n_HI) (or the transposed map on their adjoints): checks the
// Courant bound first, so nothing is written when it fails.
int advect_call(rt_grid* g, const rt_step_inputs* in, const rt_state* src, rt_state* dst, const double* rho_src,
                double* rho_dst, double* courant_max, bool transpose) {
    const bool he = g && g->desc.helium && !transpose;
    if (g && g->desc.helium && transpose) {
        set_detail("the adjoint covers hydrogen-only grids");
        return RT_EINVAL;
    }
    if (he && (!src || !dst || !src->n_HeI || !src->n_HeII || !dst->n_HeI || !dst->n_HeII)) {
        set_detail("helium grid: the advected state needs n_HeI and n_HeII");
        return RT_EINVAL;
    }
    if (!g || !in || !src || !dst || !src->E || !src->n_HI || !dst->E || !dst->n_HI || (!rho_src != !rho_dst)) {
        set_detail("null grid, inputs or state array (rho_src and rho_dst must be both set or both NULL)");
        return RT_EINVAL;
    }
    const long long n = g->n;
    auto overlaps = [n](const double* a, const double* b) { return a && b && a < b + n && b < a + n; };
    const double* reads[5] = {src->E, src->n_HI, rho_src, he ? src->n_HeI : nullptr, he ? src->n_HeII : nullptr};
    const double* writes[5] = {dst->E, dst->n_HI, rho_dst, he ? dst->n_HeI : nullptr, he ? dst->n_HeII : nullptr};
    for (int w = 0; w < 5; ++w) {
        for (int r = 0; r < 5; ++r)
            if (overlaps(writes[w], reads[r])) {
                set_detail("advection source and destination arrays overlap");
                return RT_EINVAL;
            }
        for (int w2 = w + 1; w2 < 5; ++w2)
            if (overlaps(writes[w], writes[w2])) {
                set_detail("advection destination arrays overlap");
                return RT_EINVAL;
            }
    }
    if (!(in->a > 0.0) || !(in->dt >= 0.0) || !std::isfinite(in->a) || !std::isfinite(in->dt)) {
        set_detail("invalid expansion factor or time step (a = %g, dt = %g)", in->a, in->dt);
        return RT_EINVAL;
    }
    if (has_outflow(g->desc)) {
        set_detail("the advection pre-step covers periodic and reflecting faces");
        return RT_EINVAL;
    }
    RT_CUDA(cudaSetDevice(g->desc.device));
    AdvectArgs A;
    std::memset(&A, 0, sizeof(A));
    A.nx = g->desc.nx;
    A.ny = g->desc.ny;
    A.nz = g->desc.nz;
    for (int d = 0; d < 3; ++d) A.per[d] = g->desc.bc[2 * d] == RT_BC_PERIODIC;
    A.k = in->dt / (in->a * g->desc.dx);
    A.v[0] = in->vx;
    A.v[1] = in->vy;
    A.v[2] = in->vz;
    A.qE = src->E;
    A.qn = src->n_HI;
    A.oE = dst->E;
    A.on = dst->n_HI;
    A.qr = rho_src;
    A.orh = rho_dst;
    if (he) {
        A.qh1 = src->n_HeI;
        A.qh2 = src->n_HeII;
        A.oh1 = dst->n_HeI;
        A.oh2 = dst->n_HeII;
    }
    A.partials = g->partials;
    const double N = (double)n;
    const int nv = (in->vx != nullptr) + (in->vy != nullptr) + (in->vz != nullptr);
    int nb = 0;
    run(g, K_ADVECT_CHECK, N * 8.0 * nv, [&] { nb = launch_advect_courant(A, g->stream); });
    double cmax = 0.0;
    int rc = read_scalars(g, nb, 0, &cmax, 1);
    if (rc) return rc;
    if (courant_max) *courant_max = cmax;
    if (!(cmax <= 1.0)) {
        set_detail("advection Courant number %g exceeds 1", cmax);
        return RT_EINVAL;
    }
    run(g, K_ADVECT, N * 8.0 * ((rho_src ? 6 : 4) + (he ? 4 : 0) + nv), [&] { launch_advect(A, transpose, g->stream); });
    if (g->prof_on) {
        RT_CUDA(cudaStreamSynchronize(g->stream));
        harvest(g);
    }
    RT_CUDA(cudaStreamSynchronize(g->stream));
    return check_launch(transpose ? "advection adjoint" : "advection");
}

template <class T>
void swap_ptr(T*& a, T*& b) {
    T* t = a;
    a = b;
    b = t;
}

}  // namespace

extern "C" {

const char* rt_error_string(int code) {
    switch (code) {
        case RT_OK: return "ok";
        case RT_EINVAL: return "invalid argument";
        case RT_ENOMEM: return "device allocation failed";
        case RT_ECUDA: return "CUDA error";
        case RT_ENOCONV: return "Newton iteration did not converge";
        case RT_ELINESEARCH: return "line search failed to reduce the residual";
        case RT_ENONFINITE: return "non-finite value in the solve";
        case RT_ELINEAR: return "linear solver did not converge";
        default: return "unknown error";
    }
}

const char* rt_last_error_detail(void) { return g_detail; }

void rt_destroy_grid(rt_grid* g) {
    if (!g) return;
    cudaSetDevice(g->desc.device);
    double* bufs[] = {g->E0, g->n0, g->src, g->bE, g->wx, g->wy, g->wz, g->Ec, g->nc, g->ecc, g->Et, g->nt, g->ect,
                      g->step, g->diag, g->rhs, g->wE, g->x, g->r, g->z, g->p, g->q, g->partials, g->dots, g->scal,
                      g->Xec, g->Xnc, g->Xet, g->Xnt, g->He10, g->He20, g->He1c, g->He2c, g->He1t, g->He2t};
    for (double* b : bufs) cudaFree(b);
    cudaFree(g->wxf);
    cudaFree(g->wyf);
    cudaFree(g->wzf);
    cudaFree(g->bf);
    cudaFree(g->xf);
    cudaFree(g->bs);
    cudaFree(g->xs);
    cudaFree(g->d_err);
    if (g->mgf.lv.size() > 0) cudaFree(g->mgf.lv[0].diag);
    if (g->mgd.lv.size() > 0) cudaFree(g->mgd.lv[0].diag);
    free_hierarchy(g->mgf);
    free_hierarchy(g->mgd);
    cudaFreeHost(g->h_pinned);
    for (cudaEvent_t e : g->ev) cudaEventDestroy(e);
    delete g;
}

int rt_init_grid(const rt_grid_desc* desc, rt_grid** out) {
    if (!desc || !out) {
        set_detail("null descriptor or output handle");
        return RT_EINVAL;
    }
    *out = nullptr;
    const rt_grid_desc& d = *desc;
    if (check_geometry(d)) return RT_EINVAL;
    if ((d.precision != RT_FP64 && d.precision != RT_MIXED) || d.mg_nu1 < 1 || d.mg_nu2 < 1 || d.max_newton < 1 ||
        d.max_lin < 1 || !(d.newton_tol > 0) || !(d.lin_rtol > 0) || (d.helium != 0 && d.helium != 1) ||
        (d.helium && !(d.Y >= 0.0 && d.Y < 1.0))) {
        set_detail("invalid solver parameters");
        return RT_EINVAL;
    }
    if ((long long)d.nx * d.ny * d.nz > (1LL << 31)) {
        set_detail("grid too large");
        return RT_EINVAL;
    }
    if (cudaSetDevice(d.device) != cudaSuccess) {
        set_detail("cudaSetDevice(%d) failed", d.device);
        return RT_ECUDA;
    }
    rt_grid* g = new (std::nothrow) rt_grid;
    if (!g) return RT_ENOMEM;
    std::memset((void*)g, 0, sizeof(rt_grid));
    new (&g->mgf) Hierarchy<float>();
    new (&g->mgd) Hierarchy<double>();
    new (&g->ev) std::vector<cudaEvent_t>();
    new (&g->ev_cls) std::vector<int>();
    new (&g->ev_bytes) std::vector<double>();
    g->desc = d;
    g->stream = (cudaStream_t)d.stream;
    g->dims.nx = d.nx;
    g->dims.ny = d.ny;
    g->dims.nz = d.nz;
    for (int k = 0; k < 3; ++k) g->dims.per[k] = d.bc[2 * k] == RT_BC_PERIODIC;
    g->n = g->dims.n();
    g->grey = grey_constants(d.spectrum, d.T_B);

    // unit factors (Eqs. units, scalings)
    g->u_x = d.u_x;
    g->u_t = d.u_t;
    g->u_g = d.u_g;
    g->u_d = d.u_g / (d.u_x * d.u_x * d.u_x);
    g->u_v = d.u_x / d.u_t;
    g->u_E = g->u_d * g->u_v * g->u_v;
    g->u_n = g->u_d / kMH;
    g->base = base_params(d, g->grey);

    bool ok = true;
    const size_t n = (size_t)g->n;
    double** fp64[] = {&g->E0, &g->n0, &g->src, &g->bE, &g->wx, &g->wy, &g->wz, &g->Ec, &g->nc, &g->ecc, &g->Et,
                       &g->nt, &g->ect, &g->step, &g->diag, &g->rhs, &g->wE, &g->x, &g->r, &g->z, &g->p, &g->q};
    for (double** b : fp64) *b = dalloc<double>(n, ok);
    if (d.helium) {
        double** he[] = {&g->He10, &g->He20, &g->He1c, &g->He2c, &g->He1t, &g->He2t};
        for (double** b : he) *b = dalloc<double>(n, ok);
    }
    if (!d.isothermal) {
        g->Xec = dalloc<double>(n, ok);
        g->Xnc = dalloc<double>(n, ok);
        g->Xet = dalloc<double>(n, ok);
        g->Xnt = dalloc<double>(n, ok);
    }
    g->partials = dalloc<double>(RT_RED_SLOTS * RT_MAX_PARTIALS, ok);
    g->dots = dalloc<double>(16, ok);
    g->scal = dalloc<double>(16, ok);
    g->d_err = dalloc<int>(4, ok);
    if (cudaMallocHost((void**)&g->h_pinned, 64 * sizeof(double)) != cudaSuccess) ok = false;
    if (ok && d.precision == RT_MIXED) {
        g->wxf = dalloc<float>(n, ok);
        g->wyf = dalloc<float>(n, ok);
        g->wzf = dalloc<float>(n, ok);
        g->bf = dalloc<float>(n, ok);
        g->xf = dalloc<float>(n, ok);
        float* diag0 = dalloc<float>(n, ok);
        if (!ok) {
            cudaFree(diag0);
        } else {
            const HierarchyStatus hs = build_hierarchy<float>(g, g->mgf, diag0, g->wxf, g->wyf, g->wzf);
            if (hs == HIER_ODD) {
                set_detail("grid %dx%dx%d: a level above %d cells has an odd dimension", d.nx, d.ny, d.nz,
                           TailMax<float>::value);
                rt_destroy_grid(g);
                return RT_EINVAL;
            }
            if (hs == HIER_NOMEM) ok = false;
        }
    } else if (ok) {
        double* diag0 = dalloc<double>(n, ok);
        if (!ok) {
            cudaFree(diag0);
        } else {
            const HierarchyStatus hs = build_hierarchy<double>(g, g->mgd, diag0, g->wx, g->wy, g->wz);
            if (hs == HIER_ODD) {
                set_detail("grid %dx%dx%d: a level above %d cells has an odd dimension", d.nx, d.ny, d.nz,
                           TailMax<double>::value);
                rt_destroy_grid(g);
                return RT_EINVAL;
            }
            if (hs == HIER_NOMEM) ok = false;
            if (ok && g->mgd.lv[0].split) {
                g->bs = dalloc<double>(n, ok);
                g->xs = dalloc<double>(n, ok);
            }
        }
    }
    if (!ok) {
        set_detail("device allocation of the workspace failed");
        rt_destroy_grid(g);
        return RT_ENOMEM;
    }
    // the single-CTA coarse solver must fit its shared memory
    {
        const Dims tail_d = d.precision == RT_MIXED ? g->mgf.lv.back().d : g->mgd.lv.back().d;
        const size_t bytes = d.precision == RT_MIXED ? tail_smem_bytes<float>(tail_d) : tail_smem_bytes<double>(tail_d);
        if (bytes > 227 * 1024) {
            set_detail("coarse level %dx%dx%d needs %zu bytes of shared memory", tail_d.nx, tail_d.ny, tail_d.nz, bytes);
            rt_destroy_grid(g);
            return RT_EINVAL;
        }
    }
    *out = g;
    return RT_OK;
}

int rt_spectrum_constants(int spectrum, double T_B, double* out) {
    if (!out || (spectrum != RT_SPECTRUM_MONO && spectrum != RT_SPECTRUM_BLACKBODY) ||
        (spectrum == RT_SPECTRUM_BLACKBODY && !(T_B > 0.0 && T_B < 1e9))) {
        set_detail("rt_spectrum_constants needs an output array and a known spectrum with 0 < T_B < 1e9 K");
        return RT_EINVAL;
    }
    const Grey g = grey_constants(spectrum, T_B);
    const GreyHe h = helium_grey_constants(spectrum, T_B);
    const double v[7] = {g.sigma_E, g.sigma_G, g.eps_src, h.sE1, h.sG1, h.sE2, h.sG2};
    for (int k = 0; k < 7; ++k) out[k] = v[k];
    return RT_OK;
}

int rt_grey_constants(const rt_grid* g, double* sigma_E, double* sigma_G, double* eps_src) {
    if (!g) {
        set_detail("null grid");
        return RT_EINVAL;
    }
    if (sigma_E) *sigma_E = g->grey.sigma_E;
    if (sigma_G) *sigma_G = g->grey.sigma_G;
    if (eps_src) *eps_src = g->grey.eps_src;
    return RT_OK;
}

int rt_implicit_step(rt_grid* g, const rt_step_inputs* in, rt_state* io, rt_step_stats* stats) {
    if (!g || !io || !io->E || !io->n_HI || !io->e_c || (g->desc.helium && (!io->n_HeI || !io->n_HeII))) {
        set_detail("null grid or state array");
        return RT_EINVAL;
    }
    int rc = validate_inputs(g, in);
    if (rc) return rc;
    RT_CUDA(cudaSetDevice(g->desc.device));
    g->launches = 0;
    PhysParams P = step_params(g, in);
    rc = step_setup(g, in, P, io->E, io->n_HI, io->n_HeI, io->n_HeII);
    if (rc) return rc;
    cudaStream_t s = g->stream;
    const long long n = g->n;
    const bool he = g->desc.helium != 0;
    const double nunk = (he ? 5.0 : 3.0) * (double)n;   // N (N_s + 2) unknowns of Eq. rmsnorm
    rt_step_stats st;
    std::memset(&st, 0, sizeof(st));
    HeliumArgs H;
    std::memset(&H, 0, sizeof(H));
    H.nHeI0 = g->He10;
    H.nHeII0 = g->He20;

    AssembleArgs A = base_args(g, in);
    double lam = 0.0;
    double norm_cur = 0.0;   // ||f(U_k)|| with U_k's own weights
    bool have_cur = false;
    int rcode = RT_ENOCONV;
    for (int eval = 0; eval < 64 * g->desc.max_newton; ++eval) {
        A.E_cur = g->Ec;
        A.step = have_cur ? g->step : nullptr;
        A.lam = lam;
        A.n_guess = g->nc;
        A.ec_guess = g->ecc;
        A.E_out = g->Et;
        A.n_out = g->nt;
        A.ec_out = g->ect;
        A.diag = g->diag;
        A.rhs = g->rhs;
        A.wE = g->wE;
        A.Xe_cur = have_cur && !he ? g->Xec : nullptr;
        A.Xn_cur = have_cur && !he ? g->Xnc : nullptr;
        A.Xe_out = he ? nullptr : g->Xet;
        A.Xn_out = he ? nullptr : g->Xnt;
        H.HeI_guess = g->He1c;
        H.HeII_guess = g->He2c;
        H.HeI_out = g->He1t;
        H.HeII_out = g->He2t;
        // algorithmic bytes per cell: E_k, n guess, E^n, n^n, rho, e_h, b_E, src, 3 faces read;
        // trial E, n, e_c, Schur diagonal, right side and norm weight written
        double per = 8.0 * (1 + 1 + 4 + 2 + 3) + 4.0 + 8.0 * 6;
        if (A.step) per += 8.0;
        if (!P.isothermal) per += 8.0 + (in->vx ? 24.0 : 0.0) + 16.0 + (have_cur ? 16.0 : 0.0);
        int nb = 0;
        if (he) per += 8.0 * 6;
        run(g, K_ASSEMBLE, (double)n * per,
            [&] { nb = he ? launch_assemble_he(P, A, H, false, s) : launch_assemble(P, A, false, s); });
        st.residual_evals++;
        double v[3];
        rc = read_scalars(g, nb, 3, v);
        if (rc) return rc;
        const double scale = 1.0 / nunk;
        const double n_armijo = std::sqrt(v[0] * scale), n_own = std::sqrt(v[1] * scale);
        if (st.nhist < RT_STATS_HIST) {
            st.hist_norm[st.nhist] = have_cur ? n_armijo : n_own;
            st.hist_lam[st.nhist] = lam;
            st.nhist++;
        }
        if (v[2] > 0 || !std::isfinite(n_own)) {
            if (!have_cur) {
                set_detail("non-finite residual at the initial iterate");
                return RT_ENONFINITE;
            }
            lam *= 0.5;   // treat as a failed trial
            st.line_search_cuts++;
            if (lam < 1e-12) {
                set_detail("non-finite trial states down to step 1e-12");
                return RT_ENONFINITE;
            }
            continue;
        }
        bool accept = !have_cur || n_armijo <= (1.0 - 1e-4 * lam) * norm_cur;
        if (!accept) {
            lam *= 0.5;
            st.line_search_cuts++;
            if (lam < 1e-10) {
                set_detail("backtracking stalled at |f| = %.3e", norm_cur);
                rcode = RT_ELINESEARCH;
                break;
            }
            continue;
        }
        // accept: the trial becomes the current iterate
        swap_ptr(g->Ec, g->Et);
        swap_ptr(g->nc, g->nt);
        swap_ptr(g->ecc, g->ect);
        swap_ptr(g->Xec, g->Xet);
        swap_ptr(g->Xnc, g->Xnt);
        swap_ptr(g->He1c, g->He1t);
        swap_ptr(g->He2c, g->He2t);
        if (!have_cur) st.norm0 = n_own;
        else st.newton_iters++;
        have_cur = true;
        norm_cur = n_own;
        st.norm = n_own;
        if (n_own <= g->desc.newton_tol) {
            rcode = RT_OK;
            break;
        }
        if (st.newton_iters >= g->desc.max_newton) {
            set_detail("Newton reached %d iterations at |f| = %.3e", g->desc.max_newton, n_own);
            rcode = RT_ENOCONV;
            break;
        }
        // reduced Newton system S s = rhs at the accepted iterate
        bind_operator_levels(g);
        run(g, K_ZERO, (double)n * 8, [&] { launch_zero(g->step, n, s); });
        int its = 0;
        rc = pcg(g, g->rhs, g->step, g->wE, g->desc.lin_rtol, g->desc.max_lin, &its);
        st.linear_iters += its;
        if (st.newton_iters < RT_STATS_HIST) st.hist_cg[st.newton_iters] = rc == RT_OK ? its : -its;
        if (rc && rc != RT_ELINEAR) {             // a failed reduction still gives a usable direction
            st.kernel_launches = g->launches;
            if (stats) *stats = st;
            return rc;
        }
        lam = 1.0;
    }
    if (rcode == RT_OK) {
        // the solution change over the step, for time-step control
        A.E_cur = g->Ec;
        A.n_guess = g->nc;
        A.ec_guess = g->ecc;
        H.HeI_guess = g->He1c;
        H.HeII_guess = g->He2c;
        int nb = 0;
        run(g, K_RESNORM, (double)n * 8.0 * (P.isothermal ? 5 : 7 + (in->vx ? 3 : 0)) + (he ? 32.0 * n : 0.0),
            [&] { nb = he ? launch_change_norm_he(P, A, H, s) : launch_change_norm(P, A, s); });
        double v = 0.0;
        rc = read_scalars(g, nb, 1, &v);
        if (rc) return rc;
        st.change_norm = std::sqrt(v / nunk);
    }
    st.kernel_launches = g->launches;
    if (stats) *stats = st;
    if (g->prof_on) {
        RT_CUDA(cudaStreamSynchronize(s));
        harvest(g);
    }
    if (rcode != RT_OK) return rcode;
    RT_CUDA(cudaMemcpyAsync(io->E, g->Ec, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    RT_CUDA(cudaMemcpyAsync(io->n_HI, g->nc, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    RT_CUDA(cudaMemcpyAsync(io->e_c, g->ecc, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (he) {
        RT_CUDA(cudaMemcpyAsync(io->n_HeI, g->He1c, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        RT_CUDA(cudaMemcpyAsync(io->n_HeII, g->He2c, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    RT_CUDA(cudaStreamSynchronize(s));
    return check_launch("implicit step");
}

// f(U) for the step starting from U_n, by the Newton evaluation kernel in given-iterate mode
int residual_call(rt_grid* g, const rt_step_inputs* in, const rt_state* U_n, const rt_state* U, double* f_e,
                  double* f_n, double* f_HeI, double* f_HeII, double* f_E) {
    const bool he = g && g->desc.helium;
    if (!g || !U_n || !U || !U_n->E || !U_n->n_HI || !U->E || !U->n_HI || !U->e_c ||
        (he && (!U_n->n_HeI || !U_n->n_HeII || !U->n_HeI || !U->n_HeII))) {
        set_detail("null grid or state array");
        return RT_EINVAL;
    }
    int rc = validate_inputs(g, in);
    if (rc) return rc;
    RT_CUDA(cudaSetDevice(g->desc.device));
    PhysParams P = step_params(g, in);
    rc = step_setup(g, in, P, U_n->E, U_n->n_HI, U_n->n_HeI, U_n->n_HeII);
    if (rc) return rc;
    AssembleArgs A = base_args(g, in);
    A.E_cur = U->E;
    A.n_given = U->n_HI;
    A.ec_given = U->e_c;
    A.fE_out = f_E;
    A.fn_out = f_n;
    A.fe_out = f_e;
    if (he) {
        HeliumArgs H;
        std::memset(&H, 0, sizeof(H));
        H.nHeI0 = g->He10;
        H.nHeII0 = g->He20;
        H.HeI_given = U->n_HeI;
        H.HeII_given = U->n_HeII;
        H.fHeI_out = f_HeI;
        H.fHeII_out = f_HeII;
        launch_assemble_he(P, A, H, true, g->stream);
    } else {
        launch_assemble(P, A, true, g->stream);
    }
    RT_CUDA(cudaStreamSynchronize(g->stream));
    return check_launch("residual");
}

int rt_residual(rt_grid* g, const rt_step_inputs* in, const rt_state* U_n, const rt_state* U, double* f_e,
                double* f_n, double* f_E) {
    return residual_call(g, in, U_n, U, f_e, f_n, nullptr, nullptr, f_E);
}

int rt_residual_helium(rt_grid* g, const rt_step_inputs* in, const rt_state* U_n, const rt_state* U,
                       double* f_e, double* f_n, double* f_HeI, double* f_HeII, double* f_E) {
    if (g && !g->desc.helium) {
        set_detail("rt_residual_helium needs a grid with helium");
        return RT_EINVAL;
    }
    return residual_call(g, in, U_n, U, f_e, f_n, f_HeI, f_HeII, f_E);
}

int rt_schur_system(rt_grid* g, const rt_step_inputs* in, const rt_state* U_n, const rt_state* U, double* diag,
                    double* wx, double* wy, double* wz, double* rhs) {
    if (!g || !U_n || !U || !U_n->E || !U_n->n_HI || !U->E || !U->n_HI || !U->e_c ||
        (g->desc.helium && (!U_n->n_HeI || !U_n->n_HeII || !U->n_HeI || !U->n_HeII))) {
        set_detail("null grid or state array");
        return RT_EINVAL;
    }
    int rc = validate_inputs(g, in);
    if (rc) return rc;
    RT_CUDA(cudaSetDevice(g->desc.device));
    PhysParams P = step_params(g, in);
    rc = step_setup(g, in, P, U_n->E, U_n->n_HI, U_n->n_HeI, U_n->n_HeII);
    if (rc) return rc;
    AssembleArgs A = base_args(g, in);
    A.E_cur = U->E;
    A.n_given = U->n_HI;
    A.ec_given = U->e_c;
    A.diag = g->diag;
    A.rhs = g->rhs;
    A.wE = g->wE;
    if (g->desc.helium) {
        HeliumArgs H;
        std::memset(&H, 0, sizeof(H));
        H.nHeI0 = g->He10;
        H.nHeII0 = g->He20;
        H.HeI_given = U->n_HeI;
        H.HeII_given = U->n_HeII;
        launch_assemble_he(P, A, H, true, g->stream);
    } else {
        launch_assemble(P, A, true, g->stream);
    }
    const size_t bytes = (size_t)g->n * sizeof(double);
    cudaStream_t s = g->stream;
    if (diag) RT_CUDA(cudaMemcpyAsync(diag, g->diag, bytes, cudaMemcpyDeviceToDevice, s));
    if (wx) RT_CUDA(cudaMemcpyAsync(wx, g->wx, bytes, cudaMemcpyDeviceToDevice, s));
    if (wy) RT_CUDA(cudaMemcpyAsync(wy, g->wy, bytes, cudaMemcpyDeviceToDevice, s));
    if (wz) RT_CUDA(cudaMemcpyAsync(wz, g->wz, bytes, cudaMemcpyDeviceToDevice, s));
    if (rhs) RT_CUDA(cudaMemcpyAsync(rhs, g->rhs, bytes, cudaMemcpyDeviceToDevice, s));
    RT_CUDA(cudaStreamSynchronize(s));
    g->schur_ready = true;
    return check_launch("schur system");
}

int rt_schur_solve(rt_grid* g, const double* b, double* x, double rtol, int max_iters, int* iters) {
    if (!g || !b || !x || !(rtol > 0) || max_iters < 1) {
        set_detail("rt_schur_solve needs a grid, b, x, rtol > 0 and max_iters >= 1");
        return RT_EINVAL;
    }
    if (!g->schur_ready) {
        set_detail("rt_schur_solve needs a preceding rt_schur_system");
        return RT_EINVAL;
    }
    RT_CUDA(cudaSetDevice(g->desc.device));
    bind_operator_levels(g);
    int its = 0;
    int rc = pcg(g, b, x, nullptr, rtol, max_iters, &its);
    if (iters) *iters = its;
    if (rc) return rc;
    RT_CUDA(cudaStreamSynchronize(g->stream));
    return check_launch("schur solve");
}

int rt_eval_elementary(int fn, const double* x, double* y, long long n, void* stream) {
    if (fn < 0 || fn > 3 || n < 0 || (n > 0 && (!x || !y))) {
        set_detail("invalid rt_eval_elementary arguments");
        return RT_EINVAL;
    }
    if (n == 0) return RT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    launch_elementary(fn, x, y, n, s);
    RT_CUDA(cudaStreamSynchronize(s));
    return check_launch("elementary functions");
}

int rt_set_profiling(rt_grid* g, int on) {
    if (!g) {
        set_detail("null grid");
        return RT_EINVAL;
    }
    RT_CUDA(cudaSetDevice(g->desc.device));
    RT_CUDA(cudaStreamSynchronize(g->stream));
    g->prof_on = on != 0;
    g->ev_used = 0;
    for (int k = 0; k < 32; ++k) {
        g->prof_ms[k] = 0.0;
        g->prof_bytes[k] = 0.0;
        g->prof_cnt[k] = 0;
    }
    return RT_OK;
}

int rt_get_profile(rt_grid* g, rt_kernel_profile* out, int max_entries, int* n_entries) {
    if (!g || (!out && max_entries > 0)) {
        set_detail("null grid, or no output array for max_entries > 0");
        return RT_EINVAL;
    }
    RT_CUDA(cudaSetDevice(g->desc.device));
    RT_CUDA(cudaStreamSynchronize(g->stream));
    harvest(g);
    int m = 0;
    for (int k = 0; k < K_NCLASS; ++k) {
        if (g->prof_cnt[k] == 0) continue;
        if (m < max_entries) {
            std::memset(&out[m], 0, sizeof(rt_kernel_profile));
            std::snprintf(out[m].name, sizeof(out[m].name), "%s", kClassName[k]);
            out[m].launches = g->prof_cnt[k];
            out[m].ms = g->prof_ms[k];
            out[m].bytes = g->prof_bytes[k];
        }
        ++m;
    }
    if (n_entries) *n_entries = m;
    return RT_OK;
}

int rt_fold_energy(rt_grid* g, double* e_h, const double* e_c) {
    if (!g || !e_h || !e_c) {
        set_detail("null grid or energy array");
        return RT_EINVAL;
    }
    RT_CUDA(cudaSetDevice(g->desc.device));
    run(g, K_ADD, (double)g->n * 24, [&] { launch_add(g->n, e_c, e_h, g->stream); });
    if (g->prof_on) {
        RT_CUDA(cudaStreamSynchronize(g->stream));
        harvest(g);
    }
    RT_CUDA(cudaStreamSynchronize(g->stream));
    return check_launch("fold energy");
}

int rt_advect(rt_grid* g, const rt_step_inputs* in, const rt_state* src, rt_state* dst, const double* rho_src,
              double* rho_dst, double* courant_max) {
    return advect_call(g, in, src, dst, rho_src, rho_dst, courant_max, false);
}

int rt_advect_adjoint(rt_grid* g, const rt_step_inputs* in, const rt_state* lam_star, rt_state* lam) {
    return advect_call(g, in, lam_star, lam, nullptr, nullptr, nullptr, true);
}

int rt_adjoint_step(rt_grid* g, const rt_step_inputs* in, const rt_state* U_n, const rt_state* U_np1,
                    const rt_state* lam_np1, rt_state* lam_n, double* g_ndot, float* g_clump) {
    if (g && g->desc.helium) {
        set_detail("the discrete adjoint covers hydrogen-only grids");
        return RT_EINVAL;
    }
    if (g && has_outflow(g->desc)) {
        set_detail("the discrete adjoint covers periodic and reflecting faces");
        return RT_EINVAL;
    }
    if (!g || !U_n || !U_np1 || !lam_np1 || !lam_n || !U_n->E || !U_n->n_HI || !U_np1->E || !U_np1->n_HI ||
        !U_np1->e_c || !lam_np1->E || !lam_np1->n_HI || !lam_np1->e_c || !lam_n->E || !lam_n->n_HI || !lam_n->e_c) {
        set_detail("null state or adjoint array");
        return RT_EINVAL;
    }
    int rc = validate_inputs(g, in);
    if (rc) return rc;
    RT_CUDA(cudaSetDevice(g->desc.device));
    g->launches = 0;
    PhysParams P = step_params(g, in);
    rc = step_setup(g, in, P, U_n->E, U_n->n_HI);
    if (rc) return rc;
    cudaStream_t s = g->stream;
    // forward Schur operator at the converged state (symmetric: also the adjoint operator)
    AssembleArgs F = base_args(g, in);
    F.E_cur = U_np1->E;
    F.n_given = U_np1->n_HI;
    F.ec_given = U_np1->e_c;
    F.diag = g->diag;
    F.rhs = g->rhs;
    F.wE = g->wE;
    run(g, K_ASSEMBLE, 0.0, [&] { launch_assemble(P, F, true, s); });
    AdjointArgs A;
    std::memset(&A, 0, sizeof(A));
    A.rho = in->rho_b;
    A.e_h = in->e_h;
    A.vx = in->vx;
    A.vy = in->vy;
    A.vz = in->vz;
    A.clump = in->clump;
    A.E0 = g->E0;
    A.n0 = g->n0;
    A.E = U_np1->E;
    A.nHI = U_np1->n_HI;
    A.ec = U_np1->e_c;
    A.lam_E_in = lam_np1->E;
    A.lam_n_in = lam_np1->n_HI;
    A.lam_eh_in = lam_np1->e_c;
    A.rhs = g->rhs;
    run(g, K_ASSEMBLE, 0.0, [&] { launch_adj_rhs(P, A, s); });
    bind_operator_levels(g);
    run(g, K_ZERO, 0.0, [&] { launch_zero(g->step, g->n, s); });
    int its = 0;
    rc = pcg(g, g->rhs, g->step, nullptr, std::min(g->desc.lin_rtol, 1e-10), g->desc.max_lin, &its);
    if (rc) return rc;
    A.muE = g->step;
    A.lam_E_out = lam_n->E;
    A.lam_n_out = lam_n->n_HI;
    A.lam_eh_out = lam_n->e_c;
    A.g_clump = g_clump;
    A.g_ndot = g_ndot;
    A.src_cell = in->src_cell;
    run(g, K_ASSEMBLE, 0.0, [&] { launch_adj_back(P, A, g_ndot ? in->nsrc : 0, s); });
    RT_CUDA(cudaStreamSynchronize(s));
    return check_launch("adjoint step");
}

}  // extern "C"

// Step parameters from a descriptor alone (no grid handle, no allocation): the same unit
// factors, grey constants and per-step values rt_init_grid and rt_implicit_step derive.
// Used by the allocation-free entry point in noalloc.cu.
int rt_internal_step_params(const rt_grid_desc* desc, const rt_step_inputs* in, PhysParams* out) {
    if (!desc || !in || !out) return RT_EINVAL;
    if (check_geometry(*desc)) return RT_EINVAL;
    int rc = validate_inputs(nullptr, in);
    if (rc) return rc;
    PhysParams P = base_params(*desc, grey_constants(desc->spectrum, desc->T_B));
    apply_step(P, *desc, in);
    *out = P;
    return RT_OK;
}

const char* rt_internal_set_detail(const char* msg) {
    set_detail("%s", msg);
    return g_detail;
}
