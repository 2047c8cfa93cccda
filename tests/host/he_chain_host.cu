// Host builds of the GPU path's cell physics (helium.cuh and physics.cuh, compiled for the
// CPU) so that tests can compare them with the oracle across parameter regimes: the helium
// chain, the Riccati solutions with and without helium electrons, the rate fits of both
// chemistry paths and the face limiter; derivatives through the same dual numbers the kernels
// use.
#include <cstring>

#include "../../paper_0908_2654_gb300/csrc/helium.cuh"

extern "C" {

// x1, x2 = helium_chain at each of n parameter sets; d1, d2 = their derivatives in G1 and r3
void he_chain_host(int n, const double* x10, const double* x20, const double* nHe, const double* G1,
                   const double* G2, const double* r2, const double* r3, const double* dt, double* x1, double* x2,
                   double* dx1_dG1, double* dx2_dr3) {
    for (int i = 0; i < n; ++i) {
        Dual<2> a, b;
        helium_chain<Dual<2>>(x10[i], x20[i], nHe[i], dvar<2>(G1[i], 0), dconst<2>(G2[i]), dconst<2>(r2[i]),
                              dvar<2>(r3[i], 1), dt[i], a, b);
        x1[i] = a.v;
        x2[i] = b.v;
        dx1_dG1[i] = a.d[0];
        dx2_dr3[i] = b.d[1];
    }
}

void riccati_ne_host(int n, const double* y0, const double* nH, const double* neHe, const double* A,
                     const double* G, const double* dt, double* y) {
    for (int i = 0; i < n; ++i) y[i] = riccati_ne<double>(y0[i], nH[i], neHe[i], A[i], G[i], dt[i]);
}

}

extern "C" {

// rate fits of the GPU path at n temperatures (recomb = 1: Hui & Gnedin hydrogen alpha), with
// d/dT of each from the single-lane promotion the kernels use; outputs [9][n]:
// alpha_H, alpha_HeII(+di), alpha_HeIII, rec+ff, ff, ce, comp, c2, c3 (and the same for d/dT)
void rates_host(int n, const double* T, double a, double* out, double* dout) {
    PhysParams P;
    memset(&P, 0, sizeof(P));
    P.recomb = 1;
    P.a = a;
    for (int i = 0; i < n; ++i) {
        const HeRates<Dual<1>> r = he_rates<1>(P, dvar<1>(T[i], 0), true);
        const Dual<1>* v[9] = {&r.aH, &r.a2, &r.a3, &r.rf, &r.ff, &r.ce, &r.comp, &r.c2, &r.c3};
        for (int k = 0; k < 9; ++k) {
            out[k * n + i] = v[k]->v;
            dout[k * n + i] = v[k]->d[0];
        }
    }
}

}

extern "C" {

// hydrogen-only Riccati solution of the GPU path (shared expm1 decay factors)
void riccati_n_host(int n, const double* y0, const double* nH, const double* A, const double* G, const double* dt,
                    double* y) {
    for (int i = 0; i < n; ++i) y[i] = riccati_n<double>(y0[i], nH[i], A[i], G[i], dt[i]);
}

}

extern "C" {

// hydrogen-only rate fits of the GPU path (physics.cuh t_rates: one d/dT lane, chained into a
// two-lane dual with T as lane 0); outputs [4][n]: alpha (Hui & Gnedin), rf, ce, comp, with
// d/dT of each in dout and the untouched second lane in dzero
void t_rates_host(int n, const double* T, double a, double* out, double* dout, double* dzero) {
    PhysParams P;
    memset(&P, 0, sizeof(P));
    P.recomb = 1;
    P.a = a;
    for (int i = 0; i < n; ++i) {
        const TRates<Dual<2>> r = t_rates<2>(P, dvar<2>(T[i], 0), true, true);
        const Dual<2>* v[4] = {&r.alpha, &r.rf, &r.ce, &r.comp};
        for (int k = 0; k < 4; ++k) {
            out[k * n + i] = v[k]->v;
            dout[k * n + i] = v[k]->d[0];
            dzero[k * n + i] = v[k]->d[1];
        }
    }
}

// Eq. limiter on n faces (Ei, Ej, ki, kj) as the face kernels evaluate it, and its derivative
// in Ei through the dual-number form the adjoint uses
void limiter_host(int n, const double* Ei, const double* Ej, const double* ki, const double* kj, double adx,
                  double c, double E_min, double* D, double* D_t, double* dD_dEi) {
    PhysParams P;
    memset(&P, 0, sizeof(P));
    P.adx = adx;
    P.c = c;
    P.E_min = E_min;
    P.limiter = 0;
    for (int i = 0; i < n; ++i) {
        D[i] = limiter_face(P, Ei[i], Ej[i], ki[i], kj[i]);
        const Dual<1> d = limiter_face_t<Dual<1>>(P, dvar<1>(Ei[i], 0), dconst<1>(Ej[i]), dconst<1>(ki[i]),
                                                   dconst<1>(kj[i]));
        D_t[i] = d.v;
        dD_dEi[i] = d.d[0];
    }
}

}
