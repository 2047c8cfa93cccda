// Cell-local physics of step (v) in normalised units, templated on double / Dual<K>.
//
//  * flux limiter on a face (Eq. limiter), evaluated at the step's starting state;
//  * S_n: exact solution over dt of the hydrogen rate equation (Eq. RT-chemical_ionization
//    with n_e = n_HII = n_H - n_HI) with its coefficients frozen -- a Riccati equation
//    n' = A (n_H - n)^2 - G n, solved in Bernoulli form about its equilibrium root;
//  * S_e: exact solution of de/dt = -2 (adot/a) e + (G - Lambda) with frozen G - Lambda
//    and e_c^n = 0 (Eq. RT-cons_energy);
//  * rates: constant case-B alpha = 2.59e-13 cm^3/s or the Hui & Gnedin (1997) fit,
//    photo-heating n_HI c E (sigma_E - h nu_0 sigma_G), cooling by case-B recombination
//    (Hui & Gnedin 1997), collisional excitation and bremsstrahlung (Cen 1992) and
//    Compton scattering off the CMB.
#pragma once
#include <cmath>

#include "dual.cuh"
#include "fastmath.cuh"

// exp and log of the rate fits: the table-driven versions of fastmath.cuh on the device
RT_HD double fexp(double x) {
#ifdef __CUDA_ARCH__
    return rt_exp(x);
#else
    return std::exp(x);
#endif
}
RT_HD double flog(double x) {
#ifdef __CUDA_ARCH__
    return rt_log(x);
#else
    return std::log(x);
#endif
}
template <int K>
RT_HD Dual<K> fexp(const Dual<K>& a) {
    const double e = fexp(a.v);
    return dchain(a, e, e);
}
template <int K>
RT_HD Dual<K> flog(const Dual<K>& a) {
    return dchain(a, flog(a.v), 1.0 / a.v);
}

struct PhysParams {
    // grid
    int nx, ny, nz;
    int per[3];
    int outflow[6];    // per face (x-, x+, y-, y+, z-, z+): 1 = outflow boundary face
    double dx;         // comoving cell width (normalised)
    // step
    double a, a3, H;   // expansion factor, a^3, adot / a (per normalised time)
    double dt, theta;
    double wscale;     // dt * theta / (a dx)^2: face coupling w = wscale * D
    double adx;        // proper cell width a dx
    // constants in normalised units
    double c;          // speed of light
    double kE;         // kappa = kE n / a^3        (proper opacity per normalised length)
    double kG;         // Gamma = kG Ebar / a^3     (photo-ionisation rate)
    double kA;         // A = alpha[cm^3/s] kA C / a^3  (recombination coefficient of n)
    double kH;         // heating per unit mass = kH n Ebar / (a^3 rho)
    double kC;         // cooling per unit mass = kC a^3 Lambda_vol[cgs] / rho
    double kT;         // T = kT e_int rho / (2 rho - n)   [K]
    double un;         // u_n [cm^-3]: proper physical density = n un / a^3
    double E_min;      // radiation floor (limiter, rate smoothing)
    double E_floor;    // per step: smallest E scale of the residual norm, max(E_min, 1e-12 max E_init)
    double e_floor;    // specific internal energy of 1 K gas (mu = 1), for the norm
    double phi_e;      // dt * phi1(2 H dt): S_e = (G - Lambda) phi_e
    double local_tol;  // scaled residual at which the cell-local Newton iteration stops
    double T_iso;
    double D_const;    // normalised proper diffusion coefficient (limiter "const")
    double src_scale;  // 4 pi eta = src_scale * Ndot in the source's cell
    double alpha_const;
    int isothermal, recomb, cooling, limiter;
    // hydrogen + helium (helium = 1): mass fraction Y, grey constants of HeI and HeII like kE,
    // kG, kH, and the step's starting He densities (their opacity enters D^n and b_E)
    int helium;
    double Y;
    double kE1, kE2, kG1, kG2, kH1, kH2;
    const double* nHeI0;
    const double* nHeII0;
};

// proper opacity at the start of the step (hydrogen, plus helium when present)
RT_HD double kappa_start(const PhysParams& P, const double* n0, long long i) {
    double k = P.kE * n0[i];
    if (P.nHeI0) k += P.kE1 * P.nHeI0[i] + P.kE2 * P.nHeII0[i];
    return k / P.a3;
}

#define RT_T_HI 157807.0
#define RT_T_FLOOR 1.0

// smooth positive part (x + sqrt(x^2 + eps^2)) / 2, written without cancellation for x < 0
template <class T>
RT_HD T spos(const T& x, double eps) {
    T r = sqrt(x * x + eps * eps);
    if (value(x) < 0.0) return (eps * eps) / (2.0 * (r - x));
    return 0.5 * (x + r);
}

// (1 - e^-x) / x with its limit 1 at x = 0
template <class T>
RT_HD T phi1(const T& x) {
    if (fabs(value(x)) < 1e-8) return 1.0 - x * 0.5 + x * x * (1.0 / 6.0);
    return -expm1(-x) / x;
}

// e^-x and phi1(x) = (1 - e^-x)/x from one expm1 (series for phi1 at |x| < 1e-8)
template <class T>
RT_HD void decay_factors(const T& x, T& q, T& p1) {
    const T em = expm1(-x);
    q = em + 1.0;
    p1 = (fabs(value(x)) < 1e-8) ? 1.0 - x * 0.5 + x * x * (1.0 / 6.0) : -em / x;
}

// n(dt) for n' = A (nH - n)^2 - G n, n(0) = y0.
// The right side is A (n - y_eq)(n - y_2) with y_eq = 2 A nH^2 / (2 A nH + G + d),
// d = sqrt(G^2 + 4 A G nH) = A (y_2 - y_eq).  u = n - y_eq obeys u' = A u^2 - d u, so
// u(t) = u0 e^{-d t} / (1 - u0 A t phi1(d t)).
template <class T>
RT_HD T riccati_n(double y0, double nH, const T& A, const T& G, double dt) {
    T d = sqrt(G * G + 4.0 * nH * (A * G));
    T den = 2.0 * nH * A + G + d;
    T yeq = (value(den) > 0.0) ? (2.0 * nH * nH) * A / den : den * 0.0;
    T u0 = y0 - yeq;
    T q, p1;
    decay_factors(d * dt, q, p1);
    return yeq + u0 * q / (1.0 - (u0 * A) * (dt * p1));
}

// Temperature-dependent factors shared by the recombination coefficient and the cooling
// terms: every power of T or of lambda = 2 T_HI / T is taken from one log T and one sqrt T.
template <class T>
struct TFactors {
    T temp, logT, sqrtT, invT, loglam, lam, sqrtlam;
};

template <class T>
RT_HD TFactors<T> t_factors(const T& temp) {
    TFactors<T> f;
    f.temp = temp;
    f.invT = 1.0 / temp;
    f.logT = flog(temp);
    f.sqrtT = sqrt(temp);
    f.lam = (2.0 * RT_T_HI) * f.invT;
    f.loglam = 12.662275226919286 - f.logT;            // log(2 T_HI) - log T, log(315614)
    f.sqrtlam = 561.7953363992976 / f.sqrtT;           // sqrt(2 T_HI) / sqrt T, sqrt(315614)
    return f;
}

// the same solution with the initial value y0 and the coefficients all of type T (used by
// the adjoint, which differentiates with respect to the step's starting state)
template <class T>
RT_HD T riccati_n_full(const T& y0, double nH, const T& A, const T& G, double dt) {
    T d = sqrt(G * G + 4.0 * nH * (A * G));
    T den = 2.0 * nH * A + G + d;
    T yeq = (value(den) > 0.0) ? (2.0 * nH * nH) * A / den : den * 0.0;
    T u0 = y0 - yeq;
    T q, p1;
    decay_factors(d * dt, q, p1);
    return yeq + u0 * q / (1.0 - (u0 * A) * (dt * p1));
}

// case-B recombination coefficient [cm^3/s], Hui & Gnedin (1997):
// 2.753e-14 lam^1.5 / (1 + (lam/2.740)^0.407)^2.242
template <class T>
RT_HD T alpha_hg97(const TFactors<T>& f) {
    T p = fexp(0.407 * (f.loglam - 1.0079579203999789));           // (lam / 2.740)^0.407
    return 2.753e-14 * (f.lam * f.sqrtlam) * fexp(-2.242 * flog(1.0 + p));
}

// cooling per unit proper volume [erg cm^-3 s^-1] is (rf n_HII + ce n_HI + comp) n_e with
// proper densities [cm^-3] and temperature-only coefficients: rf = case-B recombination
// (Hui & Gnedin 1997) plus bremsstrahlung (Cen 1992), ce = collisional excitation (Cen 1992),
// comp = Compton scattering off the CMB (per electron)
template <class T>
struct TRates {
    T alpha;   // case-B recombination coefficient [cm^3/s]
    T rf, ce, comp;
};

template <class T>
RT_HD TRates<T> t_rates_direct(const PhysParams& P, const T& temp, bool fit_alpha, bool cool) {
    TRates<T> r;
    if (!fit_alpha && !cool) {
        r.alpha = temp * 0.0 + P.alpha_const;
        return r;
    }
    const TFactors<T> f = t_factors(temp);
    r.alpha = fit_alpha ? alpha_hg97(f) : temp * 0.0 + P.alpha_const;
    if (!cool) return r;
    T q = fexp(0.376 * (f.loglam - 0.8109302162163288));           // (lam / 2.250)^0.376
    T rec = 3.435e-30 * f.temp * fexp(1.970 * f.loglam - 3.720 * flog(1.0 + q));
    r.ce = 7.5e-19 * fexp(-118348.0 * f.invT) / (1.0 + f.sqrtT * 3.1622776601683794e-3);
    T dl = 5.5 - f.logT * 0.43429448190325176;                     // 5.5 - log10 T
    T gff = 1.1 + 0.34 * fexp(dl * dl * (-1.0 / 3.0));
    r.rf = rec + 1.42e-27 * gff * f.sqrtT;
    const double Tcmb = 2.725 / P.a;
    // 4 k_B sigma_T a_rad / (m_e c) in CGS
    const double kcomp = 4.0 * 1.380649e-16 * 6.6524587321e-25 * 7.565723e-15 / (9.1093837015e-28 * 2.99792458e10);
    r.comp = kcomp * (Tcmb * Tcmb) * (Tcmb * Tcmb) * (f.temp - Tcmb);
    return r;
}

// The rates depend on the cell's state only through T: for a dual-number T they are
// evaluated with the single derivative d/dT and carried to all partials by the chain rule,
// which keeps the transcendental-heavy fits off the K-lane arithmetic.
RT_HD TRates<double> t_rates(const PhysParams& P, double temp, bool fit_alpha, bool cool) {
    return t_rates_direct(P, temp, fit_alpha, cool);
}
template <int K>
RT_HD TRates<Dual<K>> t_rates(const PhysParams& P, const Dual<K>& temp, bool fit_alpha, bool cool) {
    const TRates<Dual<1>> r = t_rates_direct(P, dvar<1>(temp.v, 0), fit_alpha, cool);
    TRates<Dual<K>> o;
    o.alpha = dchain(temp, r.alpha.v, r.alpha.d[0]);
    if (cool) {
        o.rf = dchain(temp, r.rf.v, r.rf.d[0]);
        o.ce = dchain(temp, r.ce.v, r.ce.d[0]);
        o.comp = dchain(temp, r.comp.v, r.comp.d[0]);
    }
    return o;
}

// Cell inputs that do not depend on the iterate.
struct CellIn {
    double rho;     // n_H (= rho~ in these units)
    double nHI0;    // n_HI at the start of the step
    double E0;      // E at the start of the step
    double eh_kin;  // e_h - |v|^2 / 2 (specific internal energy from the hydro state)
    double clump;
};

// S_e and S_n at the iterate (ec, n, E) with coefficients frozen at that iterate.
template <class T>
RT_HD void local_solutions(const PhysParams& P, const CellIn& c, const T& ec, const T& n, const T& E,
                           T& Se, T& Sn) {
    T Ebar = spos(P.theta * E + (1.0 - P.theta) * c.E0, P.E_min);
    T G = (P.kG / P.a3) * Ebar;
    T temp;
    if (P.isothermal) {
        temp = ec * 0.0 + P.T_iso;
    } else {
        temp = (P.kT * c.rho) * (c.eh_kin + ec) / (2.0 * c.rho - n);
        if (value(temp) < RT_T_FLOOR) temp = temp * 0.0 + RT_T_FLOOR;
    }
    const bool cool = !P.isothermal && P.cooling;
    const TRates<T> rt = t_rates(P, temp, P.recomb != 0, cool);
    T A = rt.alpha * (P.kA * c.clump / P.a3);
    Sn = riccati_n(c.nHI0, c.rho, A, G, P.dt);
    if (P.isothermal) {
        Se = ec * 0.0;
        return;
    }
    T heat = (P.kH / (P.a3 * c.rho)) * (n * Ebar);
    T cooling = heat * 0.0;
    if (cool) {
        const double s = P.un / P.a3;
        T nHII = (c.rho - n) * s;                 // = n_e
        T nHIp = n * s;
        cooling = (P.kC * P.a3 / c.rho) * (((rt.rf * nHII + rt.ce * nHIp) + rt.comp) * nHII);
    }
    Se = (heat - cooling) * P.phi_e;
}

// local_solutions with the start-of-step values E^n, n_HI^n and the clumping factor C also
// of type T (their partial derivatives feed the adjoint of the step map)
template <class T>
RT_HD void local_solutions_full(const PhysParams& P, const CellIn& c, const T& ec, const T& n, const T& E,
                                const T& E0, const T& y0, const T& C, T& Se, T& Sn) {
    T Ebar = spos(P.theta * E + (1.0 - P.theta) * E0, P.E_min);
    T G = (P.kG / P.a3) * Ebar;
    T temp;
    if (P.isothermal) {
        temp = ec * 0.0 + P.T_iso;
    } else {
        temp = (P.kT * c.rho) * (c.eh_kin + ec) / (2.0 * c.rho - n);
        if (value(temp) < RT_T_FLOOR) temp = temp * 0.0 + RT_T_FLOOR;
    }
    const bool cool = !P.isothermal && P.cooling;
    const TRates<T> rt = t_rates(P, temp, P.recomb != 0, cool);
    T A = rt.alpha * (P.kA / P.a3) * C;
    Sn = riccati_n_full(y0, c.rho, A, G, P.dt);
    if (P.isothermal) {
        Se = ec * 0.0;
        return;
    }
    T heat = (P.kH / (P.a3 * c.rho)) * (n * Ebar);
    T cooling = heat * 0.0;
    if (cool) {
        const double s = P.un / P.a3;
        T nHII = (c.rho - n) * s;                 // = n_e
        T nHIp = n * s;
        cooling = (P.kC * P.a3 / c.rho) * (((rt.rf * nHII + rt.ce * nHIp) + rt.comp) * nHII);
    }
    Se = (heat - cooling) * P.phi_e;
}

// Eq. limiter at a face for any scalar type (the adjoint differentiates D with respect to
// the start-of-step state it is evaluated from)
template <class T>
RT_HD T limiter_face_t(const PhysParams& P, const T& Ei, const T& Ej, const T& ki, const T& kj) {
    if (P.limiter == 1) return Ei * 0.0 + P.D_const;
    T Ef = spos(0.5 * (Ei + Ej), P.E_min);
    T dE = Ej - Ei;
    T R = (value(dE) >= 0.0 ? dE : -dE) / (P.adx * Ef);
    T kT = 0.5 * (ki + kj);
    if (value(kT) == 0.0 && value(R) == 0.0) R = R * 0.0 + 1.0 / P.adx;
    return P.c * (2.0 * kT + R) / ((6.0 * kT + 3.0 * R) * kT + R * R);
}

// Eq. limiter on a face between cells with energies (Ei, Ej) and proper opacities
// (ki, kj); R from the face difference over the proper width, E_face = spos(mean E).
RT_HD double limiter_face(const PhysParams& P, double Ei, double Ej, double ki, double kj) {
    if (P.limiter == 1) return P.D_const;
    double Ef = spos(0.5 * (Ei + Ej), P.E_min);
    double R = fabs(Ej - Ei) / (P.adx * Ef);
    double kT = 0.5 * (ki + kj);
    if (kT == 0.0 && R == 0.0) R = 1.0 / P.adx;
    return P.c * (2.0 * kT + R) / ((6.0 * kT + 3.0 * R) * kT + R * R);
}

// Number of outflow boundary faces of cell (x, y, z) (0 for interior cells).
RT_HD int outflow_faces(const PhysParams& P, int x, int y, int z) {
    return (P.outflow[0] && x == 0) + (P.outflow[1] && x == P.nx - 1) + (P.outflow[2] && y == 0) +
           (P.outflow[3] && y == P.ny - 1) + (P.outflow[4] && z == 0) + (P.outflow[5] && z == P.nz - 1);
}

// Face coupling summed over the outflow faces of cell i: each face joins the cell to an empty
// ghost (E = 0, the cell's own opacity), so it couples w = dt theta D / (a dx)^2 with D from
// Eq. limiter between the two, evaluated at the step's start like every face (lagged limiter).
// Its flux w (0 - E) only removes energy: it adds w to the cell's diagonal and nothing off it.
RT_HD double outflow_coupling(const PhysParams& P, const double* E0, const double* n0, long long i, int x, int y,
                              int z) {
    const int nf = outflow_faces(P, x, y, z);
    if (nf == 0) return 0.0;
    const double ki = kappa_start(P, n0, i);
    return nf * P.wscale * limiter_face(P, E0[i], 0.0, ki, ki);
}
