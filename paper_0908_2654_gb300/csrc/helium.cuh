// Cell-local physics of step (v) for hydrogen + helium gas, templated on double / Dual<K>.
//
// Species n_HI, n_HeI, n_HeII (n_HII = n_H - n_HI, n_HeIII = n_He - n_HeI - n_HeII), number
// densities; n_e = n_HII + n_HeII + 2 n_HeIII (Eq. electron_density's helium case written for
// number densities); n_H = (1 - Y) rho~, n_He = Y rho~ / 4 in the normalised units.
//
//  * rates: hydrogen as in physics.cuh; helium case-B recombination HeII -> HeI
//    1.26e-14 (2 T_HeI/T)^0.75 plus dielectronic 1.9e-3 T^-1.5 e^{-470000/T} (1 + 0.3
//    e^{-94000/T}), HeIII -> HeII the hydrogenic fit at 2 T_HeII/T (Hui & Gnedin 1997; Cen
//    1992), all times the clumping factor; cooling adds HeII and HeIII recombination (HeIII by the
//    hydrogenic scaling of hydrogen's, Lambda_Z(T) = Z^3 Lambda_H(T / Z^2)), dielectronic
//    and HeII collisional-excitation cooling and bremsstrahlung of every ion (Z^2 = 4 for HeIII).
//    As for hydrogen the fits are evaluated with one d/dT lane and chained to all partials.
//  * S_HI: exact solution over dt of y' = A (n_H - y)(n_H + n_e,He - y) - G y with the helium
//    electrons frozen (Bernoulli form about the smaller root).
//  * S_HeI, S_HeII: exact solution over dt of the chain HeI <-> HeII <-> HeIII with n_e
//    frozen, x' = M x + c: x = x_ss + e^{M dt}(x0 - x_ss) with the steady state x_ss and
//    e^{M dt} = c1 I + s (M - mu I) from M's real eigenvalues mu +- delta (the chain is a
//    birth-death process), c1 = (e^{mu1 dt} + e^{mu2 dt})/2 and s = (e^{mu1 dt} - e^{mu2 dt}) /
//    (mu1 - mu2), the difference taken as e^{mu2 dt} expm1(z) for z = 2 delta dt < 1 and the
//    slow eigenvalue as det(M) / mu2 otherwise; when |tr M| dt < 1e-3 (where x_ss and
//    e^{M dt} would cancel) the Taylor series of the solution to (M dt)^5 instead.
#pragma once
#include "physics.cuh"

#define RT_LOG_2THEI 13.254566388120152    // log(2 x 285335 K)
#define RT_LOG_2THEII 14.049024154019651   // log(2 x 631515 K)
#define RT_SQRT_2THEII 1123.8460748696862  // sqrt(2 x 631515 K)

struct CellHe {
    double rho;     // rho~ (baryon density, normalised)
    double nH, nHe; // (1 - Y) rho~, Y rho~ / 4
    double nHI0, nHeI0, nHeII0;
    double E0;
    double eh_kin;
    double clump;
};

template <class T>
struct HeRates {
    T aH, a2, a3;              // recombination coefficients [cm^3/s]: H, HeII -> HeI, HeIII -> HeII
    T rf, ff, ce, comp;        // hydrogen cooling coefficients (rf = recombination + free-free)
    T c2, c3;                  // helium cooling per n_e n_HeII and per n_e n_HeIII
};

template <class T>
RT_HD HeRates<T> he_rates_direct(const PhysParams& P, const T& temp, bool cool) {
    const TFactors<T> f = t_factors(temp);
    HeRates<T> r;
    r.aH = P.recomb ? alpha_hg97(f) : temp * 0.0 + P.alpha_const;
    const T aHeII = 1.26e-14 * fexp(0.75 * (RT_LOG_2THEI - f.logT));
    const T edi = fexp(-470000.0 * f.invT) * (1.0 + 0.3 * fexp(-94000.0 * f.invT));
    const T adi = 1.90e-3 * (f.invT / f.sqrtT) * edi;
    r.a2 = aHeII + adi;
    const T loglam3 = RT_LOG_2THEII - f.logT;
    const T lam3 = (2.0 * 631515.0) * f.invT;
    const T p3 = fexp(0.407 * (loglam3 - 1.0079579203999789));     // (lam3 / 2.740)^0.407
    r.a3 = 5.506e-14 * (lam3 * (RT_SQRT_2THEII / f.sqrtT)) * fexp(-2.242 * flog(1.0 + p3));
    if (!cool) return r;
    const T q = fexp(0.376 * (f.loglam - 0.8109302162163288));
    const T rec = 3.435e-30 * f.temp * fexp(1.970 * f.loglam - 3.720 * flog(1.0 + q));
    r.ce = 7.5e-19 * fexp(-118348.0 * f.invT) / (1.0 + f.sqrtT * 3.1622776601683794e-3);
    const T dl = 5.5 - f.logT * 0.43429448190325176;
    const T gff = 1.1 + 0.34 * fexp(dl * dl * (-1.0 / 3.0));
    r.ff = 1.42e-27 * gff * f.sqrtT;
    r.rf = rec + r.ff;
    const double Tcmb = 2.725 / P.a;
    const double kcomp = 4.0 * 1.380649e-16 * 6.6524587321e-25 * 7.565723e-15 / (9.1093837015e-28 * 2.99792458e10);
    r.comp = kcomp * (Tcmb * Tcmb) * (Tcmb * Tcmb) * (f.temp - Tcmb);
    const T ceHe2 = 5.54e-17 * fexp(-0.397 * f.logT) * fexp(-473638.0 * f.invT) /
                    (1.0 + f.sqrtT * 3.1622776601683794e-3);
    r.c2 = 1.380649e-16 * f.temp * aHeII + 6.526e-11 * adi + ceHe2;
    const T q3 = fexp(0.376 * (loglam3 - 0.8109302162163288));
    // hydrogenic scaling Lambda_Z(T) = Z^3 Lambda_H(T / Z^2), Z = 2: Z times hydrogen's
    // coefficient at the same lambda, as for the recombination coefficient a3
    r.c3 = (2.0 * 3.435e-30) * f.temp * fexp(1.970 * loglam3 - 3.720 * flog(1.0 + q3));
    return r;
}

RT_HD HeRates<double> he_rates(const PhysParams& P, double temp, bool cool) { return he_rates_direct(P, temp, cool); }

template <int K>
RT_HD HeRates<Dual<K>> he_rates(const PhysParams& P, const Dual<K>& temp, bool cool) {
    const HeRates<Dual<1>> r = he_rates_direct(P, dvar<1>(temp.v, 0), cool);
    HeRates<Dual<K>> o;
    o.aH = dchain(temp, r.aH.v, r.aH.d[0]);
    o.a2 = dchain(temp, r.a2.v, r.a2.d[0]);
    o.a3 = dchain(temp, r.a3.v, r.a3.d[0]);
    if (cool) {
        o.rf = dchain(temp, r.rf.v, r.rf.d[0]);
        o.ff = dchain(temp, r.ff.v, r.ff.d[0]);
        o.ce = dchain(temp, r.ce.v, r.ce.d[0]);
        o.comp = dchain(temp, r.comp.v, r.comp.d[0]);
        o.c2 = dchain(temp, r.c2.v, r.c2.d[0]);
        o.c3 = dchain(temp, r.c3.v, r.c3.d[0]);
    }
    return o;
}

// The rates as (value, d/dT) pairs, carried onto the unknowns' lanes only where a rate is used:
// nine rates held on all lanes at once would not fit the registers of the five-lane Jacobian.
RT_HD HeRates<double> he_rates_lazy(const PhysParams& P, double temp, bool cool) {
    return he_rates_direct(P, temp, cool);
}
template <int K>
RT_HD HeRates<Dual<1>> he_rates_lazy(const PhysParams& P, const Dual<K>& temp, bool cool) {
    return he_rates_direct(P, dvar<1>(temp.v, 0), cool);
}
RT_HD double on_lanes(double, double r) { return r; }
template <int K>
RT_HD Dual<K> on_lanes(const Dual<K>& temp, const Dual<1>& r) {
    return dchain(temp, r.v, r.d[0]);
}

// n(dt) for n' = A (nH - n)(nH + neHe - n) - G n, n(0) = y0
template <class T>
RT_HD T riccati_ne(double y0, double nH, const T& neHe, const T& A, const T& G, double dt) {
    const T g = A * neHe + G;
    T d = sqrt(g * g + 4.0 * nH * (A * G));
    T den = A * (2.0 * nH + neHe) + G + d;
    T yeq = (value(den) > 0.0) ? (2.0 * nH) * (A * (nH + neHe)) / den : den * 0.0;
    T u0 = y0 - yeq;
    T q, p1;
    decay_factors(d * dt, q, p1);
    return yeq + u0 * q / (1.0 - (u0 * A) * (dt * p1));
}

// (HeI, HeII)(dt) of the helium chain with photo-ionisation rates G1, G2, recombination rates
// r2 (HeII -> HeI) and r3 (HeIII -> HeII), total nHe
template <class T>
RT_HD void helium_chain(double x10, double x20, double nHe, const T& G1, const T& G2, const T& r2, const T& r3,
                        double dt, T& x1, T& x2) {
    const T M11 = -G1, M12 = r2, M21 = G1 - r3, M22 = -(G2 + r2 + r3);
    const T c2 = r3 * nHe;
    const T tr = M11 + M22;
    const T det = G1 * G2 + G1 * r3 + r2 * r3;
    if (fabs(value(tr)) * dt < 1e-3 || !(value(det) > 0.0)) {
        // x = x0 + dt sum_{j<5} (M dt)^j / (j+1)! (M x0 + c), by Horner; every entry of M is
        // at most |tr M|, so the first omitted term is below (2e-3)^6 / 720 relative
        const T v1 = M11 * x10 + M12 * x20, v2 = M21 * x10 + M22 * x20 + c2;
        T u1 = v1, u2 = v2;
#pragma unroll
        for (int k = 5; k >= 2; --k) {
            const double f = dt / k;
            const T t1 = v1 + f * (M11 * u1 + M12 * u2);
            const T t2 = v2 + f * (M21 * u1 + M22 * u2);
            u1 = t1;
            u2 = t2;
        }
        x1 = x10 + dt * u1;
        x2 = x20 + dt * u2;
        return;
    }
    const T fss = c2 / det;
    const T s1 = fss * r2, s2 = fss * G1;                    // steady state
    const T mu = 0.5 * tr;
    const T dd = M11 - M22;
    T disc = dd * dd + 4.0 * (M12 * M21);
    if (value(disc) < 0.0) disc = disc * 0.0;
    const T delta = 0.5 * sqrt(disc);
    const T E2 = fexp((mu - delta) * dt);
    const T z = (2.0 * dt) * delta;
    T s, c1;
    if (value(z) < 1.0) {           // e^{mu1 dt} - e^{mu2 dt} = E2 expm1(z), without cancellation
        const T phe = (value(z) < 1e-8) ? 1.0 + z * 0.5 + z * z * (1.0 / 6.0) : expm1(z) / z;
        s = E2 * (dt * phe);
        c1 = E2 + 0.5 * (E2 * z * phe);
    } else {                        // both exponentials directly (mu1, mu2 <= 0: no overflow);
        // the slow eigenvalue as det / mu2 (mu + delta cancels when one rate dominates)
        const T mu2 = mu - delta;
        const T mu1 = det / mu2;
        const T E1 = fexp(mu1 * dt);
        s = (E1 - E2) / (mu1 - mu2);
        c1 = 0.5 * (E1 + E2);
    }
    const T y1 = x10 - s1, y2 = x20 - s2;
    x1 = s1 + c1 * y1 + s * ((M11 - mu) * y1 + M12 * y2);
    x2 = s2 + c1 * y2 + s * (M21 * y1 + (M22 - mu) * y2);
}

// S_e, S_HI, S_HeI, S_HeII at the iterate with coefficients frozen there
template <class T>
RT_HD void local_solutions_he(const PhysParams& P, const CellHe& c, const T& ec, const T& nHI, const T& nHeI,
                              const T& nHeII, const T& E, T& Se, T& SHI, T& SHeI, T& SHeII) {
    const T Ebar = spos(P.theta * E + (1.0 - P.theta) * c.E0, P.E_min);
    const T nHeIII = c.nHe - nHeI - nHeII;
    const T neHe = nHeII + 2.0 * nHeIII;
    const T ne = (c.nH - nHI) + neHe;
    T temp;
    if (P.isothermal) {
        temp = ec * 0.0 + P.T_iso;
    } else {
        temp = (P.kT * c.rho) * (c.eh_kin + ec) / ((c.nH + c.nHe) + ne);
        if (value(temp) < RT_T_FLOOR) temp = temp * 0.0 + RT_T_FLOOR;
    }
    const bool cool = !P.isothermal && P.cooling;
    const auto r = he_rates_lazy(P, temp, cool);
    const double rfac = P.kA * c.clump / P.a3;
    const T Eb = Ebar * (1.0 / P.a3);
    SHI = riccati_ne(c.nHI0, c.nH, neHe, on_lanes(temp, r.aH) * rfac, P.kG * Eb, P.dt);
    const T rne = ne * rfac;
    helium_chain(c.nHeI0, c.nHeII0, c.nHe, P.kG1 * Eb, P.kG2 * Eb, on_lanes(temp, r.a2) * rne,
                 on_lanes(temp, r.a3) * rne, P.dt, SHeI, SHeII);
    if (P.isothermal) {
        Se = ec * 0.0;
        return;
    }
    const T heat = (nHI * P.kH + nHeI * P.kH1 + nHeII * P.kH2) * Ebar * (1.0 / (P.a3 * c.rho));
    T cooling = heat * 0.0;
    if (cool) {
        const double s = P.un / P.a3;
        const T nep = ne * s, nHIIp = (c.nH - nHI) * s, nHIp = nHI * s, n2p = nHeII * s, n3p = nHeIII * s;
        const T vol = nep * (on_lanes(temp, r.rf) * nHIIp + on_lanes(temp, r.ff) * (n2p + 4.0 * n3p) +
                             on_lanes(temp, r.ce) * nHIp + on_lanes(temp, r.c2) * n2p + on_lanes(temp, r.c3) * n3p) +
                      on_lanes(temp, r.comp) * nep;
        cooling = (P.kC * P.a3 / c.rho) * vol;
    }
    Se = (heat - cooling) * P.phi_e;
}
