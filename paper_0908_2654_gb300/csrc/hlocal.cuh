// Hydrogen cell-local equations of the Newton evaluation kernel with their partial derivatives
// written out (Eqs. gas_residual and chemistry_residual with the local solutions S_e, S_n of
// physics.cuh): the same values and the same six partials d(S_e, S_n)/d(e_c, n_HI, E) as the
// dual-number evaluation local_solutions<Dual<3>>, with less FP64 work:
//
//  * the state enters the rate fits only through T, so the fits are evaluated once as values
//    and their d/dT in closed form (each fit is exp/log of log T, so d/dT = value times a
//    rational function of the fit's own factors);
//  * S_n depends on (e_c, n_HI, E) only through the recombination coefficient A(T) and the
//    photo-ionisation rate G(E): the Riccati solution carries two derivative lanes (A, G) and
//    the chain rule gives the three partials;
//  * S_e = phi_e (heating - cooling) is linear in the heating and its cooling terms are
//    products of the fits with n_HII and n_HI, differentiated term by term;
//  * everything that does not depend on the iterate (1/rho, the unit factors over a^3, the
//    clumping factor) is formed once per cell;
//  * one reciprocal serves several quotients where they share a denominator (1/T and
//    1/(2 rho - n) from 1/(kT rho e_int (2 rho - n)); sqrt(lambda) from sqrt(T) / T);
//  * the decay factors e^-x and (1 - e^-x)/x of the Riccati solution come from the table exp
//    (x >= 1/32) or their Taylor series (x < 1/32), with d/dx in the same two forms.
#pragma once
#include "physics.cuh"

// iterate-independent constants of one cell
struct HCell {
    double rho;     // n_H (= rho~ in these units)
    double y0;      // n_HI at the start of the step
    double E0;      // E at the start of the step
    double eh_kin;  // e_h - |v|^2 / 2
    double Ak;      // A = alpha[cm^3/s] * Ak  (kA C / a^3)
    double kTr;     // T = kTr e_int / (2 rho - n)
    double hk;      // heating per unit mass = hk n Ebar      (kH / (a^3 rho))
    double ck;      // cooling per unit mass = ck Lambda_vol   (kC a^3 / rho)
    double inv_a3;  // 1 / a^3
    double inv_rho; // 1 / n_H
};

RT_HD HCell make_hcell(const PhysParams& P, double inv_a3, double rho, double y0, double E0, double eh_kin,
                       double clump) {
    HCell c;
    const double inv_rho = 1.0 / rho;
    c.rho = rho;
    c.y0 = y0;
    c.E0 = E0;
    c.eh_kin = eh_kin;
    c.Ak = P.kA * clump * inv_a3;
    c.kTr = P.kT * rho;
    c.hk = P.kH * inv_a3 * inv_rho;
    c.ck = P.kC * P.a3 * inv_rho;
    c.inv_a3 = inv_a3;
    c.inv_rho = inv_rho;
    return c;
}

// the temperature-only rate fits at T with their derivatives d/dT (fits as in t_rates_direct)
struct HRates {
    double alpha, alpha_T;
    double rf, rf_T, ce, ce_T, comp, comp_T;
};

RT_HD HRates h_rates(const PhysParams& P, double T, double invT, bool fit_alpha, bool cool) {
    HRates r;
    r.rf = r.rf_T = r.ce = r.ce_T = r.comp = r.comp_T = 0.0;
    if (!fit_alpha && !cool) {
        r.alpha = P.alpha_const;
        r.alpha_T = 0.0;
        return r;
    }
    const double logT = flog(T);
    const double sqrtT = sqrt(T);
    const double loglam = 12.662275226919286 - logT;       // log(2 T_HI / T)
    if (fit_alpha) {
        // alpha = 2.753e-14 lam^1.5 (1 + p)^-2.242, p = (lam / 2.740)^0.407
        const double lam = (2.0 * RT_T_HI) * invT;
        const double sqrtlam = 561.7953363992976 * sqrtT * invT;   // sqrt(2 T_HI) / sqrt(T)
        const double p = fexp(0.407 * (loglam - 1.0079579203999789));
        const double q1 = 1.0 + p;
        r.alpha = 2.753e-14 * (lam * sqrtlam) * fexp(-2.242 * flog(q1));
        // d ln(alpha)/d ln T = -1.5 + 2.242 * 0.407 p / (1 + p)
        r.alpha_T = r.alpha * invT * (-1.5 + (2.242 * 0.407) * p / q1);
    } else {
        r.alpha = P.alpha_const;
        r.alpha_T = 0.0;
    }
    if (!cool) return r;
    // case-B recombination cooling 3.435e-30 T lam^1.970 (1 + q)^-3.720, q = (lam / 2.250)^0.376
    const double q = fexp(0.376 * (loglam - 0.8109302162163288));
    const double q1 = 1.0 + q;
    const double rec = 3.435e-30 * T * fexp(1.970 * loglam - 3.720 * flog(q1));
    const double rec_T = rec * invT * (-0.970 + (3.720 * 0.376) * q / q1);
    // collisional excitation 7.5e-19 e^{-118348/T} / (1 + sqrt(T / 1e5))
    const double ex = fexp(-118348.0 * invT);
    const double inv_den = 1.0 / (1.0 + sqrtT * 3.1622776601683794e-3);
    r.ce = 7.5e-19 * ex * inv_den;
    r.ce_T = r.ce * (118348.0 * invT * invT - (0.5 * 3.1622776601683794e-3) * sqrtT * invT * inv_den);
    // bremsstrahlung 1.42e-27 g_ff sqrt(T), g_ff = 1.1 + 0.34 e^{-(5.5 - log10 T)^2 / 3}
    const double dl = 5.5 - logT * 0.43429448190325176;
    const double eg = fexp(dl * dl * (-1.0 / 3.0));
    const double gff = 1.1 + 0.34 * eg;
    const double gff_T = 0.34 * eg * (2.0 / 3.0) * dl * 0.43429448190325176 * invT;
    const double ff = 1.42e-27 * gff * sqrtT;
    const double ff_T = 1.42e-27 * (gff_T * sqrtT + 0.5 * gff * sqrtT * invT);
    r.rf = rec + ff;
    r.rf_T = rec_T + ff_T;
    // Compton scattering off the CMB, per electron
    const double Tcmb = 2.725 / P.a;
    const double kcomp = 4.0 * 1.380649e-16 * 6.6524587321e-25 * 7.565723e-15 / (9.1093837015e-28 * 2.99792458e10);
    const double k4 = kcomp * (Tcmb * Tcmb) * (Tcmb * Tcmb);
    r.comp = k4 * (T - Tcmb);
    r.comp_T = k4;
    return r;
}

// q = e^-x and p1 = (1 - e^-x)/x for x >= 0 with dp1/dx (dq/dx = -q): below x = 1/32 from the
// Taylor series of p1, sum_k (-x)^k / (k+1)!, truncated after x^7 (p1) and x^7 (p1'), both
// within 1e-17 relative there; above it, 1 - e^-x loses at most a factor 32 in relative accuracy
RT_HD void decay_pair(double x, double& q, double& p1, double& p1_x) {
    if (x < 0.03125) {
        // p1 = 1 - x/2 + x^2/6 - x^3/24 + x^4/120 - x^5/720 + x^6/5040 - x^7/40320
        double h = fma(x, -1.0 / 40320.0, 1.0 / 5040.0);
        h = fma(h, x, -1.0 / 720.0);
        h = fma(h, x, 1.0 / 120.0);
        h = fma(h, x, -1.0 / 24.0);
        h = fma(h, x, 1.0 / 6.0);
        h = fma(h, x, -0.5);
        p1 = fma(h, x, 1.0);
        // p1' = -1/2 + 2x/6 - 3x^2/24 + 4x^3/120 - 5x^4/720 + 6x^5/5040 - 7x^6/40320 + 8x^7/362880
        double g = fma(x, 8.0 / 362880.0, -7.0 / 40320.0);
        g = fma(g, x, 6.0 / 5040.0);
        g = fma(g, x, -5.0 / 720.0);
        g = fma(g, x, 4.0 / 120.0);
        g = fma(g, x, -3.0 / 24.0);
        g = fma(g, x, 2.0 / 6.0);
        p1_x = fma(g, x, -0.5);
        q = fma(-x, p1, 1.0);
    } else {
        q = fexp(-x);
        const double ix = 1.0 / x;
        p1 = (1.0 - q) * ix;
        p1_x = (q - p1) * ix;
    }
}

// S_n = n(dt) of n' = A (nH - n)^2 - G n, n(0) = y0, in the Bernoulli form of riccati_n
// (physics.cuh), with its partials in A and G
struct Riccati {
    double v, A, G;
};
RT_HD Riccati riccati_ag(double y0, double nH, double A, double G, double dt) {
    Riccati o;
    const double d = sqrt(G * G + 4.0 * nH * (A * G));
    const double id = d > 0.0 ? 1.0 / d : 0.0;
    const double d_A = 2.0 * nH * G * id, d_G = (G + 2.0 * nH * A) * id;
    const double den = 2.0 * nH * A + G + d;
    double yeq = 0.0, yeq_A = 0.0, yeq_G = 0.0;
    if (den > 0.0) {
        const double iden = 1.0 / den;
        yeq = (2.0 * nH * nH) * A * iden;
        yeq_A = (2.0 * nH * nH - yeq * (2.0 * nH + d_A)) * iden;
        yeq_G = -yeq * (1.0 + d_G) * iden;
    }
    const double u0 = y0 - yeq;
    double q, p1, p1_x;
    decay_pair(d * dt, q, p1, p1_x);
    const double q_A = -q * d_A * dt, q_G = -q * d_G * dt;
    const double p1_A = p1_x * d_A * dt, p1_G = p1_x * d_G * dt;
    // D = 1 - dt u0 A p1, S_n = yeq + u0 q / D
    const double D = 1.0 - (u0 * A) * (dt * p1);
    const double D_A = -dt * ((-yeq_A * A + u0) * p1 + u0 * A * p1_A);
    const double D_G = -dt * (-yeq_G * A * p1 + u0 * A * p1_G);
    const double iD = 1.0 / D;
    const double R = u0 * q * iD;
    o.v = yeq + R;
    o.A = yeq_A + (-yeq_A * q + u0 * q_A - R * D_A) * iD;
    o.G = yeq_G + (-yeq_G * q + u0 * q_G - R * D_G) * iD;
    return o;
}

// S_e, S_n at the iterate (e_c, n, E) and their partials in (e_c, n, E)
struct HLocal {
    double Se, Sn;
    double Se_e, Se_n, Se_E;
    double Sn_e, Sn_n, Sn_E;
};

template <bool ISO>
RT_HD HLocal h_local(const PhysParams& P, const HCell& c, double ec, double n, double E) {
    HLocal o;
    // theta-weighted energy through the smooth positive part; d spos(x)/dx = spos(x) / r
    const double x = P.theta * E + (1.0 - P.theta) * c.E0;
    const double r = sqrt(x * x + P.E_min * P.E_min);
    const double Ebar = x < 0.0 ? (P.E_min * P.E_min) / (2.0 * (r - x)) : 0.5 * (x + r);
    const double Ebar_E = P.theta * Ebar / r;
    const double kGa = P.kG * c.inv_a3;
    const double G = kGa * Ebar;
    const double G_E = kGa * Ebar_E;
    double T, invT, T_e = 0.0, T_n = 0.0;
    if (ISO) {
        T = P.T_iso;
        invT = 1.0 / T;
    } else {
        // T = kTr e / m with e = e_int, m = 2 rho - n: 1/m = kTr e w and 1/T = m^2 w, w = 1/(kTr e m)
        const double e = c.eh_kin + ec, m = 2.0 * c.rho - n;
        const double kTe = c.kTr * e;
        const double w = 1.0 / (kTe * m);
        const double inv2 = kTe * w;
        T = kTe * inv2;
        invT = (m * m) * w;
        if (T < RT_T_FLOOR) {
            T = RT_T_FLOOR;
            invT = 1.0 / RT_T_FLOOR;
        } else {
            T_e = c.kTr * inv2;
            T_n = T * inv2;
        }
    }
    const bool cool = !ISO && P.cooling;
    const HRates rt = h_rates(P, T, invT, P.recomb != 0, cool);
    const double A = rt.alpha * c.Ak;
    const double A_T = rt.alpha_T * c.Ak;
    const Riccati R = riccati_ag(c.y0, c.rho, A, G, P.dt);
    o.Sn = R.v;
    o.Sn_e = R.A * A_T * T_e;
    o.Sn_n = R.A * A_T * T_n;
    o.Sn_E = R.G * G_E;
    if (ISO) {
        o.Se = o.Se_e = o.Se_n = o.Se_E = 0.0;
        return o;
    }
    const double heat = c.hk * n * Ebar;
    double cool_v = 0.0, cool_T = 0.0, cool_n = 0.0;
    if (cool) {
        const double s = P.un * c.inv_a3;
        const double nHII = (c.rho - n) * s;                 // = n_e
        const double nHIp = n * s;
        const double L = (rt.rf * nHII + rt.ce * nHIp) + rt.comp;
        cool_v = c.ck * (L * nHII);
        cool_T = c.ck * ((rt.rf_T * nHII + rt.ce_T * nHIp) + rt.comp_T) * nHII;
        cool_n = c.ck * ((rt.ce - rt.rf) * s * nHII - L * s);
    }
    o.Se = (heat - cool_v) * P.phi_e;
    o.Se_e = -P.phi_e * cool_T * T_e;
    o.Se_n = P.phi_e * (c.hk * Ebar - cool_n - cool_T * T_n);
    o.Se_E = P.phi_e * c.hk * n * Ebar_E;
    return o;
}
