// Host build of the Newton kernel's hydrogen local equations with written-out partials
// (hlocal.cuh) next to the dual-number evaluation (physics.cuh local_solutions<Dual<3>>), at n
// cell states: out[k][i] for k = Se, Sn, dSe/d(ec, n, E), dSn/d(ec, n, E), for each of the two.
#include <cstring>

#include "../../paper_0908_2654_gb300/csrc/hlocal.cuh"

extern "C" void hlocal_host(int n, const double* prm, const double* rho, const double* y0, const double* E0,
                            const double* eh, const double* clump, const double* ec, const double* nHI,
                            const double* E, double* out_h, double* out_d) {
    PhysParams P;
    std::memset(&P, 0, sizeof(P));
    P.a = prm[0];
    P.a3 = P.a * P.a * P.a;
    P.dt = prm[1];
    P.theta = prm[2];
    P.kG = prm[3];
    P.kT = prm[4];
    P.kA = prm[5];
    P.kH = prm[6];
    P.kC = prm[7];
    P.un = prm[8];
    P.E_min = prm[9];
    P.T_iso = prm[10];
    P.phi_e = prm[11];
    P.isothermal = (int)prm[12];
    P.recomb = (int)prm[13];
    P.cooling = (int)prm[14];
    P.alpha_const = 2.59e-13;
    const double inv_a3 = 1.0 / P.a3;
    for (int i = 0; i < n; ++i) {
        const HCell c = make_hcell(P, inv_a3, rho[i], y0[i], E0[i], eh[i], clump[i]);
        const HLocal L = P.isothermal ? h_local<true>(P, c, ec[i], nHI[i], E[i]) : h_local<false>(P, c, ec[i], nHI[i], E[i]);
        const double h[8] = {L.Se, L.Sn, L.Se_e, L.Se_n, L.Se_E, L.Sn_e, L.Sn_n, L.Sn_E};
        CellIn ci;
        ci.rho = rho[i];
        ci.nHI0 = y0[i];
        ci.E0 = E0[i];
        ci.eh_kin = eh[i];
        ci.clump = clump[i];
        Dual<3> Se, Sn;
        local_solutions<Dual<3>>(P, ci, dvar<3>(ec[i], 0), dvar<3>(nHI[i], 1), dvar<3>(E[i], 2), Se, Sn);
        const double d[8] = {Se.v, Sn.v, Se.d[0], Se.d[1], Se.d[2], Sn.d[0], Sn.d[1], Sn.d[2]};
        for (int k = 0; k < 8; ++k) {
            out_h[k * n + i] = h[k];
            out_d[k * n + i] = d[k];
        }
    }
}
