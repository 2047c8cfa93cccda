/* Prints the size and every field offset of the C ABI's structs (include/rt.h) as JSON, so
 * that a test can compare them with the ctypes mirrors of the Python binding. */
#include <stddef.h>
#include <stdio.h>

#include "../../include/rt.h"

#define F(T, f) printf("\"%s\": %zu, ", #f, offsetof(T, f))
#define OPEN(T) printf("\"%s\": {\"__size__\": %zu, ", #T, sizeof(T))
#define CLOSE() printf("\"__end__\": 0}")

int main(void) {
    printf("{");
    OPEN(rt_grid_desc);
    F(rt_grid_desc, nx); F(rt_grid_desc, ny); F(rt_grid_desc, nz); F(rt_grid_desc, dx); F(rt_grid_desc, bc);
    F(rt_grid_desc, u_x); F(rt_grid_desc, u_t); F(rt_grid_desc, u_g); F(rt_grid_desc, theta);
    F(rt_grid_desc, precision); F(rt_grid_desc, isothermal); F(rt_grid_desc, T_iso); F(rt_grid_desc, spectrum);
    F(rt_grid_desc, T_B); F(rt_grid_desc, recomb); F(rt_grid_desc, cooling); F(rt_grid_desc, helium);
    F(rt_grid_desc, Y); F(rt_grid_desc, limiter); F(rt_grid_desc, D_const); F(rt_grid_desc, E_min);
    F(rt_grid_desc, newton_tol); F(rt_grid_desc, max_newton); F(rt_grid_desc, lin_rtol); F(rt_grid_desc, max_lin);
    F(rt_grid_desc, mg_nu1); F(rt_grid_desc, mg_nu2); F(rt_grid_desc, device); F(rt_grid_desc, stream);
    CLOSE();
    printf(", ");
    OPEN(rt_step_inputs);
    F(rt_step_inputs, rho_b); F(rt_step_inputs, e_h); F(rt_step_inputs, vx); F(rt_step_inputs, vy);
    F(rt_step_inputs, vz); F(rt_step_inputs, clump); F(rt_step_inputs, a); F(rt_step_inputs, adot);
    F(rt_step_inputs, dt); F(rt_step_inputs, nsrc); F(rt_step_inputs, src_cell); F(rt_step_inputs, src_ndot);
    CLOSE();
    printf(", ");
    OPEN(rt_state);
    F(rt_state, E); F(rt_state, n_HI); F(rt_state, e_c); F(rt_state, n_HeI); F(rt_state, n_HeII);
    CLOSE();
    printf(", ");
    OPEN(rt_step_stats);
    F(rt_step_stats, newton_iters); F(rt_step_stats, residual_evals); F(rt_step_stats, linear_iters);
    F(rt_step_stats, line_search_cuts); F(rt_step_stats, norm0); F(rt_step_stats, norm);
    F(rt_step_stats, change_norm); F(rt_step_stats, kernel_launches); F(rt_step_stats, nhist);
    F(rt_step_stats, hist_norm); F(rt_step_stats, hist_lam); F(rt_step_stats, hist_cg);
    CLOSE();
    printf(", ");
    OPEN(rt_kernel_profile);
    F(rt_kernel_profile, name); F(rt_kernel_profile, launches); F(rt_kernel_profile, ms); F(rt_kernel_profile, bytes);
    CLOSE();
    printf("}\n");
    return 0;
}
