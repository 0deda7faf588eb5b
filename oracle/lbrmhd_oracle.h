/*
 * lbrmhd_oracle.h -- TEST INFRASTRUCTURE, not part of the product.
 *
 * Declarations of the FP64 CPU oracle of the lattice Boltzmann model for
 * resistive relativistic MHD (arXiv:1508.03452). Only the tests, the smoke
 * check and the benchmark's CPU-baseline legs use this. The CUDA library never
 * includes it.
 *
 * Parity status of each function against the paper:
 *   orc_feq, orc_geq, orc_heq, orc_moments, orc_em_ff, orc_landau,
 *   orc_ohm_current, orc_ohm_solve, orc_recover_cell: pinned (moment identities
 *     against the printed tensors, numpy eigen-solve, direct 3x3 solve,
 *     printed Alfven speed, closed-form limits).
 *   orc_stream_population: the flux function is a reading (the paper defers it
 *     to another paper): parity unpinned; its properties (uniform state,
 *     conservation, first-order limit, second-order convergence) are pinned.
 *   bulk-viscosity coefficient, normal-B fix, driving: parity unpinned.
 */
#ifndef LBRMHD_ORACLE_H
#define LBRMHD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_PERIODIC 0
#define ORC_OPEN 1
#define ORC_DRIVEN 2

/* test switches */
#define ORC_NO_EM_COLLISION 1 /* h is only streamed: h(x + v dt, t + dt) = h(x, t) */
#define ORC_FIRST_ORDER 2     /* limiter phi = 0: first-order upwind streaming */
#define ORC_IMPLICIT_AS_PRINTED 4 /* collision term implicit in f(t+dt) towards f^eq(t) */
#define ORC_PRINTED_FEQ 8     /* delta_{i0} term and nu^2/5 sign of Eq. Dis_fun_EM exactly as printed */
#define ORC_ONE_PASS_RECOVERY 16 /* eigen-solve once, with E and B of the previous step (R24 taken literally) */
#define ORC_GAUSS_CHARGE 32   /* R28 (option): Ohm's convection current with the charge eps0 div E (Eq. Gauss_E) */

/* primitive layout of one cell (field-major planes in the simulation) */
#define ORC_N 0
#define ORC_EPS 1
#define ORC_U 2
#define ORC_E 5
#define ORC_B 8
#define ORC_RHOC 11
#define ORC_J 12
#define ORC_NPRIM 15

typedef struct orc_params {
    int32_t nx, ny, nz;
    int32_t bc[6];        /* -x,+x,-y,+y,-z,+z: ORC_PERIODIC | ORC_OPEN | ORC_DRIVEN (-z only) */
    double tau;           /* fluid relaxation time in units of dt */
    double sigma;         /* conductivity */
    double gamma_ad;      /* adiabatic index of Eq. EOS */
    double alpha;         /* bulk-viscosity constant */
    double c;             /* speed of light; dt = dx / (sqrt(2) c) */
    double dx;            /* lattice spacing */
    double nu;            /* temperature parameter; <= 0 selects sqrt(27) */
    double drive_u0;      /* peak drive speed of the driven layers */
    int32_t drive_layers; /* number of driven z-layers above the -z face */
    int32_t flags;        /* ORC_NO_EM_COLLISION | ORC_FIRST_ORDER | ORC_IMPLICIT_AS_PRINTED | ORC_PRINTED_FEQ |
                             ORC_ONE_PASS_RECOVERY */
    int32_t threads;      /* OpenMP threads (0: runtime default) */
    int32_t max_power_iters;
    double power_tol;
    double drive_f0;      /* R25: amplitude of the photospheric body force (0: none) */
    double drive_vmax;    /* R26: the force acts while max |u| < drive_vmax (<= 0: always) */
} orc_params;

typedef struct orc_lattice {
    double nu, ca, ct_c0, c0, ct;
    double w[19], wg[19];
    double p[19][4];
    int chat[19][3];
    double v[24][3], e[24][3], b[24][3];
    int hop[24][3];
} orc_lattice;

typedef struct orc_sim orc_sim;

void orc_lattice_init(const orc_params* P, orc_lattice* L);
void orc_get_lattice(const orc_params* P, orc_lattice* L);
double orc_dt(const orc_params* P);
double orc_courant(const orc_params* P, const orc_lattice* L);
double orc_eos_pressure(const orc_params* P, double n, double eps);

void orc_feq(const orc_params* P, const orc_lattice* L, double n, double eps, const double* u,
             const double* E, const double* B, double* feq);
void orc_geq(const orc_params* P, const orc_lattice* L, double n, const double* u, double* geq);
void orc_heq(const orc_params* P, const orc_lattice* L, const double* E, const double* B, const double* J,
             double rho_c, double* heq);
void orc_ohm_current(const orc_params* P, const double* E, const double* u, const double* B, double rho_c,
                     double* J);
void orc_ohm_solve(const orc_params* P, const double* Ep, const double* u, const double* B, double rho_c,
                   double* E);
void orc_moments(const orc_lattice* L, const double* f, const double* g, const double* h, double* T16,
                 double* N4, double* Ep, double* B, double* rho_c);
void orc_maxwell_tensor(double c, const double* E, const double* B, double* F16);
void orc_em_ff(const orc_params* P, const double* E, const double* B, double* S16);
int orc_landau(const orc_params* P, const double* T16, const double* E_prev, const double* B_prev,
               const double* U_seed, double* U_out, double* lambda_out);
int orc_recover_cell(const orc_params* P, const orc_lattice* L, const double* f, const double* g,
                     const double* h, const double* prim_prev, double* prim_out);
int orc_recover_cell_rho(const orc_params* P, const orc_lattice* L, const double* f, const double* g,
                         const double* h, const double* prim_prev, double rho_ohm, double* prim_out);
void orc_stream_population(const orc_params* P, int i, const double* fi, double* out);
void orc_drive_velocity(const orc_params* P, int x, int y, double* u);
void orc_drive_force(const orc_params* P, int x, int y, double* F);
void orc_force_populations(const orc_params* P, const orc_lattice* L, const double* F, const double* u, double* df);

orc_sim* orc_create(const orc_params* P);
void orc_destroy(orc_sim* s);
int orc_init(orc_sim* s, const double* n, const double* p, const double* u, const double* B, const double* E);
int orc_step(orc_sim* s, int64_t nsteps);
int orc_force_on(const orc_sim* s);
int orc_init_relaxed(orc_sim* s, const double* n, const double* p, const double* u, const double* B, int max_iters,
                     double tol, double* residual);
void orc_get_moments(const orc_sim* s, double* out);
void orc_get_state(const orc_sim* s, double* f, double* g, double* h, double* prim);
void orc_set_state(orc_sim* s, const double* f, const double* g, const double* h, const double* prim);
int orc_update_cells(orc_sim* s, const int64_t* cells, int64_t ncells, double* f_out, double* g_out,
                     double* h_out, double* prim_out);
void orc_get_post_collision(orc_sim* s, double* fc, double* gc, double* hc);
int orc_update_cells_from(orc_sim* s, const double* fc, const double* gc, const double* hc, const double* prim,
                          const int64_t* cells, int64_t ncells, double* f_out, double* g_out, double* h_out,
                          double* prim_out);
void orc_stats(const orc_sim* s, int64_t* out4);

#ifdef __cplusplus
}
#endif
#endif
