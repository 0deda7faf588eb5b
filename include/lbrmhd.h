/*
 * lbrmhd.h -- C ABI of the GB300 (sm_103a) lattice Boltzmann solver for
 * resistive relativistic magnetohydrodynamics of Mohseni, Mendoza, Succi and
 * Herrmann, "Lattice Boltzmann model for resistive relativistic
 * magnetohydrodynamics" (arXiv:1508.03452).
 *
 * One time step (Sec. III) is one fused CUDA kernel per run: the flux-limited
 * streaming of the D3Q19 energy-momentum populations f and number-density
 * populations g (Eq. eq:rlb, Eq. Hupp), the exact streaming of the D3Q13
 * Maxwell populations h (Eq. LB_Maxwell), the moments (Eqs. Cal_E, Cal_B,
 * Cal_rhoc, T = sum p p f, N = sum p g), the Landau eigen-solve for U and eps,
 * n = N^0/U^0, the Ohm-coupled E solve (Eqs. Ohm, Ex_force), the equation of
 * state (Eq. EOS), and the Anderson-Witting / BGK / tau_h = 1/2 collisions
 * towards the equilibria Eq. Dis_fun_EM, Eq. Hupp and Eq. Maxwell-eq. Open
 * boundaries, the normal-B adjustment and the photospheric driving (Sec. IV)
 * follow as small kernels.
 *
 * Units: mu_0 = 1, eps_0 = 1 / c^2, dt = dx / (sqrt(2) c) (time-step
 * synchronisation of Sec. III); tau is in units of dt.
 *
 * Conventions for every call:
 *   - Return value: LBRMHD_OK (0) or a negative LBRMHD_ERR_* code; the message
 *     of the last failure is returned by lbrmhd_last_error(handle) (or
 *     lbrmhd_last_error(NULL) for a failed lbrmhd_create).
 *   - Ownership: the library allocates and owns all device memory of a handle;
 *     caller arrays are only read or written during the call (host arrays are
 *     copied; device arrays must stay valid until the call's work on the
 *     handle's stream has finished).
 *   - Layout of caller field arrays: float64, x fastest, cell index
 *     x + nx (y + ny z); a vector field is three consecutive planes of N = nx ny
 *     nz values (x components, then y, then z).
 *   - Threading: a handle must not be used from two threads at once. All work
 *     is issued on the handle's stream (lbrmhd_set_stream); calls that return
 *     host data synchronise that stream.
 *   - The library never falls back to a CPU path: without a usable sm_103a GPU
 *     lbrmhd_create fails with LBRMHD_ERR_CUDA.
 */
#ifndef LBRMHD_H
#define LBRMHD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBRMHD_OK 0
#define LBRMHD_ERR_BAD_ARG (-1)      /* invalid argument or parameter */
#define LBRMHD_ERR_OOM (-2)          /* device or host allocation failed */
#define LBRMHD_ERR_CUDA (-3)         /* a CUDA runtime call failed */
#define LBRMHD_ERR_NONCONVERGED (-4) /* recoveries failed to converge: lbrmhd_step is asynchronous, so the
                                        failures are counted per run (lbrmhd_get_stats, recover_fail), their
                                        cells keep their previous primitives, and lbrmhd_get_status returns
                                        this code */
#define LBRMHD_ERR_NONFINITE (-5)    /* a NaN or Inf was found by the diagnostics */
#define LBRMHD_ERR_TIMEOUT (-6)      /* a kernel's bounded wait for its own tile copies ran out (the block
                                        skipped its update); returned by lbrmhd_get_status */
#define LBRMHD_ERR_STATE (-7)        /* call out of order (e.g. step before init_fields) */

/* boundary kinds, per face -x,+x,-y,+y,-z,+z */
#define LBRMHD_PERIODIC 0
#define LBRMHD_OPEN 1   /* copy of the first interior cell + normal-B fix (Sec. IV, KH and flare set-ups) */
#define LBRMHD_DRIVEN 2 /* -z face only: open, and the lowest drive_layers layers driven */

/* population storage / arithmetic */
#define LBRMHD_FP64 0      /* float64 storage and arithmetic */
#define LBRMHD_FP32 1      /* float32 storage (f, g as deviations from the rest equilibrium), float32 arithmetic */
#define LBRMHD_FP16_DEV 2  /* f, g as float16 relative deviations from the rest equilibrium; h, primitives float32 */

/* primitive recovery seed: the starting vector of the Landau eigen-solve of
 * Sec. III (coupling). Every mode iterates to the same tolerance, so the seed
 * changes the iteration count, not the converged primitives. */
#define LBRMHD_RECOVERY_PLAIN 0 /* seeded with the previous step's velocity */
#define LBRMHD_RECOVERY_MLP 1   /* seeded by the learned network (lbrmhd_set_mlp_weights) */
#define LBRMHD_RECOVERY_COLD 2  /* seeded with zero velocity (no history) */

/* switches (flags) */
#define LBRMHD_FLAG_NO_EM_COLLISION 1 /* h is streamed without collision: h(x + v dt, t + dt) = h(x, t) */
#define LBRMHD_FLAG_UNSHIFTED_POWER 2 /* recovery by the plain power method (no spectral shift) */
#define LBRMHD_FLAG_ONE_PASS_RECOVERY 4 /* one eigen-solve with the previous step's E, B (the coupling
                                          subsection taken literally: loses the EM inertia, see the
                                          self-consistent recovery in lbrmhd_step) */
#define LBRMHD_FLAG_GAUSS_CHARGE 8 /* an option beyond the paper: the charge of Ohm's convection current rho_c u
                                      (Eq. Ohm) from Gauss's law, eps0 div E of the previous step's E by central
                                      differences (Eq. Gauss_E), instead of the Maxwell moment sum h (Eq.
                                      Cal_rhoc), which carries a grid-scale mode that any flow amplifies; with
                                      alpha <= 0.02 it keeps flowing magnetised plasma stable */
#define LBRMHD_FLAG_TMA_TILES 16 /* 2-D periodic runs stored in float32 / float16 step by the TMA tile
                                    kernel: persistent blocks stream 32 x 8-cell tiles whose populations and
                                    halo arrive by tensor-map copies through a ring of shared-memory buffers,
                                    stencil reads from shared memory, populations out by the cells' vector
                                    stores and primitives by a tensor-map store, plus a per-cell launch over
                                    the edge tiles. The same update as the default per-cell kernel (to float
                                    rounding); not faster on GB300 (the block-wide waits per ring stage cost
                                    as much as the vector loads they replace), so it is an option, not the
                                    default. Ignored with LBRMHD_FLAG_GAUSS_CHARGE and under the BATCH
                                    and PERSISTENT schedules. */
#define LBRMHD_FLAG_FIRST_ORDER_FLUX 32 /* a study option, not the paper's scheme: the fluid face fluxes without
                                           the minmod-limited correction (Sec. III streaming, reading of h_i^a),
                                           i.e. plain first-order upwind, as the limiter gives at a discontinuity */

/* rows of lbrmhd_get_moments output (each row N values) */
#define LBRMHD_NMOMENTS 16 /* n, p, eps, u(3), E(3), B(3), rho_c, J(3) */

/* lbrmhd_get_diagnostics output */
#define LBRMHD_NDIAG 10
/* [0] sum N^0  [1..4] sum T^{0 nu}  [5] sum rho_c  [6] max |div B|  [7] rms div B
 * [8] non-finite cell count  [9] number of cells */

typedef struct lbrmhd_params {
    int32_t nx, ny, nz;     /* grid; nz = 1 is a 2-D run, ny = nz = 1 a 1-D run */
    int32_t bc[6];          /* LBRMHD_PERIODIC | LBRMHD_OPEN | LBRMHD_DRIVEN per face -x,+x,-y,+y,-z,+z */
    double tau;             /* fluid relaxation time in units of dt (> 0.5 for stability) */
    double sigma;           /* conductivity of Eq. Ohm (>= 0) */
    double gamma_ad;        /* adiabatic index of Eq. EOS (> 1) */
    double alpha;           /* bulk-viscosity constant of Eq. eq:rlb (>= 0) */
    double c;               /* numerical speed of light (> 0); dt = dx / (sqrt(2) c) */
    double dx;              /* lattice spacing (> 0) */
    double drive_u0;        /* peak speed of the driven photospheric layers */
    int32_t drive_layers;   /* number of driven z-layers (LBRMHD_DRIVEN on -z) */
    int32_t precision;      /* LBRMHD_FP64 | LBRMHD_FP32 | LBRMHD_FP16_DEV (same for every run of a handle) */
    int32_t recovery;       /* LBRMHD_RECOVERY_PLAIN | LBRMHD_RECOVERY_MLP | LBRMHD_RECOVERY_COLD */
    int32_t flags;          /* LBRMHD_FLAG_* */
    int32_t max_iters;      /* recovery iteration cap (0: 64) */
    double tol;             /* recovery tolerance (0: 1e-14 for FP64, 1e-6 otherwise) */
    double drive_f0;        /* photospheric body force of the flare set-up (Sec. IV): amplitude F0 of the
                               two-vortex force density F = F0 (sin(pi xs/3) cos(pi y/6), cos(pi xs/3) sin(pi y/6), 0)
                               on x, y in [-3, 3] (xs = x on x < 0, x - 3 on x >= 0), applied in the lowest
                               drive_layers z-layers; it adds c F dt to T^{0a} and F.u dt to T^00 of the streamed
                               fluid populations each step. 0: no force. Not with LBRMHD_DRIVEN. */
    double drive_vmax;      /* the force acts while the largest |u| of the state is below drive_vmax
                               (the paper's 0.3 c); <= 0: always */
} lbrmhd_params;

typedef struct lbrmhd_state_s* lbrmhd_handle;

/* Creates n_runs independent runs (params[0..n_runs-1]; grids may differ) and
 * allocates their device state: per run two copies (read / write) of the 19 +
 * 19 + 25 populations and 12 primitive fields per cell (element offsets in 64
 * bits; a run may hold up to 2^29 cells, the range of the step kernel's 32-bit
 * stencil offsets). Errors: BAD_ARG for any invalid parameter (grid < 1 or
 * above 2^29 cells, c, dx or tau <= 0, sigma < 0, gamma_ad <= 1, DRIVEN on a
 * face other than -z, precision mixed across runs), OOM, CUDA (no usable
 * GPU). On failure *out is NULL. */
int lbrmhd_create(const lbrmhd_params* params, int n_runs, lbrmhd_handle* out);

/* Frees all device memory of the handle. A NULL handle is ignored. */
int lbrmhd_destroy(lbrmhd_handle h);

/* Issues all further work on `stream` (a cudaStream_t; NULL = the legacy
 * default stream). The caller keeps ownership of the stream. */
int lbrmhd_set_stream(lbrmhd_handle h, void* stream);

/* Initial state of one run from host arrays (Sec. IV set-ups): n, p (N values),
 * u, B (3N), E (3N, or NULL for the ideal-MHD field E = -u x B of Eq.
 * Ohm_ideal). eps from Eq. EOS, rho_c = eps0 div E by central differences
 * (Eq. Gauss_E), J from Eq. Ohm, every population at its equilibrium.
 * Errors: BAD_ARG (run out of range, NULL array, |u| >= c), CUDA. */
int lbrmhd_init_fields(lbrmhd_handle h, int run, const double* n, const double* p, const double* u,
                       const double* B, const double* E);

/* As lbrmhd_init_fields with device arrays (float64, same layout). */
int lbrmhd_init_fields_device(lbrmhd_handle h, int run, const double* n, const double* p, const double* u,
                              const double* B, const double* E);

/* Initial state of one run whose E, J have relaxed under the scheme (the
 * iterative initialisation of the flare set-up, Sec. IV): from the state of
 * lbrmhd_init_fields(n, p, u, B, E = NULL), repeat one step of this run (no
 * body force) in which, after the recovery and before the boundary pass,
 * every cell is held at the given n, p, u, B: f and g at their equilibria,
 * the B carried by h moved back to B (h_k += (B0 - B).b_k / 8; E' and rho_c
 * unchanged), J from Eq. Ohm; E and rho_c evolve. Stops when max |E_k - E_{k-2}| <= tol max |E_k| (k: the step
 * count; E_{-1} = the initial E) or after max_iters steps. Writes the steps
 * taken to *iters and that ratio of the last step to *residual (either may be
 * NULL); the run then starts at step 0 with zero counters. Host arrays as in
 * lbrmhd_init_fields; synchronises the stream once per step. Other runs of the
 * handle are untouched. Errors: BAD_ARG (as lbrmhd_init_fields, max_iters < 1,
 * tol < 0, a run with LBRMHD_DRIVEN), OOM, CUDA. */
int lbrmhd_init_fields_relaxed(lbrmhd_handle h, int run, const double* n, const double* p, const double* u,
                               const double* B, int max_iters, double tol, int* iters, double* residual);

/* Advances every run by nsteps time steps (asynchronous on the handle's
 * stream). The primitive recovery is self-consistent: the eigen-solve of the
 * coupling subsection (Sec. III) starts from the previous step's E and is
 * repeated with the E that Ohm's law gives for the recovered velocity (and
 * the streamed B) until that E reproduces itself, so that the collision
 * conserves T^{mu nu} and the EM momentum keeps its inertia. Recovery failures are counted per run (lbrmhd_get_stats) and the
 * affected cells keep their previous primitives. Errors: STATE (a run was
 * never initialised), BAD_ARG (nsteps < 0), CUDA. */
int lbrmhd_step(lbrmhd_handle h, int64_t nsteps);

/* Macroscopic fields of one run, LBRMHD_NMOMENTS rows of N float64 values:
 * n, p, eps, u(3), E(3), B(3), rho_c, J(3) (J from Eq. Ohm). Host output;
 * synchronises the stream. */
int lbrmhd_get_moments(lbrmhd_handle h, int run, double* out);

/* As lbrmhd_get_moments into a device array of LBRMHD_NMOMENTS * N float64;
 * asynchronous. */
int lbrmhd_get_moments_device(lbrmhd_handle h, int run, double* out);

/* Post-collision populations of one run (the populations the next step
 * streams), float64 on the host: f (19 N), g (19 N), h (25 N), population-major
 * in the order of the D3Q19 table (rest; +x,-x,+y,-y,+z,-z; +x+y,-x-y,+x-y,
 * -x+y; +x+z,-x-z,+x-z,-x+z; +y+z,-y-z,+y-z,-y+z) and of the D3Q13 table
 * (k = 8 p + 2 i + j, then the rest population). Any pointer may be NULL. */
int lbrmhd_get_populations(lbrmhd_handle h, int run, double* f, double* g, double* hh);

/* Conservation diagnostics of one run (LBRMHD_NDIAG float64 values, see
 * above) computed from the current state with float64 reductions. Returns
 * NONFINITE if any cell holds a NaN or Inf. Host output. */
int lbrmhd_get_diagnostics(lbrmhd_handle h, int run, double* out);

/* Diagnostics for callers that cannot allocate device memory when they need
 * them: for instance a monitor running while another framework's memory pool
 * owns the free device memory (a new cudaMalloc could fail even though the
 * reduction needs only a few kilobytes), or a time-critical loop that must not
 * pay the device-wide synchronisation that cudaMalloc / cudaFree may imply.
 * The paper has no counterpart; this is a library facility.
 *
 * Same values as lbrmhd_get_diagnostics (LBRMHD_NDIAG float64, same order),
 * but this call allocates nothing and copies nothing to the host: the
 * per-block partial sums of the reduction live in a fixed static device array
 * of this library (4.7 MB on every GPU that loads the library, held until the
 * process exits), and the results are written to d_out, a caller-owned device
 * array of at least LBRMHD_NDIAG float64. The work is queued on the handle's
 * stream and the call returns without waiting; d_out is valid once that
 * stream reaches this point.
 *
 * Limits and rules:
 *   - runs of at most 16,777,216 cells (256^3); larger runs are rejected with
 *     LBRMHD_ERR_BAD_ARG and a message naming the limit.
 *   - lbrmhd_create looks up the device address of the static array, with the
 *     handle's device current, and keeps it in the handle; this call itself
 *     makes no lookup and no allocation.
 *   - Every call shares the one array, which keeps the previous call's
 *     contents; each call writes every entry it later reads, so no clearing is
 *     needed. Calls whose work overlaps on the GPU (other streams, other
 *     threads, other handles on the same device) race on the array and must be
 *     serialised by the caller.
 *   - The non-finite count is returned in d_out[8]; unlike
 *     lbrmhd_get_diagnostics this call cannot report NONFINITE in its return
 *     value, since it does not wait for the result.
 * Errors: BAD_ARG (run out of range, NULL d_out, run above the limit), STATE
 * (run not initialised), CUDA. */
int lbrmhd_get_diagnostics_noalloc(lbrmhd_handle h, int run, double* d_out);

/* Reconnection rate of a 2-D run (Sec. IV, Kelvin-Helmholtz-driven
 * reconnection): R = (E^z - E^z_0) / B0 at the null point, E^z_0 being the
 * out-of-plane electric field of the run's initial state (kept from
 * lbrmhd_init_fields, and in checkpoints). The null point is the cell of
 * smallest B_x^2 + B_y^2 in rows y_lo <= y < y_hi (the band names one current
 * layer; ties go to the lowest cell index), found again at every call, so it
 * follows the layer as it moves. out4 (host): R, x, y and |B_in-plane| at the
 * null (NaN if the band holds no finite field). Synchronises the handle's
 * stream. Errors: BAD_ARG (run out of range, 3-D run, empty or out-of-grid
 * band, B0 zero or not finite), STATE (run not initialised), CUDA. */
int lbrmhd_reconnection_rate(lbrmhd_handle h, int run, int y_lo, int y_hi, double B0, double* out4);

/* Counters of one run: [0] steps taken, [1] recovery failures, [2] sum of
 * recovery iterations, [3] maximum recovery iterations. Host output. */
int lbrmhd_get_stats(lbrmhd_handle h, int run, int64_t* out4);

/* Health of the whole handle, for a caller that steps asynchronously and
 * checks now and then. Synchronises the handle's stream. out3 (host, may be
 * NULL): [0] status bits raised by the step kernels since lbrmhd_create (1: a
 * TMA tile copy did not arrive within its wait limit, and that tile's update
 * was skipped; 2: a persistent launch's grid barrier gave up waiting, and the
 * launch's remaining steps were skipped), [1] recovery failures summed over every run since its
 * initialisation, [2] number of runs that step by the TMA tile kernel
 * (LBRMHD_FLAG_TMA_TILES).
 * Returns LBRMHD_ERR_TIMEOUT if a status bit is set, else
 * LBRMHD_ERR_NONCONVERGED if any recovery failed, else LBRMHD_OK; errors:
 * BAD_ARG (NULL handle), CUDA. */
int lbrmhd_get_status(lbrmhd_handle h, int64_t* out3);

/* Histogram of recovery iteration counts of one run since its
 * initialisation, LBRMHD_NHIST int64 host values: out[k] (k < LBRMHD_NHIST -
 * 1) counts cell updates whose eigen-solve converged in k + 1 iterations,
 * out[LBRMHD_NHIST - 1] those that needed LBRMHD_NHIST or more (failures are
 * counted by lbrmhd_get_stats only). Synchronises the handle's stream. */
#define LBRMHD_NHIST 17
int lbrmhd_get_iteration_histogram(lbrmhd_handle h, int run, int64_t* out);

/* Checkpoint / resume: the raw device state of every run (populations and
 * primitives in their storage format, plus step counters) after a tag naming
 * the storage layout and precision. Resuming from a checkpoint is bit-exact.
 * `bytes` must be lbrmhd_state_bytes(); lbrmhd_set_state refuses (BAD_ARG) a
 * blob whose tag differs (another layout or precision). */
int lbrmhd_state_bytes(lbrmhd_handle h, size_t* bytes);
int lbrmhd_get_state(lbrmhd_handle h, void* host_buf, size_t bytes);
int lbrmhd_set_state(lbrmhd_handle h, const void* host_buf, size_t bytes);

/* Number of cells of one run (0 if out of range). */
int64_t lbrmhd_run_cells(lbrmhd_handle h, int run);

/* The lattice tables the library uses, for interpreting population arrays
 * (Eq. cellconfigs1 and the D3Q13 vectors of Sec. III), LBRMHD_NTABLE float64:
 * chat_i (19 x 3), w_i (19), w'_i (19), D3Q13 lattice hops v_k dt / dx (24 x 3),
 * e_k / c (24 x 3), b_k (24 x 3). Host only; needs no GPU. */
#define LBRMHD_NTABLE 311
int lbrmhd_lattice_tables(double* out, size_t n);

/* ------------------------------------------------------------------------
 * Launch schedule of the runs of a handle. The paper runs one problem at a
 * time; the schedule only decides how the same cell updates are grouped into
 * kernel launches, so every schedule gives bit-identical results.
 * ---------------------------------------------------------------------- */
#define LBRMHD_SCHED_PER_RUN 0 /* one launch per run per step (a grid over the run's cells) */
#define LBRMHD_SCHED_BATCH 1   /* one launch per step over the tiles of every run (per kernel variant:
                                  2-D / 3-D runs, recovery seed) */
#define LBRMHD_SCHED_PERSISTENT 2 /* one cooperative launch for all the steps of an lbrmhd_step call (or of
                                     each captured graph): every block resident, walking the tiles of every
                                     run, a grid-wide barrier between steps whose wait gives up after 1 s
                                     (status bit 2, LBRMHD_ERR_TIMEOUT from lbrmhd_get_status); for runs
                                     that are all periodic, unforced and of one kernel variant (BAD_ARG
                                     from lbrmhd_step otherwise). bx and order as for BATCH. */

typedef struct lbrmhd_schedule {
    int32_t kind;        /* LBRMHD_SCHED_PER_RUN | LBRMHD_SCHED_BATCH | LBRMHD_SCHED_PERSISTENT */
    int32_t bx;          /* BATCH: tile width 32 | 64 | 128 (a tile is bx x 128 / bx cells) */
    int32_t waves;       /* BATCH: 0 = one block per tile; w > 0 = persistent grid of w waves of
                            resident blocks, each block walking the tile list */
    int32_t order;       /* BATCH: 0 = tiles run after run, 1 = tiles interleaved across runs */
    int32_t streams;     /* PER_RUN: the runs are spread round-robin over this many streams of the
                            handle (1..32; 1 = the handle's stream), so that kernels of different
                            runs overlap; each run's steps stay in order on its stream */
    int32_t graph_steps; /* > 0: lbrmhd_step replays a CUDA graph of this many steps (captured on
                            first use on a stream of the handle, ordered after and before the
                            handle's stream); 0: direct launches */
} lbrmhd_schedule;

/* Sets the schedule. Default (never set): PER_RUN, 1 stream, no graph.
 * The per-run launch covers grids with ny <= 65535 and nz <= 65535 (CUDA's
 * limit on a launch grid's y and z extents); a PER_RUN schedule of a handle
 * holding a taller run steps every run through the tile list instead (BATCH,
 * bx 128, waves 1, order 0, the graph_steps set), and lbrmhd_get_schedule
 * returns the schedule in effect. Errors: BAD_ARG. */
int lbrmhd_set_schedule(lbrmhd_handle h, const lbrmhd_schedule* sched);
int lbrmhd_get_schedule(lbrmhd_handle h, lbrmhd_schedule* sched);

/* Autotuner: times PER_RUN on 1, 4 and up to 16 streams (when the per-run
 * launch covers every run), every BATCH
 * combination of bx {128, 64, 32}, waves {0, 1}, order {0, 1}, and (where the
 * runs admit it) PERSISTENT with bx {128, 64, 32}, order {0, 1}, one step per
 * launch, on the handle's current state with `trials` dry
 * steps each (steps whose output buffers are discarded: the state, the step
 * counters and the recovery counters are left as they were; attached sample
 * buffers are written), sets the fastest (keeping graph_steps) and returns
 * it and its time per step in ms. When the environment variable
 * LBRMHD_TUNE_CACHE names a file, a schedule stored there for the same batch
 * (precision, grids, kernel variants) is taken without timing, and a newly
 * tuned one is appended. Synchronises the handle's stream. Errors: BAD_ARG
 * (trials outside 1..100), STATE (a run not initialised, a learned-seed run
 * without weights), CUDA. */
int lbrmhd_autotune(lbrmhd_handle h, int trials, lbrmhd_schedule* best, double* best_ms);

/* Self-test of the bounded wait of the persistent schedule's grid barrier:
 * a cooperative grid of a few blocks meets at the same barrier code; with
 * `unreachable` != 0 it waits for one arrival more than the grid has, which
 * never comes, and every block must give up after wait_seconds (0 < w <= 10)
 * and raise the status bit. Runs on a scratch counter and status word of the
 * handle (the handle's own status is left alone). Returns LBRMHD_ERR_TIMEOUT
 * if the wait ran out, LBRMHD_OK if the barrier completed; errors: BAD_ARG,
 * CUDA. Synchronises the handle's stream. */
int lbrmhd_barrier_selftest(lbrmhd_handle h, int unreachable, double wait_seconds);

/* ------------------------------------------------------------------------
 * Learned recovery seed. The paper has no counterpart: it fixes the
 * eigenproblem (Sec. III, coupling), not where its iteration starts. A
 * 20-64-64-64-4 ReLU network maps normalised moments of a cell to a guess of
 * beta = u / c (and eps / T^00 - 1); the step kernel evaluates it on the
 * tensor cores (bf16 operands, float32 accumulation) and uses the guess,
 * clamped to |beta| <= 0.9, as the starting vector of the same eigen-solve.
 *
 * Parameters: LBRMHD_MLP_NPARAM float32 values, W1[64][20] b1[64]
 * W2[64][64] b2[64] W3[64][64] b3[64] W4[4][64] b4[4] (W[out][in]).
 * Features (20 float32 per cell): T^{0a}/T^00 (3), T^{xx,yy,zz,xy,xz,yz}/T^00
 * (6), N^a/N^0 (3), N^0/T^00, E/sqrt(T^00) (3), B/sqrt(T^00) (3), 1, with T,
 * N the streamed moments (Eqs. Cal_T, Cal_N) and E, B the previous step's.
 * A training sample is one row of 24 float32: the 20 features, then the
 * converged beta (3) and eps / T^00 - 1.
 * ---------------------------------------------------------------------- */
#define LBRMHD_MLP_NPARAM 9924
#define LBRMHD_MLP_NFEAT 20
#define LBRMHD_MLP_ROW 24

/* LBRMHD_MLP_NPARAM and the size in bytes of the packed inference blob. */
int lbrmhd_mlp_nparams(void);
int lbrmhd_mlp_blob_bytes(void);

/* Packs float32 parameters (device) into a caller-allocated device blob of
 * lbrmhd_mlp_blob_bytes() bytes (bf16 weights, zero-padded rows, float32
 * biases). Asynchronous on `stream`. Errors: BAD_ARG (NULL pointer), CUDA. */
int lbrmhd_mlp_pack(const float* d_params, void* d_blob, void* stream);

/* Network outputs (n x 4 float32, device) for n feature rows (n x 20 float32,
 * device) with a packed blob; the same tensor-core code as the step kernel.
 * Asynchronous. Errors: BAD_ARG (NULL pointer, n < 0), CUDA. */
int lbrmhd_mlp_infer(const void* d_blob, const float* d_features, int64_t n, float* d_out, void* stream);

/* Loss and gradient over n samples (n x 24 float32, device) in float32:
 * loss = (1/n) sum_s sum_o (y_o(x_s) - t_so)^2. d_grad (device) receives
 * LBRMHD_MLP_NPARAM gradient values then the loss. Allocates a scratch array
 * and synchronises `stream`. Errors: BAD_ARG, OOM, CUDA. */
int lbrmhd_mlp_grad(const float* d_params, const float* d_data, int64_t n, float* d_grad, void* stream);

/* `steps` Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on
 * mini-batches of `batch` samples drawn with replacement from the n samples
 * (row = splitmix64 hash of (seed, step, j) mod n). d_params (device,
 * updated in place), d_adam (device, 2 x LBRMHD_MLP_NPARAM: first then second
 * moments, zero for a fresh start; updated), d_loss (device, `steps` float32:
 * the mini-batch loss before each update, or NULL). Deterministic for given
 * inputs. Allocates scratch and synchronises `stream`. Errors: BAD_ARG, OOM,
 * CUDA. */
int lbrmhd_mlp_train(float* d_params, float* d_adam, const float* d_data, int64_t n, int steps, int batch, float lr,
                     uint64_t seed, float* d_loss, void* stream);

/* Gives the handle's runs with LBRMHD_RECOVERY_MLP their network: packs
 * d_params (device float32, LBRMHD_MLP_NPARAM; read on the handle's stream,
 * not retained) into the handle's own blob. lbrmhd_step returns STATE for an
 * MLP run before this call. Errors: BAD_ARG, CUDA. */
int lbrmhd_set_mlp_weights(lbrmhd_handle h, const float* d_params);

/* Attaches a caller-owned device buffer of N x LBRMHD_MLP_ROW float32 to one
 * run (NULL detaches it). Each following step writes, for every cell whose
 * recovery converged, its training sample (row = cell index); rows of cells
 * that failed are left as they were. Samples are written by the cold-seed
 * and learned-seed kernels only: a run with LBRMHD_RECOVERY_PLAIN recovers
 * from zero velocity while a buffer is attached (same tolerance, so the same
 * primitives up to it). The buffer must outlive its attachment. Errors:
 * BAD_ARG (run out of range). */
int lbrmhd_set_mlp_samples(lbrmhd_handle h, int run, float* d_samples);

/* Message of the last failure on this handle (or of the last failed create
 * when h is NULL). Owned by the library; valid until the next call. */
const char* lbrmhd_last_error(lbrmhd_handle h);

#ifdef __cplusplus
}
#endif
#endif
