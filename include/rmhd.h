/*
 * rmhd.h -- C ABI of the B300 (sm_103a) library for one IMEX-SSP2(2,2,2) step
 * of the resistive general-relativistic MHD system of arXiv:2510.18968
 * ("A resistive MHD module in the GPU-accelerated GRMHD code GRaM-X").
 *
 * The evolved system is Eq. GRRMHD_flux_form (Sec. II.D) on a static 3+1
 * metric (Sec. II.A):
 *   conserved U = (D, S_x, S_y, S_z, tau, B^x, B^y, B^z, E^x, E^y, E^z,
 *                  Phi, Psi, Q)                      -- all densitised by
 *                  sqrt(gamma) as in Sec. II.D (calB = sqrt(g) B, ...)
 *   primitives   = (rho, p, v^x, v^y, v^z, E^x, E^y, E^z, B^x, B^y, B^z,
 *                  psi, phi, q)                      -- Sec. III.B order, eps
 *                  follows from the ideal-gas law p = (Gamma-1) rho eps
 * with Ohm's law (Eq. Ohm_law), HLLE fluxes with light-speed bounds (Sec. III),
 * minmod / MC2 / WENO5 reconstruction, the IMEX stages of Table imex and
 * Eq. IMEX3 (Sec. III.A), and the implicit electric field solved jointly with
 * the 1D primitive recovery (Sec. III.B, steps i-v).
 *
 * Conventions for every array argument:
 *   - float64, interior cells only, structure of arrays, x fastest:
 *     a[f*N + (k*ny + j)*nx + i], N = nx*ny*nz (the library adds ghosts);
 *   - vectors are contravariant and undensitised in primitives; conserved
 *     arrays are densitised;
 *   - on_device = 0: host pointers (pageable or pinned), copied on the
 *     handle's stream and synchronised before return; on_device = 1: device
 *     pointers on the current device, copied stream-ordered.
 *   - Caller pointers are never retained.  The handle owns all device memory.
 * Thread safety: a handle is used by one host thread at a time.
 * Every function returns 0 (RMHD_OK) or a negative error code; details in
 * rmhd_last_error().
 */
#ifndef RMHD_H
#define RMHD_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
    RMHD_OK = 0,
    RMHD_EINVAL = -1,   /* bad argument; state unchanged                      */
    RMHD_ECUDA = -2,    /* a CUDA call failed (message in rmhd_last_error)    */
    RMHD_ENOMEM = -3,   /* device allocation failed                           */
    RMHD_EC2P = -4,     /* soft: some recoveries failed and were reset to the
                           atmosphere; the state is usable                    */
    RMHD_ENAN = -5      /* a non-finite conserved value appeared              */
};

enum { RMHD_BC_PERIODIC = 0, RMHD_BC_OUTFLOW = 1 /* copy nearest (Sec. IV.A) */ };
enum { RMHD_RECON_MINMOD = 0, RMHD_RECON_MC2 = 1, RMHD_RECON_WENO5 = 2 };
enum { RMHD_PREC_FP64 = 0, RMHD_PREC_MIXED = 1 };
enum {
    RMHD_SIGMA_UNIFORM = 0,  /* sigma = sigma0                                 */
    RMHD_SIGMA_FIELD = 1,    /* sigma = sigma0 * profile[cell] (rmhd_set_sigma) */
    RMHD_SIGMA_POWD = 2,     /* sigma = sigma0 * D^sigma_exp, Eq. sigma_evol    */
    RMHD_SIGMA_ATMO = 3      /* sigma0 max(1 - D_atmo/D, 0)^2, Eq. dynamo_sigma */
};
enum {
    RMHD_QFLUX_STAGE = 0,    /* charge-flux current = cell-centred current of the
                                implicit stage, reconstructed to the faces     */
    RMHD_QFLUX_FACE_OHM = 1, /* Ohm's law at the reconstructed face states      */
    RMHD_QFLUX_GAUSS = 2     /* charge not evolved: after every recovery
                                calQ = d_i calE^i by 2nd-order central
                                differences (Gauss's law, the variant of
                                Sec. IV.E); q = calQ / sqrt(gamma)            */
};

enum {
    /* IMEX-RK schemes (Sec. III.A, general form with a double Butcher
       tableau; the paper lists all four in Sec. I and prints only the
       first, Table imex; the others carry the coefficients published by
       Pareschi & Russo, J. Sci. Comput. 25 (2005)) */
    RMHD_IMEX_SSP222 = 0,    /* 2 stages, Eq. IMEX3 (default)                */
    RMHD_IMEX_SSP2332 = 1,   /* SSP2(3,3,2): 3 stages, 2nd order             */
    RMHD_IMEX_SSP3332 = 2,   /* SSP3(3,3,2): 3 stages, 2nd order, explicit
                                part 3rd order                               */
    RMHD_IMEX_SSP3433 = 3    /* SSP3(4,3,3): 4 stages, 3rd order; its first
                                stage's F has weight 0 and is not formed     */
};

typedef struct rmhd_params {
    int    n[3];        /* interior cells per direction (>= 1); n = 1 makes the
                           direction inactive (no flux, no ghosts)             */
    double x0[3];       /* lower corner of cell (0,0,0) (informational)       */
    double dx[3];       /* cell size per direction (> 0)                      */
    int    bc[3];       /* RMHD_BC_* per direction, both faces                 */
    int    recon;       /* RMHD_RECON_*                                        */
    int    precision;   /* RMHD_PREC_*                                         */
    double gamma_eos;   /* ideal-gas Gamma (> 1), Sec. III.B                   */
    double kappa;       /* divergence-cleaning damping, 1 in Sec. IV           */
    int    sigma_model; /* RMHD_SIGMA_*                                        */
    double sigma0, sigma_exp, D_atmo;
    double rho_atmo;    /* atmosphere density (Sec. IV.E.1)                    */
    double K_atmo;      /* atmosphere pressure p = K_atmo rho_atmo^Gamma       */
    double atmo_tol;    /* recovered rho < rho_atmo (1 + atmo_tol) -> reset    */
    double c2p_tol;     /* recovery stopping tolerance (1e-14)                 */
    int    c2p_maxit;   /* cap of the paper's recovery iterations (100)        */
    double c2p_wmax;    /* Lorentz-factor cap inside the recovery (100)        */
    int    qflux_mode;  /* RMHD_QFLUX_*                                        */
    int    c2p_first_pass; /* paper iterations a cell may take in the stepping
                           kernels' first recovery pass before it is listed
                           for the second pass (resumed where it stopped);
                           0 = the whole iteration (default)                 */
    int    imex;        /* RMHD_IMEX_* (the adjoint needs RMHD_IMEX_SSP222)    */
} rmhd_params;

typedef struct rmhd_s *rmhd_t;

/* Fill p with the library defaults (flat 1x1x1 grid, minmod, FP64,
 * Gamma 2, kappa 1, sigma 0, atmosphere 1e-10 / K 100 / tol 1e-2,
 * recovery 1e-14 / 100 / W<=100, stage charge current). */
void rmhd_default_params(rmhd_params *p);

/* Create a solver for the grid and options in *p on the given CUDA stream
 * (cudaStream_t, may be NULL for the legacy default stream).  Allocates all
 * device memory: about (70 + 3*14 + 17) fields x padded cells x 8 bytes,
 * plus 14 (s - 1) + 3 s fields for an s-stage scheme other than
 * RMHD_IMEX_SSP222.
 * The metric starts flat, sigma uniform.  Errors: RMHD_EINVAL (n < 1,
 * dx <= 0, Gamma <= 1, sigma0 < 0, unknown enum), RMHD_ENOMEM, RMHD_ECUDA. */
int rmhd_create(const rmhd_params *p, void *cuda_stream, rmhd_t *out);

/* Static 3+1 metric (Sec. II.A, Eq. 3plus1_metric): alpha[N], beta[3][N]
 * (contravariant shift), gamma[6][N] (gamma_xx, xy, xz, yy, yz, zz), K[6][N]
 * (extrinsic curvature, same order).  alpha == NULL resets to flat space.
 * Errors: RMHD_EINVAL if alpha <= 0 or gamma_ij is not positive definite
 * anywhere (state unchanged). */
int rmhd_set_metric(rmhd_t h, const double *alpha, const double *beta,
                    const double *gamma, const double *K, int on_device);

/* Conductivity profile for RMHD_SIGMA_FIELD: sigma = sigma0 * profile[N]
 * (Sec. II.D, Eq. Ohm_law); NULL resets to 1.  Errors: RMHD_EINVAL if any
 * value is negative or not finite. */
int rmhd_set_sigma(rmhd_t h, const double *profile, int on_device);

/* Initial primitives prims[14][N].  Forms U^n with the prim->con map
 * (Eqs. conserved_dens/tau/S, densitised EM variables) and fills ghosts.
 * Errors: RMHD_EINVAL if rho <= 0, p < 0, v^2 >= 1 or a value is not finite
 * (state unchanged). */
int rmhd_set_prims(rmhd_t h, const double *prims, int on_device);

/* Advance nsteps IMEX-RK steps of size dt.  With RMHD_IMEX_SSP222
 * (Eq. IMEX3):
 *   stage 1  U1 = U^n + gamma dt R[U1]   (implicit E + recovery, pointwise)
 *   stage 2  U2 = U^n + dt F[U1] + dt((1-2gamma) R[U1] + gamma R[U2])
 *   final    U^{n+1} = U^n + dt/2 (F[U1] + F[U2]) + dt/2 (R[U1] + R[U2]),
 *            then recovery with E fixed,
 * gamma = 1 - 1/sqrt(2) (Table imex); R acts on E only (Sec. III.A).  The
 * other schemes follow the general form of Sec. III.A,
 *   U^(i) = U^n + dt sum_{j<i} At_ij F[U^(j)] + dt sum_{j<=i} A_ij R[U^(j)],
 *   U^{n+1} = U^n + dt sum_i wt_i F[U^(i)] + dt sum_i w_i R[U^(i)],
 * each stage's implicit part solved with the recovery (guess: the previous
 * stage's primitives), then U^{n+1} recovered with E fixed.
 * Enqueued on the handle's stream; with nsteps >= 2 one step is captured
 * as a CUDA graph (once, and again when dt or another step constant
 * changes) and replayed nsteps times.  If fail_count is NULL the call returns
 * without synchronising (errors of this call then surface at the next
 * synchronising call); otherwise it synchronises, stores the number of
 * recoveries reset to the atmosphere during these steps, and returns
 * RMHD_EC2P if that number is positive or RMHD_ENAN on non-finite values. */
int rmhd_step(rmhd_t h, double dt, int nsteps, long long *fail_count);

/* Same as rmhd_step (without the failure count) but records CUDA events on
 * the handle's stream between the kernel groups of each step and adds their
 * durations, in milliseconds, to ms[RMHD_NPROF]: [0] stage-1 recovery,
 * [1] ghost fills, [2] face fluxes of stage 2 (x, y, z), [3] stage-2
 * flux difference + sources + implicit recovery, [4] face fluxes of the final
 * assembly, [5] final assembly + recovery.  With more stages, [2] and [3]
 * sum over stages 2..s (their row combinations counted in [3]) and [5]
 * includes the combination of the weights.  Synchronises after every step.
 * Instrumentation for benchmarks; not a paper operation. */
#define RMHD_NPROF 6
int rmhd_step_profiled(rmhd_t h, double dt, int nsteps, double ms[RMHD_NPROF]);

/* Copy out the current primitives prims[14][N] / conserved cons[14][N]
 * (synchronises for host destinations). */
int rmhd_get_prims(rmhd_t h, double *prims, int on_device);
int rmhd_get_cons(rmhd_t h, double *cons, int on_device);

/* Checkpoint restore from the conserved variables alone (Sec. II.D: the
 * evolved vector U = (D, S_i, tau, calB^i, calE^i, Phi, Psi, calQ), densitised,
 * field order of rmhd_get_cons).  The primitives are recovered from them with
 * the recovery of Sec. III.B at fixed calE (as after the last stage of a
 * step); the guess (p, v^i) is the handle's current primitives when it has a
 * state, otherwise v = 0 and p = (Gamma-1) max(tau/sqrt(gamma) - (E^2+B^2)/2, 0)
 * (the energy density at rest; the atmosphere pressure when that is zero).
 * A cell whose recovery fails is reset to the atmosphere as in a step (its
 * D, S_i, tau replaced) and counted (rmhd_get_stats).  Synchronises.
 * Errors: RMHD_EINVAL if a value is not finite or D <= 0 (state unchanged);
 * RMHD_EC2P (soft) if some cells were reset. */
int rmhd_set_cons(rmhd_t h, const double *cons, int on_device);

/* Checkpoint restore: set conserved cons[14][N] together with the primitives
 * that were current with them (the recovery guess), bit-exact round trip with
 * rmhd_get_cons / rmhd_get_prims.  Errors: RMHD_EINVAL on non-finite values. */
int rmhd_set_state(rmhd_t h, const double *cons, const double *prims,
                   int on_device);

/* ------------------------------------------------ z-slab decomposition
 * A grid split into z-slabs, one handle per slab (Sec. III: boxes per
 * process with ghost-zone synchronisation; the paper has no prescription
 * for how).  Each handle covers its slab extended on every internal face by
 * a halo of H layers, the reach of one step (stencil radius 3 per face-flux
 * evaluation: H = 6 for RMHD_IMEX_SSP222, 9 for the three-flux schemes; +1
 * per recovery with RMHD_QFLUX_GAUSS).  After every step the owned layers
 * next to a face are copied into the neighbour's halo; a step then computes
 * the owned cells exactly as one handle over the whole grid would, bit for
 * bit, while the halo layers absorb the error of the handle's own boundary
 * condition at the cut.  These two calls copy the state a step starts from
 * (U, the primitives and, on the mixed path, the FP64 recovery guess) of
 * interior z-layers [k0, k0 + nk) to or from a packed buffer, bit for bit:
 * U's 14 fields, then the 14 primitives in the path's storage type, then
 * (mixed) the 4 guess fields, each over the nk layers, x fastest.
 * rmhd_state_layer_bytes gives the bytes per layer (-1 for a NULL handle).
 * on_device as for rmhd_set_prims; host buffers go through the handle's
 * staging buffer (RMHD_EINVAL if nk layers do not fit it: pass device
 * memory).  Errors: RMHD_EINVAL for layers outside [0, nz) or no state. */
long long rmhd_state_layer_bytes(rmhd_t h);
int rmhd_get_state_layers(rmhd_t h, int k0, int nk, void *buf, int on_device);
int rmhd_set_state_layers(rmhd_t h, int k0, int nk, const void *buf, int on_device);

/* Counters since creation (synchronises):
 * [0] recovery calls, [1] recovery iterations (paper iteration + fallback),
 * [2] recoveries finished by the Newton fallback, [3] recoveries reset to the
 * atmosphere after failing, [4] atmosphere floor resets, [5] largest iteration
 * count of one recovery, [6] non-finite flag, [7] steps taken. */
int rmhd_get_stats(rmhd_t h, long long stats[8]);

/* Explicit right-hand side F(U) (Sec. III.A: flux differences of
 * Eq. GRRMHD_flux_form plus sources without the stiff part of -alpha J) of
 * the stage whose primitives are prims[14][N]; J[3][N] is the cell-centred
 * charge current of that stage (NULL: zero).  Result rhs[14][N].  Uses the
 * handle's metric, conductivity and options; does not change the state. */
int rmhd_rhs(rmhd_t h, const double *prims, const double *J, double *rhs,
             int on_device);

/* Pointwise implicit-E + recovery (Sec. III.A-B) on npts independent
 * points, for testing the recovery kernel alone.  Device pointers:
 * cons[14][npts] (E slots hold calE*), guess[14][npts], alpha[npts],
 * gamma[6][npts], sigma[npts]; implicit = 1 solves calE with coefficient
 * c = a_ii dt, 0 keeps calE fixed.  Outputs prim[14][npts],
 * cons_out[14][npts] (calE solved, D/S/tau recomputed after an atmosphere
 * reset), iters[npts], status[npts] (0 paper iteration, 1 Newton fallback,
 * 4 pressure-bracket fallback, 2 failed -> atmosphere, 3 floor ->
 * atmosphere).  p supplies gamma_eos,
 * rho_atmo, K_atmo, atmo_tol and the c2p_* options.  Runs on stream.
 * Errors: RMHD_EINVAL for npts < 0, a NULL array, or gamma_eos <= 1,
 * c2p_tol <= 0, c2p_maxit < 1, c2p_wmax <= 1, rho_atmo <= 0, K_atmo < 0,
 * atmo_tol < 0. */
int rmhd_con2prim_points(const rmhd_params *p, int npts, const double *cons,
                         const double *guess, const double *alpha,
                         const double *gamma, const double *sigma, int implicit,
                         double c, double *prim, double *cons_out, int *iters,
                         int *status, void *cuda_stream);

/* Capacity of the built-in work list of rmhd_con2prim_points_noalloc. */
#define RMHD_NOALLOC_MAX_POINTS 65536

/* rmhd_con2prim_points without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that may not allocate
 * device memory when they call it -- drivers that size one memory pool at
 * start-up and treat later allocations as errors, time-critical loops that
 * cannot pay for cudaMalloc's synchronisation and latency, and host programs
 * that own all device memory.  Same arguments, results and statuses as
 * rmhd_con2prim_points, computed with the stepping kernels' two-pass scheme
 * (paper iteration, then the fallbacks for the listed points) whose work
 * list is a fixed array compiled into the library (RMHD_NOALLOC_MAX_POINTS
 * indices plus a counter, about 256 KB, held by every GPU that loads the
 * library until the process exits).  npts above RMHD_NOALLOC_MAX_POINTS is
 * rejected with RMHD_EINVAL.  The first call on a device looks up that
 * device's copy of the array (cudaGetSymbolAddress with the device current);
 * make that first call before any stream capture.  Calls share the one list
 * and it keeps the previous call's contents (the counter is cleared at the
 * start of each call): calls that overlap on the GPU race, so serialise
 * them.  Calls no cudaMalloc / cudaFree.  After a device reset the next call
 * looks the array up again in the new context.  Parameter checks are those
 * of rmhd_con2prim_points.  Errors: rmhd_last_error(NULL). */
int rmhd_con2prim_points_noalloc(const rmhd_params *p, int npts, const double *cons,
                                 const double *guess, const double *alpha,
                                 const double *gamma, const double *sigma, int implicit,
                                 double c, double *prim, double *cons_out, int *iters,
                                 int *status, void *cuda_stream);

/* ---------------------------------------------------------------- adjoint
 * Discrete adjoint of the FP64 step (the paper has none; it differentiates
 * exactly the step rmhd_step takes: Table imex / Eq. IMEX3 for the stages,
 * the recovery of Sec. III.B at its converged root by the implicit-function
 * theorem).  Limiter branches, first-order fallbacks and atmosphere resets
 * are frozen at the recorded trajectory; a cell reset to the atmosphere
 * passes no derivative through rho, p, v (nor, after the last recovery of a
 * step, through D, S_i, tau).  Needs precision RMHD_PREC_FP64, qflux_mode
 * RMHD_QFLUX_STAGE and n >= 3 in every active direction (RMHD_EINVAL
 * otherwise). */

/* Set sigma0 of the conductivity model (the value rmhd_create took). */
int rmhd_set_sigma0(rmhd_t h, double sigma0);

/* Run nsteps steps of size dt from the current state, like rmhd_step, and
 * record the trajectory for rmhd_adjoint_backward: the state (U and P,
 * 28 FP64 fields of the padded grid) every checkpoint_every steps, plus
 * scratch for one segment (checkpoint_every + 1 states and the stage states
 * of its steps, which the reverse sweep keeps instead of recomputing them)
 * and the adjoint fields: about 210 + 28 nsteps / checkpoint_every + 76
 * checkpoint_every padded FP64 fields in all (90 of them hold the per-face
 * stencil contributions of the flux adjoint).  checkpoint_every = 0 keeps
 * the whole tape instead (about 240 + 76 nsteps fields: 88 GB for 60 steps
 * of a 128^3 grid), and the reverse sweep re-runs nothing.  Replaces any earlier recording.  Errors:
 * RMHD_EINVAL, RMHD_ENOMEM, RMHD_ENAN (non-finite state; nothing recorded).
 * Atmosphere resets are not an error here (rmhd_get_stats counts them). */
int rmhd_adjoint_forward(rmhd_t h, double dt, int nsteps, int checkpoint_every);  /* >= 0 */

/* Kernel groups timed by rmhd_adjoint_backward (ms[], when not NULL). */
enum {
    RMHD_ADJ_RECOMPUTE = 0,  /* segment forward steps and the per-step recompute
                                of the stage states (forward kernels)          */
    RMHD_ADJ_FLUX = 1,       /* adjoint of the face fluxes (k_adj_flux)         */
    RMHD_ADJ_SOURCES = 2,    /* adjoint of the cell sources                     */
    RMHD_ADJ_STAGES = 3,     /* adjoint of the stage recoveries and combination */
    RMHD_NADJPROF = 4
};

/* Reverse sweep of the recorded steps.  lam_prims[14][N] (interior, field
 * order of rmhd_set_prims) = dL/dP^N for a scalar loss L of the primitives
 * after the last recorded step.  Writes grad_prims0[14][N] = dL/dP^0 (the
 * primitives the recording started from) and, when grad_log_sigma0 is not
 * NULL, dL/d(log sigma0) (every conductivity model is proportional to
 * sigma0; the D-dependence of Eqs. sigma_evol, dynamo_sigma is
 * differentiated).  Each segment is recomputed from its checkpoint.  On
 * return the state, the statistics and the recording are as
 * rmhd_adjoint_forward left them, so it may be called again with another
 * lam_prims.  The sweep is deterministic (fixed summation order).
 * on_device as for rmhd_set_prims.  ms (may be NULL): CUDA-event
 * milliseconds of the kernel groups RMHD_ADJ_* summed over the sweep (the
 * stream waits for each group's events).  Errors: RMHD_EINVAL (no
 * recording, NULL array), RMHD_ENAN (a singular recovery Jacobian). */
int rmhd_adjoint_backward(rmhd_t h, const double *lam_prims, double *grad_prims0,
                          double *grad_log_sigma0, int on_device,
                          double ms[RMHD_NADJPROF]);

/* Testing entry point (no counterpart in the paper): out[i] = 1/x[i] as the
 * recovery kernels compute it (Newton-Raphson refinement of a
 * single-precision seed), for checking against FP64 division.  Device
 * pointers, n >= 0; runs on the stream. */
int rmhd_test_rcp64(const double *x, double *out, long long n, void *cuda_stream);

/* Testing entry point (no counterpart in the paper): the three-argument
 * minmod of the FP64 MC2 limiter as the flux kernels compute it (integer
 * operations on the bit patterns), out[i] = min(a, b, c) if all three are
 * > 0, max(a, b, c) if all are < 0, else +0, for checking against that
 * definition.  Device pointers, n >= 0; runs on the stream. */
int rmhd_test_mm3(const double *a, const double *b, const double *c, double *out, long long n,
                  void *cuda_stream);

/* Testing entry point (no counterpart in the paper): the three-argument
 * minmod of the FP32 MC2 limiter as the mixed path's flux kernels compute
 * it (smallest magnitude by min instructions, signs compared on the bit
 * patterns), for checking against the definition above on floats: the same
 * value for every non-NaN input, a zero result possibly carrying a's sign.
 * Device pointers, n >= 0; runs on the stream. */
int rmhd_test_mm3f(const float *a, const float *b, const float *c, float *out, long long n,
                   void *cuda_stream);

/* Testing (no counterpart in the paper): the FP32 stencil kernels stage
 * their tiles with tensor-map bulk copies (TMA) when enable != 0 (the
 * default) and the grid allows it, with plain loads when enable == 0; the
 * staged values, and so every result, are the same.  Applies to the flux
 * launches enqueued afterwards in this process (a captured step graph keeps
 * the choice it was captured with).  Returns the previous setting. */
int rmhd_test_tile_copies(int enable);
/* Testing: flux-kernel launches so far in this process that staged their
 * tiles by tensor-map copies. */
long long rmhd_test_tile_copy_launches(void);
/* Testing: the last part of the recovery's fallback chain (Sec. III.B has
 * no fallback; the pressure bracket with the velocity solved at each trial
 * pressure, then the atmosphere) on npts independent points of a flat
 * metric, as the step's deferred passes run it: one thread per point
 * (one_warp = 0) or one warp of 32 lanes per point (one_warp = 1).  Device
 * pointers, layouts as rmhd_con2prim_points: cons[14][npts] (E slots hold
 * calE*), guess[14][npts], sigma[npts]; outputs prim[14][npts],
 * status[npts] (4 root found, 2 no root: atmosphere, 3 floor: atmosphere).
 * Runs on stream.  Errors: RMHD_EINVAL as rmhd_con2prim_points. */
int rmhd_test_bracket_points(const rmhd_params *p, int npts, const double *cons,
                             const double *guess, const double *sigma, int implicit,
                             double c, int one_warp, double *prim, int *status,
                             void *cuda_stream);

/* Text of the last error on this handle (never NULL; "" if none).  With
 * h == NULL: the last error, in the calling thread, of a call that had no
 * handle (rmhd_create, rmhd_con2prim_points, rmhd_con2prim_points_noalloc,
 * ...). */
const char *rmhd_last_error(rmhd_t h);

/* Free all device memory of the handle (synchronises its stream). */
int rmhd_destroy(rmhd_t h);

#ifdef __cplusplus
}
#endif
#endif /* RMHD_H */
