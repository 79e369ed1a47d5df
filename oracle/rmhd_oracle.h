/*
 * rmhd_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, FP64 CPU restatement of one IMEX-RK step (SSP2(2,2,2) of
 * Table imex, or another of the paper's SSP tableaux) of the
 * resistive GRMHD system of arXiv:2510.18968 ("A resistive MHD module in the
 * GPU-accelerated GRMHD code GRaM-X"), Sec. II-III.  It exists so that the
 * CUDA path can be checked against something written independently from the
 * paper.  Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference legs may load it.  It shares no code, header or constant with the
 * CUDA library (paper_2510_18968_b300/csrc) and never calls it.
 *
 * Field orders follow the paper:
 *   primitives (Sec. III.B):  rho, p, v^x, v^y, v^z, E^x, E^y, E^z,
 *                             B^x, B^y, B^z, psi, phi, q
 *   conserved  (Eq. GRRMHD_flux_form): D, S_x, S_y, S_z, tau, B^x, B^y, B^z,
 *                             E^x, E^y, E^z, Phi, Psi, Q   (all densitised)
 * Grid arrays are interior-only, structure-of-arrays, x fastest:
 *   a[f*N + (k*ny + j)*nx + i],  N = nx*ny*nz.
 * Metric arrays: alpha[N], beta[3*N], gamma[6*N] (xx,xy,xz,yy,yz,zz),
 *                K[6*N] (same order).
 */
#ifndef RMHD_ORACLE_H
#define RMHD_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* The arithmetic type: double.  The tangent-linear build (rmhd_oracle.c
 * compiled as C++ with ORC_TANGENT) defines orc_real as a tangent number
 * (value and directional derivative, oracle/tangent.h) before including
 * this header; every array below then holds such pairs. */
#ifndef ORC_TANGENT
typedef double orc_real;
#endif

typedef struct {
    int    n[3];          /* interior cells per direction, n=1: inactive     */
    double dx[3];         /* spacing                                          */
    int    bc[3];         /* 0 periodic, 1 outflow (copy nearest interior)    */
    int    recon;         /* 0 minmod, 1 MC2, 2 WENO5                          */
    double gamma_eos;     /* ideal-gas Gamma                                   */
    double kappa;         /* divergence-cleaning damping                       */
    int    sigma_model;   /* 0 uniform sigma0, 1 sigma0*profile[cell],
                             2 sigma0*D^sigma_exp, 3 sigma0*max(1-D_atmo/D,0)^2 */
    double sigma0, sigma_exp, D_atmo;
    double rho_atmo, K_atmo, atmo_tol;
    double c2p_tol;
    int    c2p_maxit;
    double c2p_wmax;
    int    qflux_mode;    /* current in the charge flux: 0 the cell-centred
                             current of the implicit stage, reconstructed;
                             1 Ohm's law at the reconstructed face states;
                             2 no evolved charge: Q = d_i calE^i (Gauss's
                             law) after every recovery                      */
    int    imex;          /* IMEX-RK tableau: 0 SSP2(2,2,2) (Table imex),
                             1 SSP2(3,3,2), 2 SSP3(3,3,2), 3 SSP3(4,3,3)     */
} orc_params;

/* pointwise pieces (exported for the pin tests) */
void orc_metric_inverse(const orc_real g6[6], orc_real ginv6[6], orc_real *sqrtg);
void orc_prim2con(const orc_real prim[14], orc_real alpha, const orc_real beta[3],
                  const orc_real g6[6], orc_real gamma_eos, orc_real cons[14]);
void orc_flux(int d, const orc_real prim[14], orc_real alpha, const orc_real beta[3],
              const orc_real g6[6], orc_real sigma, orc_real gamma_eos,
              orc_real flux[14], orc_real cons[14]);
void orc_hlle(int d, const orc_real primL[14], const orc_real primR[14],
              orc_real alpha, const orc_real beta[3], const orc_real g6[6],
              orc_real sigma, orc_real gamma_eos, orc_real flux[14]);
void orc_recon_line(int method, int n, const orc_real *u, orc_real *uL, orc_real *uR);
int  orc_implicit_E(const orc_real Estar[3], const orc_real Bcons[3],
                    const orc_real v[3], orc_real alpha, const orc_real g6[6],
                    orc_real sigma, orc_real c, orc_real Eout[3]);
int  orc_con2prim(const orc_params *P, const orc_real cons_in[14], int implicit,
                  orc_real c, orc_real sigma, orc_real alpha, const orc_real g6[6],
                  const orc_real guess[14], orc_real prim[14], orc_real cons_out[14],
                  int *iters);
/* orc_con2prim on n independent points (a plain loop), arrays point-major
 * with stride 14 (cons, guess, prim, cons_out) or 6 (g6) per point */
void orc_con2prim_batch(const orc_params *P, long n, const orc_real *cons, int implicit,
                        orc_real c, const orc_real *sigma, const orc_real *alpha,
                        const orc_real *g6, const orc_real *guess, orc_real *prim,
                        orc_real *cons_out, int *iters, int *status);

/* whole-grid operations */
void orc_rhs(const orc_params *P, const orc_real *alpha, const orc_real *beta,
             const orc_real *gam, const orc_real *K, const orc_real *sigma_field,
             const orc_real *prim, const orc_real *Jcell, orc_real *rhs);
void orc_prim2con_grid(const orc_params *P, const orc_real *alpha,
                       const orc_real *beta, const orc_real *gam,
                       const orc_real *prim, orc_real *cons);
/* tableau of an IMEX scheme (row-major 4x4, zero-padded); returns the
 * number of stages, 0 for an unknown scheme */
int  orc_imex_tableau(int scheme, orc_real At[16], orc_real wt[4], orc_real A[16],
                      orc_real w[4]);
/* the general IMEX-RK form with P->imex's tableau (any scheme, 0 included;
 * orc_step runs scheme 0 through its literal equations instead).  Returns
 * -6 for an unknown scheme. */
int  orc_step_tableau(const orc_params *P, const orc_real *alpha, const orc_real *beta,
                      const orc_real *gam, const orc_real *K, const orc_real *sigma_field,
                      orc_real *cons, orc_real *prim, orc_real dt, int nsteps,
                      long long stats[8]);
int  orc_step(const orc_params *P, const orc_real *alpha, const orc_real *beta,
              const orc_real *gam, const orc_real *K, const orc_real *sigma_field,
              orc_real *cons, orc_real *prim, orc_real dt, int nsteps,
              long long stats[8]);

/* diagnostics: per-cell recovery status of the last step (3*N ints) */
void orc_set_status_buffer(int *buf);
/* diagnostics: inputs of failed recoveries (ORC_FAIL_REC doubles each:
 * stage, cell, conserved [14], guess [14], alpha, gamma_ij [6], c, sigma) */
#define ORC_FAIL_REC 39
void orc_set_fail_buffer(double *buf, long cap, long *count);
#ifdef ORC_TANGENT
/* tangent-linear build: derivative seed of log sigma0 for the next steps */
void orc_set_tangent_log_sigma0(double d);
#endif

#ifdef __cplusplus
}
#endif
#endif
