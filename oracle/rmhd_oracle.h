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
void orc_metric_inverse(const double g6[6], double ginv6[6], double *sqrtg);
void orc_prim2con(const double prim[14], double alpha, const double beta[3],
                  const double g6[6], double gamma_eos, double cons[14]);
void orc_flux(int d, const double prim[14], double alpha, const double beta[3],
              const double g6[6], double sigma, double gamma_eos,
              double flux[14], double cons[14]);
void orc_hlle(int d, const double primL[14], const double primR[14],
              double alpha, const double beta[3], const double g6[6],
              double sigma, double gamma_eos, double flux[14]);
void orc_recon_line(int method, int n, const double *u, double *uL, double *uR);
int  orc_implicit_E(const double Estar[3], const double Bcons[3],
                    const double v[3], double alpha, const double g6[6],
                    double sigma, double c, double Eout[3]);
int  orc_con2prim(const orc_params *P, const double cons_in[14], int implicit,
                  double c, double sigma, double alpha, const double g6[6],
                  const double guess[14], double prim[14], double cons_out[14],
                  int *iters);
/* orc_con2prim on n independent points (a plain loop), arrays point-major
 * with stride 14 (cons, guess, prim, cons_out) or 6 (g6) per point */
void orc_con2prim_batch(const orc_params *P, long n, const double *cons, int implicit,
                        double c, const double *sigma, const double *alpha,
                        const double *g6, const double *guess, double *prim,
                        double *cons_out, int *iters, int *status);

/* whole-grid operations */
void orc_rhs(const orc_params *P, const double *alpha, const double *beta,
             const double *gam, const double *K, const double *sigma_field,
             const double *prim, const double *Jcell, double *rhs);
void orc_prim2con_grid(const orc_params *P, const double *alpha,
                       const double *beta, const double *gam,
                       const double *prim, double *cons);
/* tableau of an IMEX scheme (row-major 4x4, zero-padded); returns the
 * number of stages, 0 for an unknown scheme */
int  orc_imex_tableau(int scheme, double At[16], double wt[4], double A[16],
                      double w[4]);
/* the general IMEX-RK form with P->imex's tableau (any scheme, 0 included;
 * orc_step runs scheme 0 through its literal equations instead).  Returns
 * -6 for an unknown scheme. */
int  orc_step_tableau(const orc_params *P, const double *alpha, const double *beta,
                      const double *gam, const double *K, const double *sigma_field,
                      double *cons, double *prim, double dt, int nsteps,
                      long long stats[8]);
int  orc_step(const orc_params *P, const double *alpha, const double *beta,
              const double *gam, const double *K, const double *sigma_field,
              double *cons, double *prim, double dt, int nsteps,
              long long stats[8]);

/* diagnostics: per-cell recovery status of the last step (3*N ints) */
void orc_set_status_buffer(int *buf);
/* diagnostics: inputs of failed recoveries (ORC_FAIL_REC doubles each:
 * stage, cell, conserved [14], guess [14], alpha, gamma_ij [6], c, sigma) */
#define ORC_FAIL_REC 39
void orc_set_fail_buffer(double *buf, long cap, long *count);

#ifdef __cplusplus
}
#endif
#endif
