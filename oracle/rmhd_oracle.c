/*
 * rmhd_oracle.c -- TEST INFRASTRUCTURE ONLY (see rmhd_oracle.h).
 *
 * A plain FP64 CPU restatement of one IMEX-SSP2(2,2,2) step of the resistive
 * GRMHD system of arXiv:2510.18968.  Every function names the passage it
 * follows.  It is deliberately slow and literal: index loops over the
 * Levi-Civita symbol, one face flux per face, no fusion.  Built with
 * -ffp-contract=off so that no multiply-add is fused behind the reader's back.
 *
 * Readings of passages the paper leaves open (all listed with reasons in the
 * design notes of the repository):
 *  - Eq. conserved_Sij carries a sqrt(gamma) prefactor, while the S_i flux and
 *    sources multiply S_ij by sqrt(gamma) again; the stress used here is the
 *    undensitised one (prefactor dropped), so that flat space is unchanged and
 *    a static pressure-only state stays static in a curved 3-metric.
 *  - In the recovery step (iii) the cross product in the numerator of v_i is
 *    eta_ijk calE^j calB^k (no sqrt(gamma)), the value consistent with
 *    Eq. conserved_S.
 *  - Sound speed (Sec. III.B): c_s^2 = Gamma(Gamma-1) eps / (1 + Gamma eps).
 *  - Characteristic speeds: the paper's literal lambda = +-sqrt(gamma^ii)
 *    - beta^i/alpha (Sec. III).
 *  - Metric derivatives: 2nd-order central differences of the cell-centred
 *    metric, ghosts of the metric follow the grid boundary condition; face
 *    metric and face conductivity are the mean of the two adjacent cells.
 *  - Reconstruction acts on (rho, p, v^i, E^i, B^i, psi, phi, q); a face state
 *    with rho<=0, p<=0 or v^2>=1 falls back to the cell value (all 14).
 *  - Stiff term stored algebraically: Dt R(i) = (calE(i) - calE*)/gamma_imex.
 *  - Cell-centred conserved quantities inside the source terms are computed
 *    from the stage primitives.
 *  - Recovery: the tolerance, the iteration cap, what to do when the
 *    paper's iteration does not converge and the atmosphere reset are not
 *    given by the paper.  Here the paper's iteration runs to its cap; if it
 *    does not converge, the one fallback brackets the pressure root (the
 *    velocity equations solved at each trial pressure); if that fails, the
 *    cell is reset to the atmosphere.
 */
#ifdef ORC_TANGENT
#include "tangent.h"
typedef tl orc_real;
#define VAL(x) ((x).v)
#else
#define VAL(x) (x)
#endif
#include "rmhd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* the arithmetic type (double; a tangent number in the tangent-linear build) */
typedef orc_real real;

enum { P_RHO, P_P, P_VX, P_VY, P_VZ, P_EX, P_EY, P_EZ, P_BX, P_BY, P_BZ,
       P_PSI, P_PHI, P_Q };
enum { C_D, C_SX, C_SY, C_SZ, C_TAU, C_BX, C_BY, C_BZ, C_EX, C_EY, C_EZ,
       C_PHI, C_PSI, C_Q };

/* gamma of the IMEX-SSP2(2,2,2) tableau (Table imex): 1 - 1/sqrt(2) */
static real imex_gamma(void) { return 1.0 - 1.0 / sqrt(2.0); }

/* Double Butcher tableaux (Sec. III.A): explicit At (strictly lower
 * triangular) with weights wt, implicit A (lower triangular, DIRK) with
 * weights w.  Scheme 0 is Table imex.  Schemes 1-3 are the other SSP
 * schemes the paper lists (Sec. I) without printing them; their values are
 * the ones published by Pareschi and Russo (J. Sci. Comput. 25, 2005), the
 * paper's reference for the IMEX form:
 *   1  SSP2(3,3,2)  At rows (1/2), (1/2, 1/2), wt = (1/3, 1/3, 1/3);
 *                   A rows (1/4), (0, 1/4), (1/3, 1/3, 1/3), w = wt
 *   2  SSP3(3,3,2)  At rows (1), (1/4, 1/4), wt = (1/6, 1/6, 2/3);
 *                   A rows (g), (1-2g, g), (1/2-g, 0, g), w = wt,
 *                   g = 1 - 1/sqrt(2)
 *   3  SSP3(4,3,3)  At rows (0), (0, 1), (0, 1/4, 1/4),
 *                   wt = (0, 1/6, 1/6, 2/3);
 *                   A rows (a), (-a, a), (0, 1-a, a), (b, e, 1/2-b-e-a, a),
 *                   w = wt, a = 0.24169426078821, b = 0.06042356519705,
 *                   e = 0.12915286960590.
 * Returns the number of stages, 0 for an unknown scheme. */
typedef struct {
    int s;
    real At[4][4], wt[4], A[4][4], w[4];
} imex_tab;

static int imex_tableau(int scheme, imex_tab *T)
{
    memset(T, 0, sizeof(*T));
    real g = imex_gamma();
    switch (scheme) {
    case 0:
        T->s = 2;
        T->At[1][0] = 1.0;
        T->wt[0] = T->wt[1] = 0.5;
        T->A[0][0] = g;
        T->A[1][0] = 1.0 - 2.0 * g;
        T->A[1][1] = g;
        T->w[0] = T->w[1] = 0.5;
        break;
    case 1:
        T->s = 3;
        T->At[1][0] = 0.5;
        T->At[2][0] = 0.5;
        T->At[2][1] = 0.5;
        T->A[0][0] = 0.25;
        T->A[1][1] = 0.25;
        T->A[2][0] = T->A[2][1] = T->A[2][2] = 1.0 / 3.0;
        for (int i = 0; i < 3; i++) T->wt[i] = T->w[i] = 1.0 / 3.0;
        break;
    case 2:
        T->s = 3;
        T->At[1][0] = 1.0;
        T->At[2][0] = 0.25;
        T->At[2][1] = 0.25;
        T->A[0][0] = g;
        T->A[1][0] = 1.0 - 2.0 * g;
        T->A[1][1] = g;
        T->A[2][0] = 0.5 - g;
        T->A[2][2] = g;
        T->wt[0] = T->wt[1] = 1.0 / 6.0;
        T->wt[2] = 2.0 / 3.0;
        for (int i = 0; i < 3; i++) T->w[i] = T->wt[i];
        break;
    case 3: {
        const real a = 0.24169426078821, b = 0.06042356519705, e = 0.12915286960590;
        T->s = 4;
        T->At[2][1] = 1.0;
        T->At[3][1] = 0.25;
        T->At[3][2] = 0.25;
        T->A[0][0] = a;
        T->A[1][0] = -a;
        T->A[1][1] = a;
        T->A[2][1] = 1.0 - a;
        T->A[2][2] = a;
        T->A[3][0] = b;
        T->A[3][1] = e;
        T->A[3][2] = 0.5 - b - e - a;
        T->A[3][3] = a;
        T->wt[1] = T->wt[2] = 1.0 / 6.0;
        T->wt[3] = 2.0 / 3.0;
        for (int i = 0; i < 4; i++) T->w[i] = T->wt[i];
        break;
    }
    default:
        return 0;
    }
    return T->s;
}

int orc_imex_tableau(int scheme, real At[16], real wt[4], real A[16], real w[4])
{
    imex_tab T;
    int s = imex_tableau(scheme, &T);
    for (int i = 0; i < 4; i++) {
        wt[i] = T.wt[i];
        w[i] = T.w[i];
        for (int j = 0; j < 4; j++) {
            At[4 * i + j] = T.At[i][j];
            A[4 * i + j] = T.A[i][j];
        }
    }
    return s;
}

/* Levi-Civita symbol eta_{ijk} (= eta^{ijk}), indices 0..2 */
static real levi(int i, int j, int k)
{
    return (real)((i - j) * (j - k) * (k - i) / 2);
}

/* symmetric 3x3 from (xx,xy,xz,yy,yz,zz) */
static void unpack6(const real g6[6], real g[3][3])
{
    g[0][0] = g6[0]; g[0][1] = g6[1]; g[0][2] = g6[2];
    g[1][0] = g6[1]; g[1][1] = g6[3]; g[1][2] = g6[4];
    g[2][0] = g6[2]; g[2][1] = g6[4]; g[2][2] = g6[5];
}

typedef struct {
    real alpha, beta[3];
    real g[3][3], gi[3][3];
    real sg; /* sqrt(det gamma_ij) */
} metric_pt;

/* Sec. II.A: gamma^{ij} is the algebraic inverse of gamma_ij; sqrt(gamma). */
static void make_metric(real alpha, const real beta[3], const real g6[6],
                        metric_pt *m)
{
    real g[3][3];
    unpack6(g6, g);
    real c00 = g[1][1] * g[2][2] - g[1][2] * g[2][1];
    real c01 = g[1][2] * g[2][0] - g[1][0] * g[2][2];
    real c02 = g[1][0] * g[2][1] - g[1][1] * g[2][0];
    real det = g[0][0] * c00 + g[0][1] * c01 + g[0][2] * c02;
    real cof[3][3];
    cof[0][0] = c00; cof[0][1] = c01; cof[0][2] = c02;
    cof[1][0] = g[0][2] * g[2][1] - g[0][1] * g[2][2];
    cof[1][1] = g[0][0] * g[2][2] - g[0][2] * g[2][0];
    cof[1][2] = g[0][1] * g[2][0] - g[0][0] * g[2][1];
    cof[2][0] = g[0][1] * g[1][2] - g[0][2] * g[1][1];
    cof[2][1] = g[0][2] * g[1][0] - g[0][0] * g[1][2];
    cof[2][2] = g[0][0] * g[1][1] - g[0][1] * g[1][0];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            m->g[i][j] = g[i][j];
            m->gi[i][j] = cof[j][i] / det; /* adjugate / det */
        }
    m->sg = sqrt(det);
    m->alpha = alpha;
    for (int i = 0; i < 3; i++) m->beta[i] = beta ? beta[i] : 0.0;
}

void orc_metric_inverse(const real g6[6], real ginv6[6], real *sqrtg)
{
    static const real zero3[3] = {0, 0, 0};
    metric_pt m;
    make_metric(1.0, zero3, g6, &m);
    ginv6[0] = m.gi[0][0]; ginv6[1] = m.gi[0][1]; ginv6[2] = m.gi[0][2];
    ginv6[3] = m.gi[1][1]; ginv6[4] = m.gi[1][2]; ginv6[5] = m.gi[2][2];
    *sqrtg = m.sg;
}

static void lower(const metric_pt *m, const real u[3], real ul[3])
{
    for (int i = 0; i < 3; i++) {
        ul[i] = 0.0;
        for (int j = 0; j < 3; j++) ul[i] += m->g[i][j] * u[j];
    }
}

static void raise(const metric_pt *m, const real ul[3], real u[3])
{
    for (int i = 0; i < 3; i++) {
        u[i] = 0.0;
        for (int j = 0; j < 3; j++) u[i] += m->gi[i][j] * ul[j];
    }
}

static real dot3(const real a[3], const real b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* Primitive quantities derived at one point (Sec. II.A, II.C). */
typedef struct {
    real rho, p, eps, h, W, v2;
    real v[3], vl[3], E[3], El[3], B[3], Bl[3];
    real E2, B2;
} prim_pt;

static void derive_prim(const real *pr, const metric_pt *m, real Gam,
                        prim_pt *q)
{
    q->rho = pr[P_RHO];
    q->p = pr[P_P];
    for (int i = 0; i < 3; i++) {
        q->v[i] = pr[P_VX + i];
        q->E[i] = pr[P_EX + i];
        q->B[i] = pr[P_BX + i];
    }
    lower(m, q->v, q->vl);
    lower(m, q->E, q->El);
    lower(m, q->B, q->Bl);
    q->v2 = dot3(q->v, q->vl);
    q->W = 1.0 / sqrt(1.0 - q->v2);              /* W = (1 - v^2)^(-1/2) */
    q->eps = q->p / ((Gam - 1.0) * q->rho);      /* p = (Gamma-1) rho eps */
    q->h = q->rho * (1.0 + q->eps) + q->p;       /* h = rho(1+eps) + p    */
    q->E2 = dot3(q->E, q->El);
    q->B2 = dot3(q->B, q->Bl);
}

/* Eqs. conserved_dens, conserved_tau, conserved_S and the densitised
 * electromagnetic variables calE = sqrt(g) E, calB = sqrt(g) B,
 * Psi = sqrt(g) psi, Phi = sqrt(g) phi, Q = sqrt(g) q (Sec. II.D). */
static void prim_to_cons(const real *pr, const metric_pt *m, real Gam,
                         const prim_pt *q, real *c)
{
    real sg = m->sg;
    real hW2 = q->h * q->W * q->W;
    c[C_D] = sg * q->rho * q->W;
    c[C_TAU] = sg * (hW2 - q->p + 0.5 * (q->E2 + q->B2)) - c[C_D];
    for (int i = 0; i < 3; i++) {
        /* epsilon_{ijk} E^j B^k with epsilon_{ijk} = sqrt(g) eta_{ijk} */
        real cross = 0.0;
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++)
                cross += sg * levi(i, j, k) * q->E[j] * q->B[k];
        c[C_SX + i] = sg * (hW2 * q->vl[i] + cross);
        c[C_BX + i] = sg * q->B[i];
        c[C_EX + i] = sg * q->E[i];
    }
    c[C_PHI] = sg * pr[P_PHI];
    c[C_PSI] = sg * pr[P_PSI];
    c[C_Q] = sg * pr[P_Q];
    (void)Gam;
}

void orc_prim2con(const real prim[14], real alpha, const real beta[3],
                  const real g6[6], real gamma_eos, real cons[14])
{
    metric_pt m;
    prim_pt q;
    make_metric(alpha, beta, g6, &m);
    derive_prim(prim, &m, gamma_eos, &q);
    prim_to_cons(prim, &m, gamma_eos, &q, cons);
}

/* Flux vector F^d of Eq. GRRMHD_flux_form in direction d.  The current in
 * the charge flux is Ohm's law (Eq. Ohm_law) at this state, or the given
 * value *Jd when Jd is not NULL.  Returns also the conserved vector. */
static void flux_point(int d, const real *pr, const metric_pt *m,
                       real sigma, real Gam, const real *Jd, real *F,
                       real *c)
{
    prim_pt q;
    derive_prim(pr, m, Gam, &q);
    prim_to_cons(pr, m, Gam, &q, c);
    real a = m->alpha, bd = m->beta[d], sg = m->sg;
    real hW2 = q.h * q.W * q.W;

    F[C_D] = (a * q.v[d] - bd) * c[C_D];
    for (int i = 0; i < 3; i++) {
        /* undensitised mixed stress S^d_i (Eq. conserved_Sij, see header) */
        real delta = (i == d) ? 1.0 : 0.0;
        real Sdi = hW2 * q.v[d] * q.vl[i] + delta * q.p
                     - q.E[d] * q.El[i] - q.B[d] * q.Bl[i]
                     + 0.5 * delta * (q.E2 + q.B2);
        F[C_SX + i] = a * sg * Sdi - bd * c[C_SX + i];
    }
    real Sup_d = 0.0;
    for (int j = 0; j < 3; j++) Sup_d += m->gi[d][j] * c[C_SX + j];
    F[C_TAU] = a * (Sup_d - q.v[d] * c[C_D]) - bd * c[C_TAU];

    real cE[3], cB[3], cEl[3], cBl[3];
    for (int i = 0; i < 3; i++) {
        cE[i] = c[C_EX + i];
        cB[i] = c[C_BX + i];
    }
    lower(m, cE, cEl);
    lower(m, cB, cBl);
    for (int i = 0; i < 3; i++) {
        real curlE = 0.0, curlB = 0.0; /* epsilon^{i d j} X_j */
        for (int j = 0; j < 3; j++) {
            curlE += levi(i, d, j) / sg * cEl[j];
            curlB += levi(i, d, j) / sg * cBl[j];
        }
        F[C_BX + i] = a * (curlE + m->gi[i][d] * c[C_PHI]) - bd * c[C_BX + i];
        F[C_EX + i] = -(a * (curlB - m->gi[i][d] * c[C_PSI]) + bd * c[C_EX + i]);
    }
    F[C_PHI] = a * c[C_BX + d] - bd * c[C_PHI];
    F[C_PSI] = a * c[C_EX + d] - bd * c[C_PSI];

    /* Ohm's law: J^d = Q v^d + W sigma [calE^d + eps^{djk} v_j calB_k
     *                                    - (v_k calE^k) v^d]              */
    real vxB = 0.0;
    for (int j = 0; j < 3; j++)
        for (int k = 0; k < 3; k++)
            vxB += levi(d, j, k) / sg * q.vl[j] * cBl[k];
    real vE = dot3(q.vl, cE);
    real J = c[C_Q] * q.v[d] + q.W * sigma * (cE[d] + vxB - vE * q.v[d]);
    if (Jd) J = *Jd;
    F[C_Q] = a * J - bd * c[C_Q];
}

void orc_flux(int d, const real prim[14], real alpha, const real beta[3],
              const real g6[6], real sigma, real gamma_eos,
              real flux[14], real cons[14])
{
    metric_pt m;
    make_metric(alpha, beta, g6, &m);
    flux_point(d, prim, &m, sigma, gamma_eos, NULL, flux, cons);
}

/* HLLE flux with the light-speed characteristic speeds of Sec. III:
 * lambda_+- = +-sqrt(gamma^dd) - beta^d/alpha. */
static void hlle_point(int d, const real *pL, const real *pR,
                       const metric_pt *m, real sigma, real Gam,
                       const real *JL, const real *JR, real *F)
{
    real FL[14], FR[14], UL[14], UR[14];
    flux_point(d, pL, m, sigma, Gam, JL, FL, UL);
    flux_point(d, pR, m, sigma, Gam, JR, FR, UR);
    real lp = sqrt(m->gi[d][d]) - m->beta[d] / m->alpha;
    real lm = -sqrt(m->gi[d][d]) - m->beta[d] / m->alpha;
    real ap = lp > 0.0 ? lp : 0.0;
    real am = lm < 0.0 ? lm : 0.0;
    for (int f = 0; f < 14; f++)
        F[f] = (ap * FL[f] - am * FR[f] + ap * am * (UR[f] - UL[f])) / (ap - am);
}

void orc_hlle(int d, const real primL[14], const real primR[14],
              real alpha, const real beta[3], const real g6[6],
              real sigma, real gamma_eos, real flux[14])
{
    metric_pt m;
    make_metric(alpha, beta, g6, &m);
    hlle_point(d, primL, primR, &m, sigma, gamma_eos, NULL, NULL, flux);
}

/* ---------------- reconstruction (Sec. III: TVD and WENO) ---------------- */

static real minmod2(real a, real b)
{
    if (a * b <= 0.0) return 0.0;
    return fabs(a) <= fabs(b) ? a : b;
}

static real minmod3(real a, real b, real c)
{
    if (a > 0.0 && b > 0.0 && c > 0.0) return fmin(a, fmin(b, c));
    if (a < 0.0 && b < 0.0 && c < 0.0) return fmax(a, fmax(b, c));
    return 0.0;
}

/* limited slope of the middle value um|u0|up */
static real tvd_slope(int method, real um, real u0, real up)
{
    if (method == 0) return minmod2(u0 - um, up - u0);           /* minmod */
    return minmod3(2.0 * (u0 - um), 0.5 * (up - um), 2.0 * (up - u0)); /* MC2 */
}

/* Jiang-Shu WENO5 value at the face between c and d, from the stencil
 * (a,b,c,d,e) = u_{i-2..i+2}; linear weights 1/10, 6/10, 3/10, eps 1e-6,
 * power 2. */
static real weno5_face(real a, real b, real c, real d, real e)
{
    const real eps = 1e-6;
    real q0 = (2.0 * a - 7.0 * b + 11.0 * c) / 6.0;
    real q1 = (-b + 5.0 * c + 2.0 * d) / 6.0;
    real q2 = (2.0 * c + 5.0 * d - e) / 6.0;
    real t;
    real b0, b1, b2;
    t = a - 2.0 * b + c;       b0 = 13.0 / 12.0 * t * t;
    t = a - 4.0 * b + 3.0 * c; b0 += 0.25 * t * t;
    t = b - 2.0 * c + d;       b1 = 13.0 / 12.0 * t * t;
    t = b - d;                 b1 += 0.25 * t * t;
    t = c - 2.0 * d + e;       b2 = 13.0 / 12.0 * t * t;
    t = 3.0 * c - 4.0 * d + e; b2 += 0.25 * t * t;
    real w0 = 0.1 / ((eps + b0) * (eps + b0));
    real w1 = 0.6 / ((eps + b1) * (eps + b1));
    real w2 = 0.3 / ((eps + b2) * (eps + b2));
    return (w0 * q0 + w1 * q1 + w2 * q2) / (w0 + w1 + w2);
}

/* Left and right states at the face between s[2] and s[3] of the six-point
 * stencil s[0..5] = u_{i-2..i+3}. */
static void recon_face(int method, const real s[6], real *uL, real *uR)
{
    if (method == 2) {
        *uL = weno5_face(s[0], s[1], s[2], s[3], s[4]);
        *uR = weno5_face(s[5], s[4], s[3], s[2], s[1]);
    } else {
        *uL = s[2] + 0.5 * tvd_slope(method, s[1], s[2], s[3]);
        *uR = s[3] - 0.5 * tvd_slope(method, s[2], s[3], s[4]);
    }
}

void orc_recon_line(int method, int n, const real *u, real *uL, real *uR)
{
    for (int i = 0; i < n; i++) {
        uL[i] = NAN;
        uR[i] = NAN;
        if (i - 2 < 0 || i + 3 > n - 1) continue;
        real s[6];
        for (int o = 0; o < 6; o++) s[o] = u[i - 2 + o];
        recon_face(method, s, &uL[i], &uR[i]);
    }
}

/* ------------- implicit electric field (Sec. III.A, Eq. 3D_NR) ------------- */

/* Solve the 3x3 system A x = b by Gaussian elimination with partial pivoting;
 * returns 0 if singular. */
static int solve_dense(int n, real *A, real *b, real *x)
{
    for (int col = 0; col < n; col++) {
        int piv = col;
        for (int r = col + 1; r < n; r++)
            if (fabs(A[r * n + col]) > fabs(A[piv * n + col])) piv = r;
        if (A[piv * n + col] == 0.0) return 0;
        if (piv != col) {
            for (int c = 0; c < n; c++) {
                real t = A[col * n + c];
                A[col * n + c] = A[piv * n + c];
                A[piv * n + c] = t;
            }
            real t = b[col]; b[col] = b[piv]; b[piv] = t;
        }
        for (int r = col + 1; r < n; r++) {
            real f = A[r * n + col] / A[col * n + col];
            for (int c = col; c < n; c++) A[r * n + c] -= f * A[col * n + c];
            b[r] -= f * b[col];
        }
    }
    for (int r = n - 1; r >= 0; r--) {
        real s = b[r];
        for (int c = r + 1; c < n; c++) s -= A[r * n + c] * x[c];
        x[r] = s / A[r * n + r];
    }
    return 1;
}

/* Newton-Raphson on f(calE) = calE - calE_init
 *   + cc * (calE + eps^{ijk} v_j calB_k - (v_k calE^k) v^i),  cc = c alpha W sigma
 * (Eq. 3D_NR with c = a_ii Dt).  Starting from E (in/out).  Being linear in
 * calE, one step lands on the root; further steps only polish rounding. */
static int implicit_E_nr(const metric_pt *m, const real Estar[3],
                         const real cB[3], const real v[3], real W,
                         real sigma, real c, real E[3])
{
    real vl[3], cBl[3];
    lower(m, v, vl);
    lower(m, cB, cBl);
    real cc = c * m->alpha * W * sigma;
    real vxB[3];
    for (int i = 0; i < 3; i++) {
        vxB[i] = 0.0;
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++)
                vxB[i] += levi(i, j, k) / m->sg * vl[j] * cBl[k];
    }
    for (int it = 0; it < 4; it++) {
        real vE = dot3(vl, E);
        real f[3], J[9], dE[3];
        for (int i = 0; i < 3; i++) {
            f[i] = E[i] - Estar[i] + cc * (E[i] + vxB[i] - vE * v[i]);
            for (int j = 0; j < 3; j++)
                J[i * 3 + j] = (i == j ? 1.0 + cc : 0.0) - cc * v[i] * vl[j];
        }
        if (!solve_dense(3, J, f, dE)) return 0;
        real dmax = 0.0, emax = 0.0;
        for (int i = 0; i < 3; i++) {
            E[i] -= dE[i];
            if (fabs(dE[i]) > dmax) dmax = fabs(dE[i]);
            if (fabs(E[i]) > emax) emax = fabs(E[i]);
        }
        if (dmax <= 1e-15 * emax || dmax == 0.0) break;
    }
    return 1;
}

int orc_implicit_E(const real Estar[3], const real Bcons[3],
                   const real v[3], real alpha, const real g6[6],
                   real sigma, real c, real Eout[3])
{
    metric_pt m;
    make_metric(alpha, NULL, g6, &m);
    real vl[3];
    lower(&m, v, vl);
    real W = 1.0 / sqrt(1.0 - dot3(v, vl));
    for (int i = 0; i < 3; i++) Eout[i] = Estar[i];
    return implicit_E_nr(&m, Estar, Bcons, v, W, sigma, c, Eout);
}

/* ----------- recovery of primitives (Sec. III.B, steps i-v) ----------- */

typedef struct {
    const orc_params *P;
    const metric_pt *m;
    real D, Sl[3], tau, cB[3], cE0[3];
    int implicit;
    real c, sigma, v2max;
} c2p_in;

/* Step (iii): velocity, W, rho, eps from the conserved variables, the current
 * electric field and pressure p.  Returns 0 when v^2 >= v2max or the
 * denominator is not positive. */
static int recover_fluid(const c2p_in *in, const real cE[3], real p,
                         real vl[3], real v[3], real *v2, real *W,
                         real *rho, real *eps)
{
    const metric_pt *m = in->m;
    real sg = m->sg;
    real cEl[3], cBl[3];
    lower(m, cE, cEl);
    lower(m, in->cB, cBl);
    real EM = (dot3(cE, cEl) + dot3(in->cB, cBl)) / (2.0 * sg);
    real den = in->tau + in->D + sg * p - EM;
    for (int i = 0; i < 3; i++) {
        real cross = 0.0; /* eta_{ijk} calE^j calB^k */
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++)
                cross += levi(i, j, k) * cE[j] * in->cB[k];
        vl[i] = (in->Sl[i] - cross) / den;
    }
    raise(m, vl, v);
    *v2 = dot3(v, vl);
    if (!(den > 0.0) || !(*v2 < in->v2max)) return 0;
    *W = 1.0 / sqrt(1.0 - *v2);
    *rho = in->D / (sg * *W);
    *eps = (in->tau - in->D * (*W - 1.0) - sg * p * (*W * *W - 1.0) - EM)
           / (in->D * *W);
    return 1;
}

/* energy scale used in the pressure stopping test: tau + D + sqrt(g) p */
static int p_converged(const c2p_in *in, real dp, real p)
{
    real sg = in->m->sg;
    return fabs(dp) * sg <= in->P->c2p_tol * (in->tau + in->D + sg * p);
}

/* Steps (i)-(v): guess (p, v) from the previous stage; (ii) calE from the
 * implicit solve at the current v; (iii) fluid variables; (iv) Newton update
 * of p with f = p(rho,eps) - p, f' = v^2 c_s^2 - 1; (v) repeat until the
 * changes of p and v are below the tolerance, at most c2p_maxit times.
 * Returns 1 on convergence, 0 when the cap is reached or an iterate leaves
 * the physical region (v^2 >= v2max, a non-positive denominator in step
 * (iii), a non-finite value). */
static int c2p_paper(const c2p_in *in, real *p_io, real v_io[3],
                     real cE[3], real *rho_o, int *iters)
{
    real Gam = in->P->gamma_eos;
    real p = *p_io, v[3] = {v_io[0], v_io[1], v_io[2]};
    for (int it = 1; it <= in->P->c2p_maxit; it++) {
        *iters = it;
        if (in->implicit) {
            real vl[3];
            lower(in->m, v, vl);
            real v2 = dot3(v, vl);
            if (!(v2 < in->v2max)) return 0;
            real W = 1.0 / sqrt(1.0 - v2);
            if (!implicit_E_nr(in->m, in->cE0, in->cB, v, W, in->sigma, in->c, cE))
                return 0;
        }
        real vl[3], vn[3], v2, W, rho, eps;
        if (!recover_fluid(in, cE, p, vl, vn, &v2, &W, &rho, &eps)) return 0;
        real f = (Gam - 1.0) * rho * eps - p;
        real cs2 = eps > 0.0 ? Gam * (Gam - 1.0) * eps / (1.0 + Gam * eps) : 0.0;
        real fp = v2 * cs2 - 1.0;
        real pn = p - f / fp;
        if (!(pn > 0.0)) pn = 0.1 * p;
        real dv = 0.0;
        for (int i = 0; i < 3; i++)
            if (fabs(vn[i] - v[i]) > dv) dv = fabs(vn[i] - v[i]);
        real dp = pn - p;
        if (!isfinite(pn) || !isfinite(dv)) return 0;
        p = pn;
        for (int i = 0; i < 3; i++) v[i] = vn[i];
        *rho_o = rho;
        if (p_converged(in, dp, p) && dv <= in->P->c2p_tol) {
            *p_io = p;
            for (int i = 0; i < 3; i++) v_io[i] = v[i];
            return 1;
        }
    }
    return 0;
}

/* Residual of the velocity equations at fixed pressure p:
 *   g_i = [v_i (tau + D + sqrt(g) p - EM) - (S_i - eta_ijk calE^j calB^k)] / scale
 * with calE from the implicit solve at v (or fixed); x = v_lower. */
static int vel_resid(const c2p_in *in, real p, const real vl[3], real g[3],
                     real cE[3])
{
    real v[3];
    raise(in->m, vl, v);
    real v2 = dot3(v, vl);
    if (!(v2 < in->v2max)) return 0;
    real W = 1.0 / sqrt(1.0 - v2);
    for (int i = 0; i < 3; i++) cE[i] = in->cE0[i];
    if (in->implicit &&
        !implicit_E_nr(in->m, in->cE0, in->cB, v, W, in->sigma, in->c, cE))
        return 0;
    real sg = in->m->sg, cEl[3], cBl[3];
    lower(in->m, cE, cEl);
    lower(in->m, in->cB, cBl);
    real EM = (dot3(cE, cEl) + dot3(in->cB, cBl)) / (2.0 * sg);
    real scale = in->tau + in->D + sg * p;
    real den = scale - EM;
    for (int i = 0; i < 3; i++) {
        real cross = 0.0;
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++)
                cross += levi(i, j, k) * cE[j] * in->cB[k];
        g[i] = (vl[i] * den - (in->Sl[i] - cross)) / scale;
    }
    return 1;
}

static real norm3(const real g[3])
{
    return sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
}

/* Velocity at fixed p: damped Newton on vel_resid from vl (in/out); gives
 * up after eight damped steps in a row. */
static int solve_velocity(const c2p_in *in, real p, real vl[3])
{
    real g[3], cE[3];
    int damped = 0;
    if (!vel_resid(in, p, vl, g, cE)) return 0;
    for (int it = 0; it < 30; it++) {
        real J[9], rhs[3], dv[3];
        for (int col = 0; col < 3; col++) {
            real vh[3] = {vl[0], vl[1], vl[2]}, gh[3], h = 1e-7;
            vh[col] += h;
            if (!vel_resid(in, p, vh, gh, cE)) {
                h = -h;
                vh[col] = vl[col] + h;
                if (!vel_resid(in, p, vh, gh, cE)) return 0;
            }
            for (int row = 0; row < 3; row++) J[row * 3 + col] = (gh[row] - g[row]) / h;
        }
        for (int i = 0; i < 3; i++) rhs[i] = -g[i];
        if (!solve_dense(3, J, rhs, dv)) return 0;
        real lam = 1.0, vt[3], gt[3];
        int ok = 0;
        for (int ls = 0; ls < 40; ls++) {
            for (int i = 0; i < 3; i++) vt[i] = vl[i] + lam * dv[i];
            if (vel_resid(in, p, vt, gt, cE) && norm3(gt) < norm3(g)) {
                ok = 1;
                break;
            }
            lam *= 0.5;
        }
        if (!ok) return norm3(g) < 1e-13;
        /* eight damped steps in a row: creeping toward a minimum of |g|
         * that is not a solution; the pressure counts as undefined */
        damped = lam < 1.0 ? damped + 1 : 0;
        if (damped >= 8) return 0;
        real step = fmax(fabs(lam * dv[0]), fmax(fabs(lam * dv[1]), fabs(lam * dv[2])));
        for (int i = 0; i < 3; i++) { vl[i] = vt[i]; g[i] = gt[i]; }
        if (step <= 1e-15) break;
    }
    /* solved only if the equations hold (scaled residual at rounding level) */
    return norm3(g) < 1e-13;
}

/* f(p) = (Gamma-1) rho eps - p (scaled) with the velocity solved at p
 * (Newton from vl; if that does not converge, from rest) */
static int pressure_fn(const c2p_in *in, real p, real vl[3], real *f)
{
    if (!(p > 0.0)) return 0;
    if (!solve_velocity(in, p, vl)) {
        vl[0] = vl[1] = vl[2] = 0.0;
        if (!solve_velocity(in, p, vl)) return 0;
    }
    real cE[3], v[3], g[3];
    vel_resid(in, p, vl, g, cE);
    raise(in->m, vl, v);
    real v2 = dot3(v, vl), W = 1.0 / sqrt(1.0 - v2), sg = in->m->sg;
    real cEl[3], cBl[3];
    lower(in->m, cE, cEl);
    lower(in->m, in->cB, cBl);
    real EM = (dot3(cE, cEl) + dot3(in->cB, cBl)) / (2.0 * sg);
    real rho = in->D / (sg * W);
    real eps = (in->tau - in->D * (W - 1.0) - sg * p * (W * W - 1.0) - EM) / (in->D * W);
    *f = ((in->P->gamma_eos - 1.0) * rho * eps - p) * sg / (in->tau + in->D + sg * p);
    return 1;
}

/* Fallback, defined by the root itself: the pressure root of f(p), the
 * velocity equations solved at every trial pressure.  f is defined only
 * above the lowest pressure at which those equations have a solution with
 * v^2 < 1 (a lower pressure leaves too little enthalpy for the momentum),
 * so a pressure where the solve fails lies below the root.  Search: from
 * the guess, real the pressure while f is undefined or positive, halve
 * it while f is negative; a halving that lands where f is undefined is
 * replaced by geometric bisection between that pressure and the last one
 * where f was defined.  Once f changes sign, the Illinois variant of regula
 * falsi on the bracket. */
static int c2p_bracket(const c2p_in *in, real *p_io, real v_io[3], real cE[3],
                       real *rho_o, int *iters)
{
    real vl[3], v0[3], f0 = 0.0;
    lower(in->m, v_io, v0);
    for (int i = 0; i < 3; i++) vl[i] = v0[i];
    real p0 = *p_io > 0.0 ? *p_io : in->P->K_atmo * pow(in->P->rho_atmo, in->P->gamma_eos);
    int n = 0, ok = pressure_fn(in, p0, vl, &f0);
    /* f undefined at the guess: the root is above.  f is defined exactly
     * above the lowest pressure p* at which the velocity equations have a
     * solution, so the smallest defined pressure p0 2^k, k = 1 ... 60, each
     * tried from the guess velocity, is found by bisection on k */
    if (!ok) {
        int klo = 0, khi = 60;
        real vk[3] = {v0[0], v0[1], v0[2]}, fk;
        if (!pressure_fn(in, p0 * ldexp(1.0, khi), vk, &fk)) return 0;
        for (int i = 0; i < 3; i++) vl[i] = vk[i];
        f0 = fk;
        while (khi - klo > 1) {
            const int km = (klo + khi) / 2;
            for (int i = 0; i < 3; i++) vk[i] = v0[i];
            if (pressure_fn(in, p0 * ldexp(1.0, km), vk, &fk)) {
                khi = km;
                f0 = fk;
                for (int i = 0; i < 3; i++) vl[i] = vk[i];
            } else {
                klo = km;
            }
        }
        n = khi;
        p0 = p0 * ldexp(1.0, khi);
    }
    real lo = p0, hi = p0, flo = f0, fhi = f0;
    real vlo[3] = {vl[0], vl[1], vl[2]}, vhi[3] = {vl[0], vl[1], vl[2]};
    if (f0 > 0.0) {
        while (fhi > 0.0) {
            if (++n > 60) return 0;
            lo = hi; flo = fhi;
            for (int i = 0; i < 3; i++) vlo[i] = vhi[i];
            hi = 2.0 * hi;
            if (!pressure_fn(in, hi, vhi, &fhi)) return 0;
        }
    } else {
        /* hi: f < 0 and defined; und: a pressure below where f is undefined */
        real und = 0.0;
        while (flo < 0.0) {
            if (++n > 120) return 0;
            real pt = und > 0.0 ? sqrt(und * hi) : 0.5 * hi;
            real vt[3] = {vhi[0], vhi[1], vhi[2]}, ft;
            if (!pressure_fn(in, pt, vt, &ft)) {
                und = pt;
                /* f < 0 down to within 1e-9 of the lowest defined pressure:
                 * no root */
                if (und > hi * (1.0 - 1e-9)) return 0;
                continue;
            }
            if (ft < 0.0) {
                hi = pt; fhi = ft;
                for (int i = 0; i < 3; i++) vhi[i] = vt[i];
            } else {
                lo = pt; flo = ft;
                for (int i = 0; i < 3; i++) vlo[i] = vt[i];
            }
        }
    }
    int side = 0;
    real sg = in->m->sg;
    for (int it = 0; it < 100; it++) {
        *iters = n + it + 1;
        real pm = (lo * fhi - hi * flo) / (fhi - flo);
        if (!(pm > lo && pm < hi)) pm = 0.5 * (lo + hi);
        real vm[3] = {vlo[0], vlo[1], vlo[2]}, fm;
        if (!pressure_fn(in, pm, vm, &fm)) return 0;
        if (fm > 0.0) {
            lo = pm; flo = fm;
            for (int i = 0; i < 3; i++) vlo[i] = vm[i];
            if (side == 1) fhi *= 0.5;
            side = 1;
        } else {
            hi = pm; fhi = fm;
            for (int i = 0; i < 3; i++) vhi[i] = vm[i];
            if (side == -1) flo *= 0.5;
            side = -1;
        }
        if ((hi - lo) * sg <= in->P->c2p_tol * (in->tau + in->D + sg * hi) || fm == 0.0) {
            real g[3], v[3];
            *p_io = pm;
            for (int i = 0; i < 3; i++) vl[i] = vm[i];
            vel_resid(in, pm, vl, g, cE);
            raise(in->m, vl, v);
            real W = 1.0 / sqrt(1.0 - dot3(v, vl));
            for (int i = 0; i < 3; i++) v_io[i] = v[i];
            *rho_o = in->D / (sg * W);
            return 1;
        }
    }
    return 0;
}

#ifdef ORC_TANGENT
/* Tangent-linear build only.  The recovery's root x = (p, v_i) solves
 * R(x; inputs) = 0, R = (the velocity equations of vel_resid, the EOS
 * residual (Gamma-1) rho eps - p of step (iii)-(iv)).  The iterations that
 * found it carry derivatives that need not have converged when the values
 * have (the stage guess often sits at the root, so the iteration stops after
 * one or two steps while the guess's derivative is that of another state):
 * the derivative of the root is therefore taken from the implicit-function
 * theorem, dx = -R_x^-1 (dR/d inputs), at the converged values; then calE
 * and rho are re-formed at the root for their derivatives.  Values are left
 * as the recovery returned them. */
static int eos_resid(const c2p_in *in, real p, const real vl[3], real R[4], real cE[3])
{
    if (!vel_resid(in, p, vl, R, cE)) return 0;
    const metric_pt *m = in->m;
    real v[3], cEl[3], cBl[3];
    raise(m, vl, v);
    real v2 = dot3(v, vl);
    real W = 1.0 / sqrt(1.0 - v2);
    lower(m, cE, cEl);
    lower(m, in->cB, cBl);
    real EM = (dot3(cE, cEl) + dot3(in->cB, cBl)) / (2.0 * m->sg);
    real rho = in->D / (m->sg * W);
    real eps = (in->tau - in->D * (W - 1.0) - m->sg * p * (W * W - 1.0) - EM) / (in->D * W);
    R[3] = ((in->P->gamma_eos - 1.0) * rho * eps - p) / (in->tau + in->D + m->sg * p);
    return 1;
}

static real strip(real x) { return tl(x.v, 0.0); }

static void recovery_tangent(const c2p_in *in, real *p, real v[3], real cE[3], real *rho)
{
    const metric_pt *m = in->m;
    real vl[3], x[4], R[4], Eh[3];
    lower(m, v, vl);
    x[0] = strip(*p);
    for (int i = 0; i < 3; i++) x[1 + i] = strip(vl[i]);
    /* inputs without derivatives, for the Jacobian R_x */
    c2p_in in0 = *in;
    in0.D = strip(in->D);
    in0.tau = strip(in->tau);
    in0.c = strip(in->c);
    in0.sigma = strip(in->sigma);
    for (int i = 0; i < 3; i++) {
        in0.Sl[i] = strip(in->Sl[i]);
        in0.cB[i] = strip(in->cB[i]);
        in0.cE0[i] = strip(in->cE0[i]);
    }
    /* dR/d inputs along the direction: x without derivative */
    if (!eos_resid(in, x[0], &x[1], R, Eh)) return;
    real J[16], b[4], dx[4];
    for (int r = 0; r < 4; r++) b[r] = tl(-R[r].d, 0.0);
    for (int col = 0; col < 4; col++) {
        real xs[4] = {x[0], x[1], x[2], x[3]}, Rc[4];
        xs[col].d = 1.0;
        if (!eos_resid(&in0, xs[0], &xs[1], Rc, Eh)) return;
        for (int r = 0; r < 4; r++) J[r * 4 + col] = tl(Rc[r].d, 0.0);
    }
    if (!solve_dense(4, J, b, dx)) return;
    /* the root with its derivative; calE and rho re-formed there */
    real xt[4];
    for (int k = 0; k < 4; k++) xt[k] = tl(x[k].v, dx[k].v);
    real vu[3];
    raise(m, &xt[1], vu);
    real v2 = dot3(vu, &xt[1]);
    real W = 1.0 / sqrt(1.0 - v2);
    real Et[3] = {in->cE0[0], in->cE0[1], in->cE0[2]};
    if (in->implicit && !implicit_E_nr(m, in->cE0, in->cB, vu, W, in->sigma, in->c, Et))
        return;
    p->d = xt[0].d;
    for (int i = 0; i < 3; i++) {
        v[i].d = vu[i].d;
        cE[i].d = Et[i].d;
    }
    rho->d = (in->D / (m->sg * W)).d;
}
#endif

/* Returns status: 0 converged (paper iteration), 4 converged (pressure
 * bracket), 2 failed -> atmosphere, 3 converged but rho < rho_atmo ->
 * atmosphere.  (Status 1 is not produced here.)  The recovery is: the
 * paper's iteration (steps i-v) to its cap; if it does not converge, the
 * pressure bracket from the same guess; if that fails too, the atmosphere. */
int orc_con2prim(const orc_params *P, const real cons_in[14], int implicit,
                 real c, real sigma, real alpha, const real g6[6],
                 const real guess[14], real prim[14], real cons_out[14],
                 int *iters)
{
    metric_pt m;
    make_metric(alpha, NULL, g6, &m);
    c2p_in in;
    in.P = P;
    in.m = &m;
    in.D = cons_in[C_D];
    in.tau = cons_in[C_TAU];
    for (int i = 0; i < 3; i++) {
        in.Sl[i] = cons_in[C_SX + i];
        in.cB[i] = cons_in[C_BX + i];
        in.cE0[i] = cons_in[C_EX + i];
    }
    in.implicit = implicit;
    in.c = c;
    in.sigma = sigma;
    in.v2max = 1.0 - 1.0 / (P->c2p_wmax * P->c2p_wmax);

    real p = guess[P_P], v[3] = {guess[P_VX], guess[P_VY], guess[P_VZ]};
    real cE[3] = {in.cE0[0], in.cE0[1], in.cE0[2]};
    real rho = 0.0;
    int it1 = 0, it2 = 0, status;
    /* atmosphere without iterating: rho = D / (W sqrt(gamma)) <= D / sqrt(gamma)
     * for every velocity, so a density D / sqrt(gamma) below the floor puts
     * every root below it (reading of the atmosphere treatment, Sec. IV.E) */
    if (!(in.D / m.sg >= P->rho_atmo * (1.0 + P->atmo_tol))) {
        status = 3;
    } else if (c2p_paper(&in, &p, v, cE, &rho, &it1)) {
        status = 0;
    } else {
        p = guess[P_P];
        for (int i = 0; i < 3; i++) {
            v[i] = guess[P_VX + i];
            cE[i] = in.cE0[i];
        }
        status = c2p_bracket(&in, &p, v, cE, &rho, &it2) ? 4 : 2;
    }
    *iters = it1 + it2;
#ifdef ORC_TANGENT
    if (status == 0 || status == 4) recovery_tangent(&in, &p, v, cE, &rho);
#endif
    /* atmosphere floor: rho below rho_atmo (1 + atmo_tol) is reset */
    int ok = status == 0 || status == 4;
    if (ok && !(rho >= P->rho_atmo * (1.0 + P->atmo_tol))) status = 3;
    int reset = status == 2 || status == 3;

    for (int f = 0; f < 14; f++) cons_out[f] = cons_in[f];
    if (reset) {
        /* atmosphere: rho_atmo, v = 0, p = K rho^Gamma; calE from the
         * implicit solve at v = 0 */
        rho = P->rho_atmo;
        p = P->K_atmo * pow(P->rho_atmo, P->gamma_eos);
        v[0] = v[1] = v[2] = 0.0;
        for (int i = 0; i < 3; i++)
            cE[i] = implicit ? in.cE0[i] / (1.0 + c * alpha * sigma) : in.cE0[i];
    }
    real sg = m.sg;
    prim[P_RHO] = rho;
    prim[P_P] = p;
    for (int i = 0; i < 3; i++) {
        prim[P_VX + i] = v[i];
        prim[P_EX + i] = cE[i] / sg;
        prim[P_BX + i] = in.cB[i] / sg;
        cons_out[C_EX + i] = cE[i];
    }
    prim[P_PSI] = cons_in[C_PSI] / sg;
    prim[P_PHI] = cons_in[C_PHI] / sg;
    prim[P_Q] = cons_in[C_Q] / sg;
    if (reset) {
        real full[14];
        orc_prim2con(prim, alpha, NULL, g6, P->gamma_eos, full);
        cons_out[C_D] = full[C_D];
        cons_out[C_TAU] = full[C_TAU];
        for (int i = 0; i < 3; i++) cons_out[C_SX + i] = full[C_SX + i];
    }
    return status;
}

void orc_con2prim_batch(const orc_params *P, long n, const real *cons, int implicit,
                        real c, const real *sigma, const real *alpha,
                        const real *g6, const real *guess, real *prim,
                        real *cons_out, int *iters, int *status)
{
    for (long i = 0; i < n; i++)
        status[i] = orc_con2prim(P, cons + 14 * i, implicit, c, sigma[i], alpha[i],
                                 g6 + 6 * i, guess + 14 * i, prim + 14 * i,
                                 cons_out + 14 * i, &iters[i]);
}

/* --------------------------- grid operations --------------------------- */

typedef struct {
    const orc_params *P;
    const real *alpha, *beta, *gam, *K, *sigma_field;
    int nx, ny, nz;
    long N;
} grid;

/* boundary-condition index map: periodic wrap or copy nearest (Sec. IV) */
static int bmap(int i, int n, int bc)
{
    if (n == 1) return 0;
    if (bc == 0) return ((i % n) + n) % n;
    return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

static long cidx(const grid *G, int i, int j, int k)
{
    i = bmap(i, G->nx, G->P->bc[0]);
    j = bmap(j, G->ny, G->P->bc[1]);
    k = bmap(k, G->nz, G->P->bc[2]);
    return ((long)k * G->ny + j) * G->nx + i;
}

static void cell_metric(const grid *G, long c, metric_pt *m)
{
    real beta[3], g6[6];
    for (int i = 0; i < 3; i++) beta[i] = G->beta[i * G->N + c];
    for (int i = 0; i < 6; i++) g6[i] = G->gam[i * G->N + c];
    make_metric(G->alpha[c], beta, g6, m);
}

/* sigma0; in the tangent-linear build it carries the derivative seeded for
 * log sigma0 (orc_set_tangent_log_sigma0), d sigma0 = sigma0 d log sigma0 */
#ifdef ORC_TANGENT
static double tl_dlog_sigma0 = 0.0;
void orc_set_tangent_log_sigma0(double d) { tl_dlog_sigma0 = d; }
static real sigma0_of(const orc_params *P) { return tl(P->sigma0, P->sigma0 * tl_dlog_sigma0); }
#else
static real sigma0_of(const orc_params *P) { return P->sigma0; }
#endif

/* Conductivity models: uniform, tabulated profile, sigma0 D^gamma_sigma
 * (Eq. sigma_evol) and sigma0 max(1 - D_atmo/D, 0)^2 (Eq. dynamo_sigma). */
static real sigma_of(const orc_params *P, const real *field, long c, real D)
{
    switch (P->sigma_model) {
    case 1: return sigma0_of(P) * field[c];
    case 2: return sigma0_of(P) * pow(D, P->sigma_exp);
    case 3: {
        real t = 1.0 - P->D_atmo / D;
        if (!(t > 0.0)) t = 0.0;
        return sigma0_of(P) * t * t;
    }
    default: return sigma0_of(P);
    }
}

static real sigma_cell_from_prim(const grid *G, const real *prim, long c)
{
    if (G->P->sigma_model < 2) return sigma_of(G->P, G->sigma_field, c, 0.0);
    real pr[14], cons[14];
    metric_pt m;
    prim_pt q;
    for (int f = 0; f < 14; f++) pr[f] = prim[f * G->N + c];
    cell_metric(G, c, &m);
    derive_prim(pr, &m, G->P->gamma_eos, &q);
    prim_to_cons(pr, &m, G->P->gamma_eos, &q, cons);
    return sigma_of(G->P, G->sigma_field, c, cons[C_D]);
}

/* Flux through the face between cell (i,j,k) and its +d neighbour.  With
 * Jcell (3 x N, the cell-centred current of the stage) the charge-flux
 * current J^d is reconstructed from it like a primitive; without it Ohm's
 * law is evaluated at the reconstructed face states. */
static void face_flux(const grid *G, const real *prim, const real *Jcell,
                      int d, int i, int j, int k, real F[14])
{
    const orc_params *P = G->P;
    int o[3] = {0, 0, 0};
    real sL[15], sR[15];
    long cL = cidx(G, i, j, k);
    long cR = cidx(G, i + (d == 0), j + (d == 1), k + (d == 2));
    for (int f = 0; f < 14; f++) {
        real s[6];
        for (int t = -2; t <= 3; t++) {
            o[d] = t;
            s[t + 2] = prim[f * G->N + cidx(G, i + o[0], j + o[1], k + o[2])];
        }
        recon_face(P->recon, s, &sL[f], &sR[f]);
    }
    if (Jcell) {
        real s[6];
        for (int t = -2; t <= 3; t++) {
            o[d] = t;
            s[t + 2] = Jcell[d * G->N + cidx(G, i + o[0], j + o[1], k + o[2])];
        }
        recon_face(P->recon, s, &sL[14], &sR[14]);
    }
    /* face metric: mean of the two cells */
    real alpha = 0.5 * (G->alpha[cL] + G->alpha[cR]);
    real beta[3], g6[6];
    for (int a = 0; a < 3; a++)
        beta[a] = 0.5 * (G->beta[a * G->N + cL] + G->beta[a * G->N + cR]);
    for (int a = 0; a < 6; a++)
        g6[a] = 0.5 * (G->gam[a * G->N + cL] + G->gam[a * G->N + cR]);
    metric_pt m;
    make_metric(alpha, beta, g6, &m);
    /* unphysical reconstructed states fall back to the cell values */
    real *side[2] = {sL, sR};
    long cell[2] = {cL, cR};
    for (int s = 0; s < 2; s++) {
        real v[3] = {side[s][P_VX], side[s][P_VY], side[s][P_VZ]}, vl[3];
        lower(&m, v, vl);
        real v2 = dot3(v, vl);
        if (!(side[s][P_RHO] > 0.0) || !(side[s][P_P] > 0.0) || !(v2 < 1.0)) {
            for (int f = 0; f < 14; f++) side[s][f] = prim[f * G->N + cell[s]];
            if (Jcell) side[s][14] = Jcell[d * G->N + cell[s]];
        }
    }
    real sigma = 0.5 * (sigma_cell_from_prim(G, prim, cL)
                          + sigma_cell_from_prim(G, prim, cR));
    if (Jcell)
        hlle_point(d, sL, sR, &m, sigma, P->gamma_eos, &sL[14], &sR[14], F);
    else
        hlle_point(d, sL, sR, &m, sigma, P->gamma_eos, NULL, NULL, F);
}

/* d(field)/dx_d at cell (i,j,k) by 2nd-order central differences */
static real dcell(const grid *G, const real *fld, int d, int i, int j, int k)
{
    int n[3] = {G->nx, G->ny, G->nz};
    if (n[d] == 1) return 0.0;
    long cp = cidx(G, i + (d == 0), j + (d == 1), k + (d == 2));
    long cm = cidx(G, i - (d == 0), j - (d == 1), k - (d == 2));
    return (fld[cp] - fld[cm]) / (2.0 * G->P->dx[d]);
}

/* Source vector S of Eq. GRRMHD_flux_form without the stiff part of -alpha J
 * (i.e. with -alpha Q v^i only, Sec. III.A split F_E / R_E). */
static void sources(const grid *G, const real *prim, int i, int j, int k,
                    real S[14])
{
    const orc_params *P = G->P;
    long c = cidx(G, i, j, k);
    metric_pt m;
    cell_metric(G, c, &m);
    real pr[14], cons[14];
    for (int f = 0; f < 14; f++) pr[f] = prim[f * G->N + c];
    prim_pt q;
    derive_prim(pr, &m, P->gamma_eos, &q);
    prim_to_cons(pr, &m, P->gamma_eos, &q, cons);

    real da[3], db[3][3], dg[3][3][3], Kij[3][3];
    real k6[6];
    for (int a = 0; a < 6; a++) k6[a] = G->K[a * G->N + c];
    unpack6(k6, Kij);
    for (int d = 0; d < 3; d++) {
        da[d] = dcell(G, G->alpha, d, i, j, k);
        for (int a = 0; a < 3; a++) db[d][a] = dcell(G, G->beta + a * G->N, d, i, j, k);
        real d6[6];
        for (int a = 0; a < 6; a++) d6[a] = dcell(G, G->gam + a * G->N, d, i, j, k);
        unpack6(d6, dg[d]); /* dg[d][a][b] = d_d gamma_ab */
    }
    /* Christoffel symbols Gamma^a_bc = 1/2 g^{al}(d_b g_lc + d_c g_lb - d_l g_bc) */
    real Chr[3][3][3];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            for (int cc = 0; cc < 3; cc++) {
                real s = 0.0;
                for (int l = 0; l < 3; l++)
                    s += m.gi[a][l] * (dg[b][l][cc] + dg[cc][l][b] - dg[l][b][cc]);
                Chr[a][b][cc] = 0.5 * s;
            }
    real Ktr = 0.0;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) Ktr += m.gi[a][b] * Kij[a][b];

    /* undensitised stress with both indices up */
    real hW2 = q.h * q.W * q.W;
    real Sup[3][3];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            Sup[a][b] = hW2 * q.v[a] * q.v[b] + m.gi[a][b] * q.p
                        - q.E[a] * q.E[b] - q.B[a] * q.B[b]
                        + 0.5 * m.gi[a][b] * (q.E2 + q.B2);
    real Sl[3] = {cons[C_SX], cons[C_SY], cons[C_SZ]}, Su[3];
    raise(&m, Sl, Su);
    real al = m.alpha, sg = m.sg;

    for (int f = 0; f < 14; f++) S[f] = 0.0;
    for (int a = 0; a < 3; a++) {
        real s = 0.0;
        for (int b = 0; b < 3; b++)
            for (int cc = 0; cc < 3; cc++) s += Sup[b][cc] * dg[a][b][cc];
        s *= 0.5 * al * sg;
        for (int b = 0; b < 3; b++) s += Sl[b] * db[a][b];
        s -= (cons[C_TAU] + cons[C_D]) * da[a];
        S[C_SX + a] = s;
    }
    {
        real s = 0.0;
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) s += Sup[a][b] * Kij[a][b];
        s *= al * sg;
        for (int a = 0; a < 3; a++) s -= Su[a] * da[a];
        S[C_TAU] = s;
    }
    for (int a = 0; a < 3; a++) {
        /* gamma^{ab} d_b alpha - alpha gamma^{bc} Gamma^a_bc */
        real G1 = 0.0;
        for (int b = 0; b < 3; b++) G1 += m.gi[a][b] * da[b];
        real G2 = 0.0;
        for (int b = 0; b < 3; b++)
            for (int cc = 0; cc < 3; cc++) G2 += m.gi[b][cc] * Chr[a][b][cc];
        real geo = G1 - al * G2;
        real sB = 0.0, sE = 0.0;
        for (int b = 0; b < 3; b++) {
            sB -= cons[C_BX + b] * db[b][a];
            sE -= cons[C_EX + b] * db[b][a];
        }
        S[C_BX + a] = sB + cons[C_PHI] * geo;
        S[C_EX + a] = sE + cons[C_PSI] * geo - al * cons[C_Q] * q.v[a];
    }
    real Bda = 0.0, Eda = 0.0;
    for (int b = 0; b < 3; b++) {
        Bda += cons[C_BX + b] * da[b];
        Eda += cons[C_EX + b] * da[b];
    }
    S[C_PHI] = -al * cons[C_PHI] * Ktr + Bda - al * P->kappa * cons[C_PHI];
    S[C_PSI] = -al * cons[C_PSI] * Ktr + Eda + al * cons[C_Q] - al * P->kappa * cons[C_PSI];
}

/* Non-stiff right-hand side F(U) = -d_k F^k + S (Sec. II.D / III.A) */
static void rhs_grid(const grid *G, const real *prim, const real *Jcell,
                     real *rhs)
{
    const orc_params *P = G->P;
    int n[3] = {G->nx, G->ny, G->nz};
    long N = G->N;
    for (long a = 0; a < 14 * N; a++) rhs[a] = 0.0;
    for (int d = 0; d < 3; d++) {
        if (n[d] == 1) continue;
        /* face fluxes: face index fi = 0..n[d] lies between cells fi-1, fi */
        int m[3] = {n[0], n[1], n[2]};
        m[d] += 1;
        long Mf = (long)m[0] * m[1] * m[2];
        real *Ff = (real *)malloc(sizeof(real) * 14 * Mf);
        for (int k = 0; k < m[2]; k++)
            for (int j = 0; j < m[1]; j++)
                for (int i = 0; i < m[0]; i++) {
                    real F[14];
                    face_flux(G, prim, Jcell, d, i - (d == 0), j - (d == 1),
                              k - (d == 2), F);
                    long fidx = ((long)k * m[1] + j) * m[0] + i;
                    for (int f = 0; f < 14; f++) Ff[f * Mf + fidx] = F[f];
                }
        for (int k = 0; k < n[2]; k++)
            for (int j = 0; j < n[1]; j++)
                for (int i = 0; i < n[0]; i++) {
                    long c = ((long)k * n[1] + j) * n[0] + i;
                    long fm = ((long)k * m[1] + j) * m[0] + i;
                    long fp = ((long)(k + (d == 2)) * m[1] + (j + (d == 1))) * m[0]
                              + (i + (d == 0));
                    for (int f = 0; f < 14; f++)
                        rhs[f * N + c] -= (Ff[f * Mf + fp] - Ff[f * Mf + fm]) / P->dx[d];
                }
        free(Ff);
    }
    for (int k = 0; k < n[2]; k++)
        for (int j = 0; j < n[1]; j++)
            for (int i = 0; i < n[0]; i++) {
                long c = ((long)k * n[1] + j) * n[0] + i;
                real S[14];
                sources(G, prim, i, j, k, S);
                for (int f = 0; f < 14; f++) rhs[f * N + c] += S[f];
            }
}

static void make_grid(grid *G, const orc_params *P, const real *alpha,
                      const real *beta, const real *gam, const real *K,
                      const real *sigma_field)
{
    G->P = P;
    G->alpha = alpha;
    G->beta = beta;
    G->gam = gam;
    G->K = K;
    G->sigma_field = sigma_field;
    G->nx = P->n[0];
    G->ny = P->n[1];
    G->nz = P->n[2];
    G->N = (long)G->nx * G->ny * G->nz;
}

void orc_rhs(const orc_params *P, const real *alpha, const real *beta,
             const real *gam, const real *K, const real *sigma_field,
             const real *prim, const real *Jcell, real *rhs)
{
    grid G;
    make_grid(&G, P, alpha, beta, gam, K, sigma_field);
    rhs_grid(&G, prim, Jcell, rhs);
}

void orc_prim2con_grid(const orc_params *P, const real *alpha,
                       const real *beta, const real *gam,
                       const real *prim, real *cons)
{
    grid G;
    make_grid(&G, P, alpha, beta, gam, NULL, NULL);
    for (long c = 0; c < G.N; c++) {
        metric_pt m;
        cell_metric(&G, c, &m);
        real pr[14], cn[14];
        for (int f = 0; f < 14; f++) pr[f] = prim[f * G.N + c];
        prim_pt q;
        derive_prim(pr, &m, P->gamma_eos, &q);
        prim_to_cons(pr, &m, P->gamma_eos, &q, cn);
        for (int f = 0; f < 14; f++) cons[f * G.N + c] = cn[f];
    }
}

/* Optional per-cell recovery status of the last step, 3 records per cell
 * (stage 1, stage 2, final), for diagnostics in the tests. */
static int *dbg_status = NULL;
void orc_set_status_buffer(int *buf) { dbg_status = buf; }

/* Optional record of the inputs of every failed recovery (status 2) of the
 * following steps, for diagnostics in the tests: per failure ORC_FAIL_REC
 * doubles (stage, cell, conserved input [14], guess [14], alpha, gamma_ij
 * [6], c, sigma), up to cap records; *count counts all failures. */
static double *dbg_fail = NULL;
static long dbg_fail_cap = 0, *dbg_fail_count = NULL;
void orc_set_fail_buffer(double *buf, long cap, long *count)
{
    dbg_fail = buf;
    dbg_fail_cap = cap;
    dbg_fail_count = count;
}

/* Pointwise recovery over the grid.  implicit: solve the stiff calE with
 * c = gamma_imex dt; cons is updated in place (calE and, after an
 * atmosphere reset, D, S_i, tau). */
static void c2p_grid(const grid *G, real *cons, const real *guess,
                     real *prim, int implicit, real c, long long stats[8],
                     int stage)
{
    const orc_params *P = G->P;
    long N = G->N;
    for (long cell = 0; cell < N; cell++) {
        real cin[14], g[14], pr[14], cout[14], g6[6];
        for (int f = 0; f < 14; f++) {
            cin[f] = cons[f * N + cell];
            g[f] = guess[f * N + cell];
        }
        for (int a = 0; a < 6; a++) g6[a] = G->gam[a * N + cell];
        real sigma = implicit ? sigma_of(P, G->sigma_field, cell, cin[C_D]) : 0.0;
        int it = 0;
        int st = orc_con2prim(P, cin, implicit, c, sigma, G->alpha[cell], g6, g,
                              pr, cout, &it);
        stats[0] += 1;
        stats[1] += it;
        if (st == 1 || st == 4) stats[2] += 1;
        if (st == 2) stats[3] += 1;
        if (st == 3) stats[4] += 1;
        if (it > stats[5]) stats[5] = it;
        if (dbg_status) dbg_status[stage * N + cell] = st;
        if (dbg_fail && st == 2) {
            long k = (*dbg_fail_count)++;
            if (k < dbg_fail_cap) {
                double *r = dbg_fail + k * ORC_FAIL_REC;
                r[0] = stage;
                r[1] = (double)cell;
                for (int f = 0; f < 14; f++) {
                    r[2 + f] = VAL(cin[f]);
                    r[16 + f] = VAL(g[f]);
                }
                r[30] = VAL(G->alpha[cell]);
                for (int a = 0; a < 6; a++) r[31 + a] = VAL(g6[a]);
                r[37] = VAL(c);
                r[38] = VAL(sigma);
            }
        }
        for (int f = 0; f < 14; f++) {
            prim[f * N + cell] = pr[f];
            cons[f * N + cell] = cout[f];
        }
    }
}

/* Cell-centred current of an implicit stage.  Ohm's law (Eq. Ohm_law) is
 * J = Q v + W sigma [...] and the stiff source is R_E = -alpha W sigma [...],
 * so at the stage's root J^i = Q v^i - (Dt R_E^i) / (alpha Dt), with Dt R_E
 * the stored stiff increment: bounded for any sigma. */
static void stage_current(const grid *G, const real *U, const real *prim,
                          const real *dR, real dt, real *J)
{
    long N = G->N;
    for (int a = 0; a < 3; a++)
        for (long c = 0; c < N; c++)
            J[a * N + c] = U[C_Q * N + c] * prim[(P_VX + a) * N + c]
                           - dR[a * N + c] / (G->alpha[c] * dt);
}

/* Charge from Gauss's law instead of its evolution equation (the variant
 * the paper tests for the magnetised star, Sec. IV.E): Q = sqrt(gamma) q =
 * d_i calE^i, by 2nd-order central differences of the densitised field with
 * the grid's boundary condition; q = Q / sqrt(gamma). */
static void gauss_charge(const grid *G, real *cons, real *prim)
{
    long N = G->N;
    for (int k = 0; k < G->nz; k++)
        for (int j = 0; j < G->ny; j++)
            for (int i = 0; i < G->nx; i++) {
                long c = cidx(G, i, j, k);
                real Q = 0.0;
                for (int d = 0; d < 3; d++)
                    Q += dcell(G, &cons[(C_EX + d) * N], d, i, j, k);
                metric_pt m;
                cell_metric(G, c, &m);
                cons[C_Q * N + c] = Q;
                prim[P_Q * N + c] = Q / m.sg;
            }
}

/* IMEX-SSP2(2,2,2) steps, literally Eqs. (U^(1), U^(2), IMEX3):
 *   U1 = U^n + gamma dt R[U1]
 *   U2 = U^n + dt F[U1] + dt ((1-2gamma) R[U1] + gamma R[U2])
 *   U^{n+1} = U^n + dt/2 (F[U1] + F[U2]) + dt/2 (R[U1] + R[U2])
 * R acts on calE only (Sec. III.A); each implicit stage is solved jointly
 * with the recovery (Sec. III.B); U^{n+1} is then recovered with calE fixed. */
static int step_ssp222(const orc_params *P, const real *alpha, const real *beta,
                       const real *gam, const real *K, const real *sigma_field,
                       real *cons, real *prim, real dt, int nsteps,
                       long long stats[8])
{
    grid G;
    make_grid(&G, P, alpha, beta, gam, K, sigma_field);
    long N = G.N;
    real g = imex_gamma();
    real *U1 = (real *)malloc(sizeof(real) * 14 * N);
    real *U2 = (real *)malloc(sizeof(real) * 14 * N);
    real *W1 = (real *)malloc(sizeof(real) * 14 * N);
    real *W2 = (real *)malloc(sizeof(real) * 14 * N);
    real *F1 = (real *)malloc(sizeof(real) * 14 * N);
    real *F2 = (real *)malloc(sizeof(real) * 14 * N);
    real *dR1 = (real *)malloc(sizeof(real) * 3 * N);
    real *dR2 = (real *)malloc(sizeof(real) * 3 * N);
    real *Jc = (real *)malloc(sizeof(real) * 3 * N);
    real *Es2 = (real *)malloc(sizeof(real) * 3 * N);
    /* mode 2 (Gauss's law) overwrites Q after every recovery, so its charge
     * flux row is irrelevant; it is formed as in mode 0 */
    const real *Jarg = P->qflux_mode != 1 ? Jc : NULL;
    const int gauss = P->qflux_mode == 2;
    int status = 0;
    for (int s = 0; s < 8; s++) stats[s] = 0;
    for (int step = 0; step < nsteps; step++) {
        /* stage 1: purely implicit */
        memcpy(U1, cons, sizeof(real) * 14 * N);
        c2p_grid(&G, U1, prim, W1, 1, g * dt, stats, 0);
        if (gauss) gauss_charge(&G, U1, W1);
        for (int a = 0; a < 3; a++)
            for (long c = 0; c < N; c++)
                dR1[a * N + c] = (U1[(C_EX + a) * N + c] - cons[(C_EX + a) * N + c]) / g;
        /* stage 2: explicit part, then implicit */
        stage_current(&G, U1, W1, dR1, dt, Jc);
        rhs_grid(&G, W1, Jarg, F1);
        for (long a = 0; a < 14 * N; a++) U2[a] = cons[a] + dt * F1[a];
        for (int a = 0; a < 3; a++)
            for (long c = 0; c < N; c++)
                U2[(C_EX + a) * N + c] += (1.0 - 2.0 * g) * dR1[a * N + c];
        for (int a = 0; a < 3; a++)   /* keep calE* of stage 2 */
            for (long c = 0; c < N; c++) Es2[a * N + c] = U2[(C_EX + a) * N + c];
        c2p_grid(&G, U2, W1, W2, 1, g * dt, stats, 1);
        if (gauss) gauss_charge(&G, U2, W2);
        for (int a = 0; a < 3; a++)
            for (long c = 0; c < N; c++)
                dR2[a * N + c] = (U2[(C_EX + a) * N + c] - Es2[a * N + c]) / g;
        /* final assembly (Eq. IMEX3) */
        stage_current(&G, U2, W2, dR2, dt, Jc);
        rhs_grid(&G, W2, Jarg, F2);
        for (long a = 0; a < 14 * N; a++) cons[a] = cons[a] + 0.5 * dt * (F1[a] + F2[a]);
        for (int a = 0; a < 3; a++)
            for (long c = 0; c < N; c++)
                cons[(C_EX + a) * N + c] += 0.5 * (dR1[a * N + c] + dR2[a * N + c]);
        for (long a = 0; a < 14 * N; a++)
            if (!isfinite(cons[a])) { status = -5; stats[6] = 1; }
        /* recovery of U^{n+1} with calE fixed */
        c2p_grid(&G, cons, W2, prim, 0, 0.0, stats, 2);
        if (gauss) gauss_charge(&G, cons, prim);
        if (status) break;
    }
    free(U1); free(U2); free(W1); free(W2); free(F1); free(F2);
    free(dR1); free(dR2); free(Jc); free(Es2);
    if (status) return status;
    return stats[3] > 0 ? -4 : 0;
}

/* IMEX-RK steps in the general form of Sec. III.A with the tableau of
 * P->imex:
 *   U^(i)   = U^n + dt sum_{j<i} At_ij F[U^(j)] + dt sum_{j<=i} A_ij R[U^(j)]/eps
 *   U^{n+1} = U^n + dt sum_i wt_i F[U^(i)] + dt sum_i w_i R[U^(i)]/eps.
 * R acts on calE only.  Stage i's implicit part is solved jointly with the
 * recovery (c = A_ii dt, guess: the previous stage's primitives, P^n for the
 * first); its stiff increment dR_i = dt R[U^(i)]/eps is kept algebraically,
 * (calE^(i) - calE*_i)/A_ii, calE*_i the stage's calE before the solve.
 * Terms with a zero coefficient are skipped, and F[U^(i)] is formed only
 * when a later row or wt uses it.  U^{n+1} is then recovered with calE
 * fixed (guess: the last stage's primitives). */
int orc_step_tableau(const orc_params *P, const real *alpha, const real *beta,
                     const real *gam, const real *K, const real *sigma_field,
                     real *cons, real *prim, real dt, int nsteps,
                     long long stats[8])
{
    imex_tab T;
    const int s = imex_tableau(P->imex, &T);
    if (!s) return -6;
    grid G;
    make_grid(&G, P, alpha, beta, gam, K, sigma_field);
    long N = G.N;
    real *Ui = (real *)malloc(sizeof(real) * 14 * N);
    real *Es = (real *)malloc(sizeof(real) * 3 * N);
    real *Jc = (real *)malloc(sizeof(real) * 3 * N);
    real *W[4], *F[4], *dR[4];
    int needF[4];
    for (int i = 0; i < s; i++) {
        W[i] = (real *)malloc(sizeof(real) * 14 * N);
        F[i] = (real *)malloc(sizeof(real) * 14 * N);
        dR[i] = (real *)malloc(sizeof(real) * 3 * N);
        needF[i] = T.wt[i] != 0.0;
        for (int k = i + 1; k < s; k++) needF[i] |= T.At[k][i] != 0.0;
    }
    const real *Jarg = P->qflux_mode != 1 ? Jc : NULL;
    const int gauss = P->qflux_mode == 2;
    int status = 0;
    for (int a = 0; a < 8; a++) stats[a] = 0;
    for (int step = 0; step < nsteps; step++) {
        for (int i = 0; i < s; i++) {
            /* explicit part of the stage */
            memcpy(Ui, cons, sizeof(real) * 14 * N);
            for (int j = 0; j < i; j++)
                if (T.At[i][j] != 0.0)
                    for (long a = 0; a < 14 * N; a++) Ui[a] += dt * T.At[i][j] * F[j][a];
            for (int j = 0; j < i; j++)
                if (T.A[i][j] != 0.0)
                    for (int a = 0; a < 3; a++)
                        for (long c = 0; c < N; c++)
                            Ui[(C_EX + a) * N + c] += T.A[i][j] * dR[j][a * N + c];
            for (int a = 0; a < 3; a++)
                for (long c = 0; c < N; c++) Es[a * N + c] = Ui[(C_EX + a) * N + c];
            /* implicit part with the recovery */
            c2p_grid(&G, Ui, i == 0 ? prim : W[i - 1], W[i], 1, T.A[i][i] * dt, stats,
                     i == 0 ? 0 : 1);
            if (gauss) gauss_charge(&G, Ui, W[i]);
            for (int a = 0; a < 3; a++)
                for (long c = 0; c < N; c++)
                    dR[i][a * N + c] = (Ui[(C_EX + a) * N + c] - Es[a * N + c]) / T.A[i][i];
            if (needF[i]) {
                stage_current(&G, Ui, W[i], dR[i], dt, Jc);
                rhs_grid(&G, W[i], Jarg, F[i]);
            }
        }
        /* U^{n+1} */
        for (int i = 0; i < s; i++)
            if (T.wt[i] != 0.0)
                for (long a = 0; a < 14 * N; a++) cons[a] += dt * T.wt[i] * F[i][a];
        for (int i = 0; i < s; i++)
            if (T.w[i] != 0.0)
                for (int a = 0; a < 3; a++)
                    for (long c = 0; c < N; c++)
                        cons[(C_EX + a) * N + c] += T.w[i] * dR[i][a * N + c];
        for (long a = 0; a < 14 * N; a++)
            if (!isfinite(cons[a])) { status = -5; stats[6] = 1; }
        c2p_grid(&G, cons, W[s - 1], prim, 0, 0.0, stats, 2);
        if (gauss) gauss_charge(&G, cons, prim);
        if (status) break;
    }
    for (int i = 0; i < s; i++) {
        free(W[i]);
        free(F[i]);
        free(dR[i]);
    }
    free(Ui); free(Es); free(Jc);
    if (status) return status;
    return stats[3] > 0 ? -4 : 0;
}

/* Steps with the scheme of P->imex: Table imex through its literal
 * equations, the other tableaux through the general form. */
int orc_step(const orc_params *P, const real *alpha, const real *beta,
             const real *gam, const real *K, const real *sigma_field,
             real *cons, real *prim, real dt, int nsteps,
             long long stats[8])
{
    if (P->imex == 0)
        return step_ssp222(P, alpha, beta, gam, K, sigma_field, cons, prim, dt, nsteps, stats);
    return orc_step_tableau(P, alpha, beta, gam, K, sigma_field, cons, prim, dt, nsteps, stats);
}
