// recovery.cuh -- implicit electric field fused with the 1D primitive recovery
// (arXiv:2510.18968, Sec. III.A Eq. 3D_NR and Sec. III.B steps i-v), FP64.
//
// Per cell the unknowns are the pressure p, the velocity v and the stiff field
// calE of the stage.  At fixed v the stage equation of calE,
//   calE - calE* + cc W (calE + eps^{ijk} v_j calB_k - (v.calE) v) = 0,
//   cc = a_ii dt alpha sigma,
// is linear, so the paper's 3D Newton-Raphson lands on its root in one step;
// here that root is written in closed form (Sherman-Morrison on the rank-one
// matrix (1+C) I - C v v_lower^T):
//   calE = [r (1 + C(1-v^2)) + C v (v_lower.r)] / [(1+C)(1 + C(1-v^2))],
//   r = calE* - C eps v x calB,  C = cc W.
// The outer loop is the paper's: (iii) v, W, rho, eps from the conserved
// variables at the current p and calE, (iv) p <- p - f/f' with
// f = (Gamma-1) rho eps - p, f' = v^2 c_s^2 - 1, c_s^2 = Gamma(Gamma-1)eps/(1+Gamma eps).
// In a strongly magnetised cell of an implicit stage that iteration diverges
// (the field's feedback on v grows by kappa = k B^2/(sqrt(g) den) > 1 per
// iteration); there a Newton method on (p, v_i) whose Jacobian keeps the
// terms of that feedback (stiff_newton) takes over from the stage guess.
// When the paper iteration gives up otherwise, or the stiff Newton fails, a
// damped Newton method on (p, v_i) with a forward-difference Jacobian takes
// over from the stage guess; if that stalls, the pressure root is bracketed
// and refined by regula falsi with the velocity equations solved at each
// pressure.  All stop on the same criteria and find the same root.  A state
// with no root is reset to the atmosphere.  Every loop is bounded.
#pragma once
#include "physics.cuh"

namespace rmhd {

struct RecOpts {
    double Gam;          // Gamma
    double tol;          // stopping tolerance
    double v2max;        // 1 - 1/W_max^2
    double rho_atmo, p_atmo, atmo_floor;  // atmo_floor = rho_atmo (1 + atmo_tol)
    int maxit;           // cap of the paper iteration
    int first_cap;       // paper iterations of the first pass (REC_FIRST)
    double kappa0;       // stiff-coupling switch to Newton after one paper
                         // iteration (0: never); see paper_run
};

struct RecIn {
    double D, S[3], tau, cB[3], cE0[3];   // cE0: calE* (implicit) or calE (fixed)
};

template <bool FLAT> struct RecCtx;
// sqrt(gamma) and its inverse, folded to 1 on a flat metric
template <bool FLAT> __device__ __forceinline__ double sgv(const RecCtx<FLAT> &c);
template <bool FLAT> __device__ __forceinline__ double isgv(const RecCtx<FLAT> &c);

template <bool FLAT> struct RecCtx {
    const RecIn &in;
    const Met<double> &m;
    const RecOpts &o;
    bool implicit;
    double cc;          // a_ii dt alpha sigma (0 when not implicit)
    double sg, isg, iD;
    double cBl[3];      // lowered calB
    double B2;          // calB . calB_lower
};

template <bool FLAT> __device__ __forceinline__ double sgv(const RecCtx<FLAT> &c)
{
    return FLAT ? 1.0 : c.sg;
}
template <bool FLAT> __device__ __forceinline__ double isgv(const RecCtx<FLAT> &c)
{
    return FLAT ? 1.0 : c.isg;
}

// closed-form implicit calE at fixed contravariant v (see file comment)
template <bool FLAT>
__device__ __forceinline__ void implicit_field(const RecCtx<FLAT> &c, const double v[3],
                                               const double vl[3], double v2, double W,
                                               double E[3])
{
    const double C = c.cc * W;
    double vxB[3];
    cross3(vl, c.cBl, vxB);            // eta v_j calB_k (lowered): sqrt(g) (v x B)
    double r[3];
#pragma unroll
    for (int i = 0; i < 3; i++) r[i] = c.in.cE0[i] - C * (FLAT ? vxB[i] : vxB[i] * c.isg);
    const double s = dot3(vl, r);
    const double q = 1.0 + C * (1.0 - v2);
    const double inv = rcp64((1.0 + C) * q);
#pragma unroll
    for (int i = 0; i < 3; i++) E[i] = (r[i] * q + C * v[i] * s) * inv;
}

template <bool FLAT>
__device__ __forceinline__ bool p_conv(const RecCtx<FLAT> &c, double dp, double p)
{
    return fabs(dp) * sgv(c) <= c.o.tol * (c.in.tau + c.in.D + sgv(c) * p);
}

// Step (iii) at (p, calE), division-lean form used by the paper iteration:
// returns v_lower, v, v^2, W, 1/W and num = tau - D(W-1) - sqrt(g) p (W^2-1) - EM
// (so that D W eps = num and rho eps = num (1-v^2)/sqrt(g)).
template <bool FLAT>
__device__ __forceinline__ bool fluid_step(const RecCtx<FLAT> &c, const double E[3], double p,
                                           double vl[3], double v[3], double &v2, double &W,
                                           double &Winv, double &num, double *den_out = nullptr)
{
    double El[3];
    lower<double, FLAT>(c.m, E, El);
    const double EM = 0.5 * (dot3(E, El) + c.B2) * isgv(c);
    double P[3];
    cross3(E, c.in.cB, P);
    const double den = c.in.tau + c.in.D + sgv(c) * p - EM;
    if (den_out) *den_out = den;
    const double iden = rcp64(den);
#pragma unroll
    for (int i = 0; i < 3; i++) vl[i] = (c.in.S[i] - P[i]) * iden;
    raise<double, FLAT>(c.m, vl, v);
    v2 = dot3(v, vl);
    if (!(den > 0.0) || !(v2 < c.o.v2max)) return false;
    const double omv = 1.0 - v2;
    W = rsqrt(omv);
    Winv = omv * W;
    num = c.in.tau - c.in.D * (W - 1.0) - sgv(c) * p * (v2 * W * W) - EM;
    return true;
}

// Iterate of the paper's iteration, complete enough to stop after any
// iteration and continue later with bit-identical arithmetic.
enum { PSTATE = 15 };
struct PaperState {
    int it;                   // iterations done
    double p, v[3], vl[3];    // current iterate
    double v2, W;             // of v
    float prev0, prev1, prev2;   // change measures of the last iterations
    int outcome;              // -1 undecided, 0 gave up (fallbacks next)
    int slow;                 // gave up for slow convergence
};

__device__ __forceinline__ void pstate_save(const PaperState &s, double *dst, long long stride)
{
    const double vals[PSTATE] = {(double)s.it, s.p,     s.v[0],  s.v[1],  s.v[2],
                                 s.vl[0],      s.vl[1], s.vl[2], s.v2,    s.W,
                                 (double)s.prev0, (double)s.prev1, (double)s.prev2, (double)s.outcome,
                                 (double)s.slow};
    for (int k = 0; k < PSTATE; k++) dst[k * stride] = vals[k];
}

__device__ __forceinline__ void pstate_load(PaperState &s, const double *src, long long stride)
{
    s.it = (int)src[0];
    s.p = src[1 * stride];
    for (int a = 0; a < 3; a++) {
        s.v[a] = src[(2 + a) * stride];
        s.vl[a] = src[(5 + a) * stride];
    }
    s.v2 = src[8 * stride];
    s.W = src[9 * stride];
    s.prev0 = (float)src[10 * stride];
    s.prev1 = (float)src[11 * stride];
    s.prev2 = (float)src[12 * stride];
    s.outcome = (int)src[13 * stride];
    s.slow = (int)src[14 * stride];
}

// Start of the paper iteration at the guess; false if the guess is outside
// the physical region.
template <bool FLAT>
__device__ __forceinline__ bool paper_start(const RecCtx<FLAT> &c, double p, const double v[3],
                                            PaperState &s)
{
    s.it = 0;
    s.p = p;
    for (int a = 0; a < 3; a++) s.v[a] = v[a];
    lower<double, FLAT>(c.m, s.v, s.vl);
    s.v2 = dot3(s.v, s.vl);
    if (!(s.v2 < c.o.v2max)) return false;
    // the first implicit solve needs W of the guess; with calE fixed the
    // first use of W is after fluid_step has set it
    s.W = c.implicit ? rsqrt(1.0 - s.v2) : 0.0;
    s.prev0 = s.prev1 = s.prev2 = 0.0f;
    s.outcome = -1;
    s.slow = 0;
    return true;
}

// The paper's iteration (steps ii-v) from state s, up to iteration `limit`.
// Returns 1 converged, 0 gave up, -1 reached `limit` (< maxit) undecided.
// The Lorentz factor and lowered velocity of an iterate are carried to the
// next implicit solve; f and f/f' are formed without dividing by D:
//   f = (Gamma-1) num (1-v^2)/sqrt(g) - p,
//   f/f' = f (D + Gamma num/W) / (v^2 Gamma(Gamma-1) num/W - D - Gamma num/W).
// p_guess fixes the energy scale of the change measure.
template <bool FLAT>
__device__ int paper_run(const RecCtx<FLAT> &c, PaperState &s, double p_guess, int limit,
                         double E[3], double &rho_out, bool allow_slow, bool &slow_stop)
{
    slow_stop = false;
    const double Gam = c.o.Gam, g1 = Gam - 1.0;
    const double D = c.in.D;
    // FP32 copies for 1/f' and for the change measures and decisions (a
    // derivative and magnitudes compared with the tolerance: their rounding
    // moves neither the iteration's fixed point nor its FP64 iterate)
    const float Gam_f = d2f_ftz(Gam), gg1_f = d2f_ftz(Gam * (Gam - 1.0)), D_f = d2f_ftz(D);
    const float tol_f = d2f_ftz(c.o.tol), sg_f = FLAT ? 1.0f : d2f_ftz(c.sg);
    const float tD_f = d2f_ftz(c.in.tau + D);   // energy scale: tau + D + sqrt(g) p
    // scale of the change measure (energy at the guess), needed only from
    // the second iteration on
    float iscale0 = 0.0f;
    const int last = limit < c.o.maxit ? limit : c.o.maxit;
    while (s.it < last) {
        const int it = ++s.it;
        if (c.implicit) implicit_field<FLAT>(c, s.v, s.vl, s.v2, s.W, E);
        const double W1 = s.W;   // W of this iteration's implicit solve
        double vn[3], Winv, num, den;
        if (!fluid_step<FLAT>(c, E, s.p, s.vl, vn, s.v2, s.W, Winv, num, &den)) return 0;
        const double omv = 1.0 - s.v2;
        const double f = g1 * num * omv * isgv(c) - s.p;
        double ratio;
        if (num > 0.0) {
            const float num_f = d2f_ftz(num), Winv_f = d2f_ftz(Winv), v2_f = d2f_ftz(s.v2);
            const float gn = Gam_f * num_f * Winv_f;
            ratio = f * f2d_ftz(__fdividef(D_f + gn, v2_f * gg1_f * num_f * Winv_f - D_f - gn));
        } else {
            ratio = -f;
        }
        double pn = s.p - ratio;
        if (!(pn > 0.0)) pn = 0.1 * s.p;
        const float dv = fmaxf(fabsf(d2f_ftz(vn[0] - s.v[0])),
                               fmaxf(fabsf(d2f_ftz(vn[1] - s.v[1])), fabsf(d2f_ftz(vn[2] - s.v[2]))));
        const float dp = fabsf(d2f_ftz(pn - s.p));
        s.p = pn;
        s.v[0] = vn[0]; s.v[1] = vn[1]; s.v[2] = vn[2];
        // step (v): |dp| sqrt(g) <= tol (tau + D + sqrt(g) p) and max|dv| <= tol
        if (dp * sg_f <= tol_f * (tD_f + sg_f * d2f_ftz(pn)) && dv <= tol_f) {
            rho_out = D * Winv * isgv(c);
            return 1;
        }
        // Stiff magnetised states: the velocity update of step (iii) through
        // the implicit field contracts by about kappa = C/(1+C) B^2/den per
        // iteration (C = cc W); a cell that has not converged in its first
        // iteration while kappa > kappa0 would crawl or diverge, and is
        // handed to the stiff-coupling Newton at once (same root)
        if (it == 1 && c.implicit && c.o.kappa0 > 0.0) {
            const float C1_f = d2f_ftz(c.cc) * d2f_ftz(W1);   // coupling cc W
            if (C1_f * d2f_ftz(c.B2) * (FLAT ? 1.0f : d2f_ftz(c.isg)) >
                d2f_ftz(c.o.kappa0) * (1.0f + C1_f) * d2f_ftz(den)) {
                s.slow = 2;
                return 0;
            }
        }
        if (iscale0 == 0.0f) iscale0 = __fdividef(sg_f, tD_f + sg_f * d2f_ftz(p_guess));
        const float meas = dv + dp * iscale0;
        if (!isfinite(meas)) return 0;
        // diverging: three successive growing changes above the noise
        if (it >= 3 && meas > s.prev0 && s.prev0 > s.prev1 && s.prev1 > s.prev2 &&
            meas > 1e3f * tol_f)
            return 0;
        // converging too slowly: more than 24 further iterations predicted
        if (!allow_slow && it >= 6 && meas < s.prev0 && s.prev0 > 0.0f) {
            const float rate = meas / s.prev0;
            if (rate > 0.0f && __logf(tol_f / meas) / __logf(rate) > 24.0f) {
                slow_stop = true;
                return 0;
            }
        }
        s.prev2 = s.prev1; s.prev1 = s.prev0; s.prev0 = meas;
    }
    return s.it >= c.o.maxit ? 0 : -1;
}

// The paper's iteration from the guess, to its cap.  Returns 1 converged,
// 0 gave up.
template <bool FLAT>
__device__ int paper_iteration(const RecCtx<FLAT> &c, double &p, double v[3], double E[3],
                               double &rho_out, int &iters, bool allow_slow, bool &slow_stop)
{
    PaperState s;
    slow_stop = false;
    if (!paper_start<FLAT>(c, p, v, s)) {
        iters = 0;
        return 0;
    }
    const int r = paper_run<FLAT>(c, s, p, c.o.maxit, E, rho_out, allow_slow, slow_stop);
    iters = s.it;
    p = s.p;
    v[0] = s.v[0]; v[1] = s.v[1]; v[2] = s.v[2];
    return r == 1;
}

// residual of the joint system at x = (p, v_lower), scaled by the energy scale
template <bool FLAT>
__device__ __forceinline__ bool joint_residual(const RecCtx<FLAT> &c, const double x[4],
                                               double r[4], double E[3], double &rho,
                                               double v[3])
{
    const double p = x[0];
    const double vl[3] = {x[1], x[2], x[3]};
    raise<double, FLAT>(c.m, vl, v);
    const double v2 = dot3(v, vl);
    if (!(p > 0.0) || !(v2 < c.o.v2max)) return false;
    const double W = rsqrt(1.0 - v2);
    if (c.implicit) {
        implicit_field<FLAT>(c, v, vl, v2, W, E);
    } else {
        E[0] = c.in.cE0[0]; E[1] = c.in.cE0[1]; E[2] = c.in.cE0[2];
    }
    double El[3];
    lower<double, FLAT>(c.m, E, El);
    const double EM = 0.5 * (dot3(E, El) + c.B2) * c.isg;
    double P[3];
    cross3(E, c.in.cB, P);
    const double scale = c.in.tau + c.in.D + c.sg * p;
    const double iscale = 1.0 / scale;
    const double den = scale - EM;
#pragma unroll
    for (int i = 0; i < 3; i++) r[1 + i] = (vl[i] * den - (c.in.S[i] - P[i])) * iscale;
    const double Winv = (1.0 - v2) * W;
    rho = c.in.D * Winv * c.isg;
    const double num = c.in.tau - c.in.D * (W - 1.0) - c.sg * p * (v2 * W * W) - EM;
    const double eps = num * Winv * c.iD;
    r[0] = ((c.o.Gam - 1.0) * rho * eps - p) * c.sg * iscale;
    return true;
}

__device__ __forceinline__ double nrm4(const double r[4])
{
    return sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3]);
}

// A x = b, 4x4, partial pivoting; false if singular
__device__ __forceinline__ bool solve4(double A[16], double b[4], double x[4])
{
#pragma unroll
    for (int col = 0; col < 4; col++) {
        int piv = col;
        double best = fabs(A[col * 4 + col]);
#pragma unroll
        for (int r = col + 1; r < 4; r++)
            if (fabs(A[r * 4 + col]) > best) { best = fabs(A[r * 4 + col]); piv = r; }
        if (best == 0.0) return false;
        if (piv != col) {
#pragma unroll
            for (int k = 0; k < 4; k++) {
                double t = A[col * 4 + k]; A[col * 4 + k] = A[piv * 4 + k]; A[piv * 4 + k] = t;
            }
            double t = b[col]; b[col] = b[piv]; b[piv] = t;
        }
        const double ip = 1.0 / A[col * 4 + col];
#pragma unroll
        for (int r = col + 1; r < 4; r++) {
            const double f = A[r * 4 + col] * ip;
#pragma unroll
            for (int k = col; k < 4; k++) A[r * 4 + k] -= f * A[col * 4 + k];
            b[r] -= f * b[col];
        }
    }
#pragma unroll
    for (int r = 3; r >= 0; r--) {
        double s = b[r];
#pragma unroll
        for (int k = r + 1; k < 4; k++) s -= A[r * 4 + k] * x[k];
        x[r] = s / A[r * 4 + r];
    }
    return true;
}

// Warp-cooperative form of the pressure bracket's velocity solves (WARP =
// true): all 32 lanes of a warp hold the same record and take the same
// branches; the independent evaluations of an iteration run side by side,
// the forward-difference Jacobian's columns on lanes 0..2 and a line
// search's candidate step lengths 2^-k, k = 0..39, on lane k mod 32.  The
// sequential search takes the first k whose candidate is accepted; the warp
// takes the lowest accepted k of each round of 32: the same k for the same
// candidates.  The two compiled forms may round a candidate's residual
// differently (fused multiply-adds), so their roots agree to rounding.
constexpr unsigned WARP_ALL = 0xffffffffu;
constexpr int LS_MAX = 40;   // step halvings of a line search

// 2^-k exactly (the sequential search's step length after k halvings)
__device__ __forceinline__ double halvings(int k)
{
    return __hiloint2double((1023 - k) << 20, 0);
}

// lowest k in [0, LS_MAX) with eval(2^-k, payload) true, its payload
// broadcast to every lane; -1 if none
template <int NP, class F>
__device__ __forceinline__ int warp_line_search(F eval, double out[NP])
{
    const int lane = threadIdx.x & 31;
    for (int base = 0; base < LS_MAX; base += 32) {
        const int k = base + lane;
        double pay[NP];
        const bool ok = k < LS_MAX && eval(halvings(k), pay);
        const unsigned m = __ballot_sync(WARP_ALL, ok);
        if (m) {
            const int src = __ffs(m) - 1;
#pragma unroll
            for (int i = 0; i < NP; i++) out[i] = __shfl_sync(WARP_ALL, pay[i], src);
            return base + src;
        }
    }
    return -1;
}

// Fallback: damped Newton on (p, v_lower) with a forward-difference Jacobian.
template <bool FLAT>
__device__ int newton_fallback(const RecCtx<FLAT> &c, double &p, double v[3], double E[3],
                               double &rho_out, int &iters)
{
    double x[4], r[4], vtmp[3], rho;
    double vl[3];
    lower<double, FLAT>(c.m, v, vl);
    x[0] = p; x[1] = vl[0]; x[2] = vl[1]; x[3] = vl[2];
    if (!joint_residual<FLAT>(c, x, r, E, rho, vtmp)) {
        x[1] = x[2] = x[3] = 0.0;
        if (!(x[0] > 0.0)) x[0] = c.o.p_atmo;
        if (!joint_residual<FLAT>(c, x, r, E, rho, vtmp)) return 0;
    }
    for (int it = 1; it <= 50; it++) {
        iters = it;
        double J[16];
        for (int col = 0; col < 4; col++) {
            double xh[4] = {x[0], x[1], x[2], x[3]}, rh[4], Eh[3], rhoh, vh[3];
            double h = col == 0 ? 1e-7 * x[0] : 1e-7;
            xh[col] += h;
            if (!joint_residual<FLAT>(c, xh, rh, Eh, rhoh, vh)) {
                h = -h;
                xh[col] = x[col] + h;
                if (!joint_residual<FLAT>(c, xh, rh, Eh, rhoh, vh)) return 0;
            }
            const double ih = 1.0 / h;
            for (int row = 0; row < 4; row++) J[row * 4 + col] = (rh[row] - r[row]) * ih;
        }
        double b[4] = {-r[0], -r[1], -r[2], -r[3]}, dx[4];
        if (!solve4(J, b, dx)) return 0;
        const double n0 = nrm4(r);
        double lam = 1.0, xt[4], rt[4], Et[3], rhot, vt[3];
        bool ok = false;
        for (int ls = 0; ls < LS_MAX; ls++) {
            for (int k = 0; k < 4; k++) xt[k] = x[k] + lam * dx[k];
            if (joint_residual<FLAT>(c, xt, rt, Et, rhot, vt) && nrm4(rt) < n0) {
                ok = true;
                break;
            }
            lam *= 0.5;
        }
        if (!ok) {
            const double dvm = fmax(fabs(dx[1]), fmax(fabs(dx[2]), fabs(dx[3])));
            if (p_conv<FLAT>(c, dx[0], x[0]) && dvm <= c.o.tol) break;
            return 0;
        }
        // converged when the full Newton step is below the tolerance (not
        // the damped one, which a line search can make small anywhere)
        const double sv = fmax(fabs(dx[1]), fmax(fabs(dx[2]), fabs(dx[3])));
        for (int k = 0; k < 4; k++) { x[k] = xt[k]; r[k] = rt[k]; }
        if (p_conv<FLAT>(c, dx[0], x[0]) && sv <= c.o.tol) break;
        if (it == 50) return 0;
    }
    if (!joint_residual<FLAT>(c, x, r, E, rho, v)) return 0;
    p = x[0];
    rho_out = rho;
    return 1;
}

// Stiff magnetised cells: Newton on (p, v_lower) for the same two equations the
// paper iteration solves,
//   m_i = v_i den - (S_i - eta_ijk calE^j calB^k) = 0,  den = tau + D + sqrt(g) p - EM,
//   f   = (Gamma-1) num (1-v^2)/sqrt(g) - p = 0,
// with calE = calE(v) from the closed-form implicit solve, and a Jacobian made
// of the terms that dominate when C = cc W >> 1 (calE -> -eps v x calB):
//   dm/dv = (den + k B^2/sqrt(g)) I - (k/sqrt(g)) calB_lower calB^T + v_lower g^T,
//   dm/dp = sqrt(g) v_lower,   g^j = d den/dv_j = (k/gamma) (calB_lower x calE_lower)^j,
//   df/dp = -(Gamma-1) v^2 - 1,
//   df/dv_j = (Gamma-1)/sqrt(g) [(1-v^2)(g^j - D W^3 v^j - 2 sqrt(g) p W^4 v^j) - 2 num v^j],
// k = C/(1+C).  The paper iteration's velocity step multiplies the field's
// feedback by kappa = k B^2/(sqrt(g) den) per iteration, which exceeds 1 in
// a strongly magnetised plasma (B^2 >> rho h); here that linear feedback is on
// the left-hand side.  dm/dv is the identity times a scalar plus two rank-one
// terms, so the 4x4 step is formed by block elimination with two
// Sherman-Morrison solves (no pivoting, no 4x4 factorisation).  Converges in a
// few iterations from the stage guess; a step that leaves the physical
// region is halved, and failure (no convergence in STIFF_MAXIT) leaves the cell
// to the fallbacks.  Same stopping rule as the paper iteration.
constexpr int STIFF_MAXIT = 30;

// E_guess (optional): the implicit field already formed at the starting
// point (the paper iteration's first implicit solve, at the same guess).
template <bool FLAT>
__device__ bool stiff_newton(const RecCtx<FLAT> &c, double &p, double v[3], double E[3],
                             double &rho_out, int &iters, const double *E_guess = nullptr)
{
    const double Gam = c.o.Gam, g1 = Gam - 1.0;
    const double sg = sgv(c), isg = isgv(c);
    // the cell's constants of the FP32 Newton step
    float cB_[3], cBl_[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        cB_[i] = d2f_ftz(c.in.cB[i]);
        cBl_[i] = FLAT ? cB_[i] : d2f_ftz(c.cBl[i]);
    }
    const float B2_ = d2f_ftz(c.B2), cc_ = d2f_ftz(c.cc), D_ = d2f_ftz(c.in.D);
    const float sg_ = FLAT ? 1.0f : d2f_ftz(sg), isg_ = FLAT ? 1.0f : d2f_ftz(isg);
    const float g1_ = d2f_ftz(g1);
    const float tol_f = d2f_ftz(c.o.tol), tD_f = d2f_ftz(c.in.tau + c.in.D);
    double vl[3];
    lower<double, FLAT>(c.m, v, vl);
    double pp = p;
    iters = 0;
    for (int it = 1; it <= STIFF_MAXIT; it++) {
        iters = it;
        double vu[3];
        raise<double, FLAT>(c.m, vl, vu);
        const double v2 = dot3(vu, vl);
        if (!(pp > 0.0) || !(v2 < c.o.v2max)) return false;
        const double W = rsqrt(1.0 - v2);
        if (!c.implicit) {
            E[0] = c.in.cE0[0]; E[1] = c.in.cE0[1]; E[2] = c.in.cE0[2];
        } else if (it == 1 && E_guess) {
            E[0] = E_guess[0]; E[1] = E_guess[1]; E[2] = E_guess[2];
        } else {
            implicit_field<FLAT>(c, vu, vl, v2, W, E);
        }
        double El[3], P[3];
        lower<double, FLAT>(c.m, E, El);
        const double EM = 0.5 * (dot3(E, El) + c.B2) * isg;
        cross3(E, c.in.cB, P);
        const double den = c.in.tau + c.in.D + sg * pp - EM;
        if (!(den > 0.0)) return false;
        double m[3];
#pragma unroll
        for (int i = 0; i < 3; i++) m[i] = vl[i] * den - (c.in.S[i] - P[i]);
        const double W2 = W * W;
        const double num = c.in.tau - c.in.D * (W - 1.0) - sg * pp * (v2 * W2) - EM;
        const double f = g1 * num * (1.0 - v2) * isg - pp;
        // The Newton step from the FP64 residual (m, f): its Jacobian terms
        // and the two solves in FP32 (the step is a correction: an error of
        // ~1e-6 of its own size changes neither the root nor, measured on
        // the blast's stiff cells, the iterations to reach it), which moves
        // about 60% of an iteration's arithmetic off the FP64 pipe.
        double dp, dv[3];
        float dp_abs, sv;   // sizes of the step (stopping rule)
        {
            float vu_[3], vl_[3], El_[3], m_[3];
#pragma unroll
            for (int i = 0; i < 3; i++) {
                vu_[i] = d2f_ftz(vu[i]);
                vl_[i] = FLAT ? vu_[i] : d2f_ftz(vl[i]);
                El_[i] = d2f_ftz(El[i]);
                m_[i] = d2f_ftz(m[i]);
            }
            const float v2_ = d2f_ftz(v2), W_ = d2f_ftz(W), den_ = d2f_ftz(den);
            const float num_ = d2f_ftz(num), f_ = d2f_ftz(f), p_ = d2f_ftz(pp);
            const float C = cc_ * W_;
            const float k = __fdividef(C, 1.0f + C);
            const float kb = FLAT ? k : k * isg_;
            float g[3];
            cross3(cBl_, El_, g);
            const float gk = FLAT ? k : k * isg_ * isg_;
#pragma unroll
            for (int j = 0; j < 3; j++) g[j] *= gk;
            const float W2f = W_ * W_;
            const float fp = -g1_ * v2_ - 1.0f;
            const float cv = -D_ * W2f * W_ - 2.0f * sg_ * p_ * W2f * W2f;
            float fv[3];
#pragma unroll
            for (int j = 0; j < 3; j++)
                fv[j] = g1_ * isg_ * ((1.0f - v2_) * (g[j] + cv * vu_[j]) - 2.0f * num_ * vu_[j]);
            // N0 = alpha I - kb calB_lower calB^T: N0^-1 x = [x + kb calB_lower (calB.x)/den]/alpha
            const float ialpha = __fdividef(1.0f, den_ + kb * B2_);
            const float kd = __fdividef(kb, den_);
            float y[3], z[3];
            const float bv = dot3(cB_, vl_), bm = dot3(cB_, m_);
#pragma unroll
            for (int i = 0; i < 3; i++) {
                y[i] = (vl_[i] + kd * bv * cBl_[i]) * ialpha;   // N0^-1 v_lower
                z[i] = (m_[i] + kd * bm * cBl_[i]) * ialpha;    // N0^-1 m
            }
            // N = N0 + v_lower g^T; a = -N^-1 m, b = N^-1 (sqrt(g) v_lower)
            const float is = __fdividef(1.0f, 1.0f + dot3(g, y));
            const float gz = dot3(g, z) * is;
            float a[3], b[3];
#pragma unroll
            for (int i = 0; i < 3; i++) {
                a[i] = y[i] * gz - z[i];
                b[i] = sg_ * y[i] * is;
            }
            const float dp_ = -__fdividef(f_ + dot3(fv, a), fp - dot3(fv, b));
            dp = f2d_ftz(dp_);
            dp_abs = fabsf(dp_);
            sv = 0.0f;
#pragma unroll
            for (int i = 0; i < 3; i++) {
                const float d = a[i] - b[i] * dp_;
                dv[i] = f2d_ftz(d);
                sv = fmaxf(sv, fabsf(d));
            }
        }
        // keep the iterate physical: halve a step that leaves the region
        double lam = 1.0, pn = 0.0, vln[3];
        bool ok = false;
        for (int h = 0; h < 8; h++) {
            pn = pp + lam * dp;
#pragma unroll
            for (int i = 0; i < 3; i++) vln[i] = vl[i] + lam * dv[i];
            double vt[3];
            raise<double, FLAT>(c.m, vln, vt);
            if (pn > 0.0 && dot3(vt, vln) < c.o.v2max) {
                ok = true;
                break;
            }
            lam *= 0.5;
        }
        if (!ok || !isfinite(dp)) return false;
        pp = pn;
        vl[0] = vln[0]; vl[1] = vln[1]; vl[2] = vln[2];
        // converged when the full Newton step is below the tolerance (a
        // halved step is small near the edge of the region without the
        // equations being solved)
        if (lam == 1.0 && dp_abs * sg_ <= tol_f * (tD_f + sg_ * d2f_ftz(pp)) && sv <= tol_f) {
            raise<double, FLAT>(c.m, vl, v);
            const double v2f = dot3(v, vl);
            const double Wf = rsqrt(1.0 - v2f);
            if (c.implicit) implicit_field<FLAT>(c, v, vl, v2f, Wf, E);
            p = pp;
            rho_out = c.in.D * ((1.0 - v2f) * Wf) * isg;
            return true;
        }
    }
    return false;
}

// Velocity equations at fixed p (x = v_lower):
//   g_i = [v_i (tau + D + sqrt(g) p - EM) - (S_i - eta_ijk calE^j calB^k)] / scale
template <bool FLAT>
__device__ __forceinline__ bool vel_residual(const RecCtx<FLAT> &c, double p, const double vl[3],
                                             double g[3], double E[3], double &v2o)
{
    double v[3];
    raise<double, FLAT>(c.m, vl, v);
    const double v2 = dot3(v, vl);
    if (!(v2 < c.o.v2max)) return false;
    if (c.implicit) {
        implicit_field<FLAT>(c, v, vl, v2, rsqrt(1.0 - v2), E);
    } else {
        E[0] = c.in.cE0[0]; E[1] = c.in.cE0[1]; E[2] = c.in.cE0[2];
    }
    double El[3];
    lower<double, FLAT>(c.m, E, El);
    const double EM = 0.5 * (dot3(E, El) + c.B2) * c.isg;
    double P[3];
    cross3(E, c.in.cB, P);
    const double scale = c.in.tau + c.in.D + c.sg * p;
    const double iscale = 1.0 / scale;
    const double den = scale - EM;
#pragma unroll
    for (int i = 0; i < 3; i++) g[i] = (vl[i] * den - (c.in.S[i] - P[i])) * iscale;
    v2o = v2;
    return true;
}

__device__ __forceinline__ double nrm3(const double g[3])
{
    return sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
}

// velocity at fixed p: damped Newton with a forward-difference Jacobian;
// gives up after eight damped steps in a row
template <bool FLAT, bool WARP = false>
__device__ bool velocity_at(const RecCtx<FLAT> &c, double p, double vl[3])
{
    double g[3], E[3], v2;
    int damped = 0;
    if (!vel_residual<FLAT>(c, p, vl, g, E, v2)) return false;
    for (int it = 0; it < 30; it++) {
        double J[9];
        if constexpr (WARP) {
            // column `lane` on lanes 0..2, then every column on every lane
            const int lane = threadIdx.x & 31;
            double colv[3] = {0.0, 0.0, 0.0};
            bool bad = false;
            if (lane < 3) {
                double vh[3], gh[3], Eh[3], v2h, h = 1e-7;
                const double v0 = lane == 0 ? vl[0] : lane == 1 ? vl[1] : vl[2];
                double vc = v0 + h;
                vh[0] = lane == 0 ? vc : vl[0];
                vh[1] = lane == 1 ? vc : vl[1];
                vh[2] = lane == 2 ? vc : vl[2];
                if (!vel_residual<FLAT>(c, p, vh, gh, Eh, v2h)) {
                    h = -h;
                    vc = v0 + h;
                    vh[0] = lane == 0 ? vc : vl[0];
                    vh[1] = lane == 1 ? vc : vl[1];
                    vh[2] = lane == 2 ? vc : vl[2];
                    bad = !vel_residual<FLAT>(c, p, vh, gh, Eh, v2h);
                }
                if (!bad) {
                    const double ih = 1.0 / h;
                    for (int row = 0; row < 3; row++) colv[row] = (gh[row] - g[row]) * ih;
                }
            }
            if (__any_sync(WARP_ALL, bad)) return false;
#pragma unroll
            for (int col = 0; col < 3; col++)
#pragma unroll
                for (int row = 0; row < 3; row++)
                    J[row * 3 + col] = __shfl_sync(WARP_ALL, colv[row], col);
        } else {
            for (int col = 0; col < 3; col++) {
                double vh[3] = {vl[0], vl[1], vl[2]}, gh[3], h = 1e-7;
                vh[col] += h;
                if (!vel_residual<FLAT>(c, p, vh, gh, E, v2)) {
                    h = -h;
                    vh[col] = vl[col] + h;
                    if (!vel_residual<FLAT>(c, p, vh, gh, E, v2)) return false;
                }
                const double ih = 1.0 / h;
                for (int row = 0; row < 3; row++) J[row * 3 + col] = (gh[row] - g[row]) * ih;
            }
        }
        // 3x3 solve by Cramer's rule on -g
        const double det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
                           J[2] * (J[3] * J[7] - J[4] * J[6]);
        if (!(fabs(det) > 0.0)) return false;
        const double id = 1.0 / det;
        const double b0 = -g[0], b1 = -g[1], b2 = -g[2];
        double dv[3];
        dv[0] = (b0 * (J[4] * J[8] - J[5] * J[7]) - J[1] * (b1 * J[8] - J[5] * b2) +
                 J[2] * (b1 * J[7] - J[4] * b2)) * id;
        dv[1] = (J[0] * (b1 * J[8] - J[5] * b2) - b0 * (J[3] * J[8] - J[5] * J[6]) +
                 J[2] * (J[3] * b2 - b1 * J[6])) * id;
        dv[2] = (J[0] * (J[4] * b2 - b1 * J[7]) - J[1] * (J[3] * b2 - b1 * J[6]) +
                 b0 * (J[3] * J[7] - J[4] * J[6])) * id;
        const double n0 = nrm3(g);
        double lam = 1.0, vt[3], gt[3];
        bool ok = false;
        if constexpr (WARP) {
            double pay[6];
            const int k = warp_line_search<6>(
                [&](double lm, double *q) {
                    double vq[3], gq[3], Eq[3], v2q;
                    for (int i = 0; i < 3; i++) vq[i] = vl[i] + lm * dv[i];
                    const bool good = vel_residual<FLAT>(c, p, vq, gq, Eq, v2q) && nrm3(gq) < n0;
                    for (int i = 0; i < 3; i++) { q[i] = vq[i]; q[3 + i] = gq[i]; }
                    return good;
                },
                pay);
            if (k >= 0) {
                ok = true;
                lam = halvings(k);
                for (int i = 0; i < 3; i++) { vt[i] = pay[i]; gt[i] = pay[3 + i]; }
            }
        } else {
            for (int ls = 0; ls < LS_MAX; ls++) {
                for (int i = 0; i < 3; i++) vt[i] = vl[i] + lam * dv[i];
                if (vel_residual<FLAT>(c, p, vt, gt, E, v2) && nrm3(gt) < n0) {
                    ok = true;
                    break;
                }
                lam *= 0.5;
            }
        }
        if (!ok) return n0 < 1e-13;
        // eight damped steps in a row: creeping toward a minimum of |g| that
        // is not a solution; the pressure counts as undefined
        damped = lam < 1.0 ? damped + 1 : 0;
        if (damped >= 8) return false;
        const double step = lam * fmax(fabs(dv[0]), fmax(fabs(dv[1]), fabs(dv[2])));
        for (int i = 0; i < 3; i++) { vl[i] = vt[i]; g[i] = gt[i]; }
        if (step <= 1e-15) break;
    }
    // solved only if the equations hold (scaled residual at rounding level)
    return nrm3(g) < 1e-13;
}

// scaled f(p) = (Gamma-1) rho eps - p with the velocity solved at p
// (Newton from vl; if that does not converge, from rest)
template <bool FLAT, bool WARP = false>
__device__ bool pressure_function(const RecCtx<FLAT> &c, double p, double vl[3], double &f,
                                  double E[3], double &rho)
{
    if (!(p > 0.0)) return false;
    if (!velocity_at<FLAT, WARP>(c, p, vl)) {
        vl[0] = vl[1] = vl[2] = 0.0;
        if (!velocity_at<FLAT, WARP>(c, p, vl)) return false;
    }
    double g[3], v2;
    vel_residual<FLAT>(c, p, vl, g, E, v2);
    double El[3];
    lower<double, FLAT>(c.m, E, El);
    const double EM = 0.5 * (dot3(E, El) + c.B2) * c.isg;
    const double W = rsqrt(1.0 - v2);
    const double Winv = (1.0 - v2) * W;
    rho = c.in.D * Winv * c.isg;
    const double num = c.in.tau - c.in.D * (W - 1.0) - c.sg * p * (v2 * W * W) - EM;
    const double eps = num * Winv * c.iD;
    f = ((c.o.Gam - 1.0) * rho * eps - p) * c.sg / (c.in.tau + c.in.D + c.sg * p);
    return true;
}

// Second fallback: the pressure root with the velocity solved at every trial
// pressure.  f is defined only above the lowest pressure at which the
// velocity equations have a solution with v^2 < 1, so a pressure where the
// solve fails lies below the root: where f is undefined at the guess, the
// smallest defined guess x 2^k (k <= 60) by bisection on k; from there,
// double the pressure while f is positive, halve it while f is negative,
// replacing a halving that lands where f is undefined by geometric bisection
// between that pressure and the last one where f was defined (to 1e-9);
// then Illinois regula falsi on the bracket.
template <bool FLAT, bool WARP = false>
__device__ int bracket_fallback(const RecCtx<FLAT> &c, double &p, double v[3], double E[3],
                                double &rho_out, int &iters)
{
    double vl[3], v0[3], f0 = 0.0, rho;
    lower<double, FLAT>(c.m, v, v0);
    vl[0] = v0[0]; vl[1] = v0[1]; vl[2] = v0[2];
    double p0 = p > 0.0 ? p : c.o.p_atmo;
    int n = 0;
    bool ok = pressure_function<FLAT, WARP>(c, p0, vl, f0, E, rho);
    if (!ok) {
        // f undefined at the guess: the root is above.  f is defined exactly
        // above the lowest pressure where the velocity equations have a
        // solution, so the smallest defined p0 2^k, k = 1 ... 60 (each tried
        // from the guess velocity), is found by bisection on k
        int klo = 0, khi = 60;
        double vk[3] = {v0[0], v0[1], v0[2]}, fk;
        if (!pressure_function<FLAT, WARP>(c, p0 * ldexp(1.0, khi), vk, fk, E, rho)) return 0;
        vl[0] = vk[0]; vl[1] = vk[1]; vl[2] = vk[2];
        f0 = fk;
        while (khi - klo > 1) {
            const int km = (klo + khi) / 2;
            vk[0] = v0[0]; vk[1] = v0[1]; vk[2] = v0[2];
            if (pressure_function<FLAT, WARP>(c, p0 * ldexp(1.0, km), vk, fk, E, rho)) {
                khi = km;
                f0 = fk;
                vl[0] = vk[0]; vl[1] = vk[1]; vl[2] = vk[2];
            } else {
                klo = km;
            }
        }
        n = khi;
        p0 = p0 * ldexp(1.0, khi);
    }
    double lo = p0, hi = p0, flo = f0, fhi = f0;
    double vlo[3] = {vl[0], vl[1], vl[2]}, vhi[3] = {vl[0], vl[1], vl[2]};
    if (f0 > 0.0) {
        while (fhi > 0.0) {
            if (++n > 60) return 0;
            lo = hi; flo = fhi;
            for (int i = 0; i < 3; i++) vlo[i] = vhi[i];
            hi = 2.0 * hi;
            if (!pressure_function<FLAT, WARP>(c, hi, vhi, fhi, E, rho)) return 0;
        }
    } else {
        // hi: f < 0 and defined; und: a lower pressure where f is undefined
        double und = 0.0;
        while (flo < 0.0) {
            if (++n > 120) return 0;
            const double pt = und > 0.0 ? sqrt(und * hi) : 0.5 * hi;
            double vt[3] = {vhi[0], vhi[1], vhi[2]}, ft;
            if (!pressure_function<FLAT, WARP>(c, pt, vt, ft, E, rho)) {
                und = pt;
                // f < 0 down to within 1e-9 of the lowest defined pressure:
                // no root
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
    for (int it = 0; it < 100; it++) {
        iters = n + it + 1;
        double pm = (lo * fhi - hi * flo) / (fhi - flo);
        if (!(pm > lo && pm < hi)) pm = 0.5 * (lo + hi);
        double vm[3] = {vlo[0], vlo[1], vlo[2]}, fm;
        if (!pressure_function<FLAT, WARP>(c, pm, vm, fm, E, rho)) return 0;
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
        if ((hi - lo) * c.sg <= c.o.tol * (c.in.tau + c.in.D + c.sg * hi) || fm == 0.0) {
            p = pm;
            raise<double, FLAT>(c.m, vm, v);
            rho_out = rho;
            return 1;
        }
    }
    return 0;
}

// phases of recover(): everything inline, only the paper iteration (a cell it
// does not converge is handed back as REC_DEFER for a later fallback pass),
// or only the fallbacks (the deferred pass)
// REC_FIRST: at most RecOpts::first_cap paper iterations; a point still
// undecided then is handed back with its iterate in *ps, and a later pass
// with REC_RESUME continues from exactly there (same arithmetic, same
// decisions, same result as REC_ALL inline).
// REC_RESUME_NEWTON: as REC_RESUME, but a point whose paper iteration and
// both Newton methods fail is handed back as REC_HARD (its iterate in *ps
// marked given up) for the rest of the chain; REC_CHAIN_REST runs that rest
// (the pressure bracket, the atmosphere), with WARP = true on a whole warp
// per point.
enum { REC_ALL = 0, REC_PRIMARY = 1, REC_FALLBACK = 2, REC_FIRST = 3, REC_RESUME = 4,
       REC_RESUME_NEWTON = 5, REC_CHAIN_REST = 6 };
enum { REC_DEFER = -1, REC_HARD = -2 };

// Full pointwise recovery.  Writes the 14 primitives and the solved calE;
// returns the status 0 (paper iteration), 1 (Newton fallback), 4 (pressure
// bracket fallback), 2 (failed, atmosphere), 3 (rho below the floor,
// atmosphere), or REC_DEFER (phase REC_PRIMARY only; nothing written).
// guess_p, guess_v: previous stage.
template <bool FLAT, bool WARP = false>
__device__ int recover(const RecIn &in, const Met<double> &m, const RecOpts &o,
                       bool implicit, double cc, double guess_p, const double guess_v[3],
                       double Phi, double Psi, double Q, double prim[NPR],
                       double Eout[3], int &iters, int phase = REC_ALL,
                       PaperState *ps = nullptr)
{
    RecCtx<FLAT> c{in, m, o, implicit, implicit ? cc : 0.0, 1.0, 1.0, 0.0, {0, 0, 0}, 0.0};
    if (!FLAT) {
        c.sg = m.sg;
        c.isg = m.isg;
    }
    lower<double, FLAT>(m, in.cB, c.cBl);
    c.B2 = dot3(in.cB, c.cBl);

    double p = guess_p, v[3] = {guess_v[0], guess_v[1], guess_v[2]};
    double E[3] = {in.cE0[0], in.cE0[1], in.cE0[2]};
    double rho = 0.0;
    int it1 = 0, it2 = 0, status;
    bool slow = false;
    bool newton_inline = false;   // REC_FIRST: the stiff switch's Newton converged
    int first = -2;   // REC_FIRST / REC_RESUME outcome of the paper iteration
    // atmosphere without iterating: rho = D / (W sqrt(gamma)) <= D / sqrt(gamma)
    // for every velocity, so below the floor there every root is reset
    const bool atmo = !((FLAT ? in.D : in.D / m.sg) >= o.atmo_floor);
    if (atmo) {
        status = 3;
    } else {
        const bool resume =
            phase == REC_RESUME || phase == REC_RESUME_NEWTON || phase == REC_CHAIN_REST;
        if (phase == REC_FIRST || resume) {
            PaperState s;
            if (phase == REC_FIRST) {
                // undecided or given up: both go to the second pass
                if (!paper_start<FLAT>(c, p, v, s)) {
                    s.it = 0;
                    s.p = p;
                    first = 0;
                } else {
                    first = paper_run<FLAT>(c, s, guess_p, o.first_cap, E, rho, false, slow);
                }
                if (first == 0 && s.slow == 2) {
                    // stiff switch (paper_run): the stiff-coupling Newton here,
                    // from the stage guess; deferred only if it fails
                    double pn = guess_p, vn[3] = {guess_v[0], guess_v[1], guess_v[2]};
                    double En[3] = {in.cE0[0], in.cE0[1], in.cE0[2]}, rhon = 0.0;
                    int itn = 0;
                    if (stiff_newton<FLAT>(c, pn, vn, En, rhon, itn, E)) {
                        newton_inline = true;
                        it1 = s.it;
                        it2 = itn;
                        p = pn; rho = rhon;
                        v[0] = vn[0]; v[1] = vn[1]; v[2] = vn[2];
                        E[0] = En[0]; E[1] = En[1]; E[2] = En[2];
                    }
                }
                if (first != 1 && !newton_inline) {
                    s.outcome = first;
                    s.slow = slow || s.slow == 2 ? 1 : 0;
                    *ps = s;
                    iters = s.it;
                    return REC_DEFER;
                }
            } else {
                s = *ps;
                if (s.outcome == 0) {
                    first = 0;
                    slow = s.slow != 0;
                } else {
                    first = paper_run<FLAT>(c, s, guess_p, o.maxit, E, rho, false, slow);
                }
            }
            if (!newton_inline) {
                it1 = s.it;
                p = s.p;
                v[0] = s.v[0]; v[1] = s.v[1]; v[2] = s.v[2];
            }
        }
        // outcome of the paper iteration: 1 converged, 0 gave up
        int paper;
        if (newton_inline)
            paper = 2;
        else if (first != -2)
            paper = first;
        else if (phase == REC_FALLBACK)
            paper = 0;
        else
            paper = paper_iteration<FLAT>(c, p, v, E, rho, it1, false, slow) ? 1 : 0;
        if (paper == 2) {
            status = 1;
        } else if (paper == 1) {
            status = 0;
        } else if (phase == REC_PRIMARY) {
            iters = it1;
            return REC_DEFER;
        } else {
            c.iD = 1.0 / in.D;
            p = guess_p;
            v[0] = guess_v[0]; v[1] = guess_v[1]; v[2] = guess_v[2];
            E[0] = in.cE0[0]; E[1] = in.cE0[1]; E[2] = in.cE0[2];
            // the Newton method with the field-feedback Jacobian (exact with
            // the field fixed), then the damped forward-difference Newton,
            // then the pressure bracket
            // (REC_CHAIN_REST: both Newton methods failed in the pass before)
            const bool rest = phase == REC_CHAIN_REST;
            status = rest ? 2 : stiff_newton<FLAT>(c, p, v, E, rho, it2) ? 1 : 2;
            if (status == 2) {
                p = guess_p;
                v[0] = guess_v[0]; v[1] = guess_v[1]; v[2] = guess_v[2];
                E[0] = in.cE0[0]; E[1] = in.cE0[1]; E[2] = in.cE0[2];
            }
            if (status == 2 && !rest) {
                int itn = 0;
                status = newton_fallback<FLAT>(c, p, v, E, rho, itn) ? 1 : 2;
                it2 += itn;
            }
            if (status == 2 && phase == REC_RESUME_NEWTON) {
                ps->outcome = 0;
                ps->slow = slow ? 1 : 0;
                iters = it1 + it2;
                return REC_HARD;
            }
            if (status == 2) {
                int it3 = 0;
                p = guess_p;
                v[0] = guess_v[0]; v[1] = guess_v[1]; v[2] = guess_v[2];
                E[0] = in.cE0[0]; E[1] = in.cE0[1]; E[2] = in.cE0[2];
                if (bracket_fallback<FLAT, WARP>(c, p, v, E, rho, it3)) status = 4;
                it2 += it3;
            }
            if (status == 2) {
                // both fallbacks failed: if the paper iteration was stopped only
                // for being slow (decided again here in the deferred pass), let
                // it run to its cap
                int it4 = 0;
                bool slow2 = false;
                double p4 = guess_p, v4[3] = {guess_v[0], guess_v[1], guess_v[2]};
                double E4[3] = {in.cE0[0], in.cE0[1], in.cE0[2]}, rho4 = 0.0;
                if (phase == REC_FALLBACK || slow) {
                    if (phase == REC_FALLBACK)
                        paper_iteration<FLAT>(c, p4, v4, E4, rho4, it4, false, slow2);
                    if ((slow || slow2)) {
                        p4 = guess_p;
                        v4[0] = guess_v[0]; v4[1] = guess_v[1]; v4[2] = guess_v[2];
                        E4[0] = in.cE0[0]; E4[1] = in.cE0[1]; E4[2] = in.cE0[2];
                        int it5 = 0;
                        bool dummy;
                        if (paper_iteration<FLAT>(c, p4, v4, E4, rho4, it5, true, dummy)) {
                            status = 0;
                            p = p4; rho = rho4;
                            v[0] = v4[0]; v[1] = v4[1]; v[2] = v4[2];
                            E[0] = E4[0]; E[1] = E4[1]; E[2] = E4[2];
                        }
                        it4 += it5;
                    }
                }
                it2 += it4;
            }
        }
    }   // not atmosphere
    iters = it1 + it2;
    if ((status == 0 || status == 1 || status == 4) && !(rho >= o.atmo_floor)) status = 3;
    if (status == 2 || status == 3) {
        rho = o.rho_atmo;
        p = o.p_atmo;
        v[0] = v[1] = v[2] = 0.0;
        const double s = implicit ? 1.0 / (1.0 + c.cc) : 1.0;
        for (int i = 0; i < 3; i++) E[i] = in.cE0[i] * s;
    }
    prim[PR_RHO] = rho;
    prim[PR_P] = p;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        prim[PR_VX + i] = v[i];
        prim[PR_EX + i] = FLAT ? E[i] : E[i] * c.isg;
        prim[PR_BX + i] = FLAT ? in.cB[i] : in.cB[i] * c.isg;
        Eout[i] = E[i];
    }
    prim[PR_PSI] = FLAT ? Psi : Psi * c.isg;
    prim[PR_PHI] = FLAT ? Phi : Phi * c.isg;
    prim[PR_Q] = FLAT ? Q : Q * c.isg;
    return status;
}

} // namespace rmhd
