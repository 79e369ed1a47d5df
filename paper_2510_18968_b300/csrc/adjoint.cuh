// adjoint.cuh -- discrete adjoint of the FP64 IMEX-SSP2(2,2,2) step.
//
// The paper has no adjoint; this is the reverse of the step the stepping
// kernels take (Table imex, Eq. IMEX3, Sec. III.B), per cell and per face:
//   stage 1   (P1, calE1) = Rec(U^n),            dR1 = (calE1 - calE^n)/gamma,
//             J1 = Q^n v1 - dR1/(alpha dt)
//   stage 2   U* = U^n + dt F(P1, J1) + (1 - 2gamma) dR1   (calE rows),
//             (P2, calE2) = Rec(U*),             dR2 = (calE2 - calE*)/gamma,
//             J2 = Q* v2 - dR2/(alpha dt)
//   final     U^{n+1} = U^n + dt/2 (F(P1, J1) + F(P2, J2)) + (dR1 + dR2)/2
// F(P, J) = sources(P) - sum_d (F_d(i+1/2) - F_d(i-1/2))/dx_d with the face
// flux HLLE(recon(P, J)).  The face flux is reversed by hand (WENO5 / TVD
// gradients and the reverse of the one-side face physics); the sources and
// prim-to-con Jacobians come from the forward device code evaluated on dual
// numbers; the recovery is differentiated at its
// converged root by the implicit-function theorem, so the iteration that
// found the root (paper iteration or fallback) does not matter.  Branches
// (limiters, first-order fallbacks, atmosphere resets) are frozen at the
// primal point: a reset cell passes no derivative through rho, p, v.
#pragma once
#include "dual.cuh"
#include "kernels.cuh"

namespace rmhd {

// ------------------------------------------------------------ recovery

// inputs of the pointwise recovery: D, S_i, tau, calB^i, calE^i (calE* of
// the stage when implicit), cc = gamma dt alpha sigma
enum { RU_D = 0, RU_S = 1, RU_TAU = 4, RU_B = 5, RU_E = 8, RU_CC = 11, NRU = 12 };
// outputs: rho, p, v^i, primitive E^i, densitised calE^i
enum { RH_RHO = 0, RH_P = 1, RH_V = 2, RH_EP = 5, RH_CE = 8, NRH = 11 };

// The recovery's equations at x = (p, v_i): r = 0 at the root the stepping
// kernels converge to (the velocity equations v_i den = S_i - (calE x calB)_i
// and the EOS residual (Gamma-1) rho eps - p of Sec. III.B, with calE the
// closed-form stage field at fixed v), and the outputs h at x.
template <bool FLAT, class R>
__device__ __forceinline__ void rec_system(const Met<double> &m, bool implicit, double Gam,
                                           const R u[NRU], const R x[4], R r[4], R h[NRH])
{
    const Met<R> mr = met_cast<R>(m);
    const double sg = FLAT ? 1.0 : m.sg, isg = FLAT ? 1.0 : m.isg;
    const R p = x[0];
    R vl[3] = {x[1], x[2], x[3]}, v[3];
    raise<R, FLAT>(mr, vl, v);
    const R v2 = dot3(v, vl);
    const R omv = 1.0 - v2;
    const R W = 1.0 / sqrt(omv);
    R cB[3] = {u[RU_B], u[RU_B + 1], u[RU_B + 2]}, cBl[3];
    lower<R, FLAT>(mr, cB, cBl);
    R E[3];
    if (implicit) {
        const R C = u[RU_CC] * W;
        R vxB[3];
        cross3(vl, cBl, vxB);
        R rr[3];
#pragma unroll
        for (int i = 0; i < 3; i++) rr[i] = u[RU_E + i] - C * vxB[i] * isg;
        const R s = dot3(vl, rr);
        const R q = 1.0 + C * omv;
        const R inv = 1.0 / ((1.0 + C) * q);
#pragma unroll
        for (int i = 0; i < 3; i++) E[i] = (rr[i] * q + C * v[i] * s) * inv;
    } else {
#pragma unroll
        for (int i = 0; i < 3; i++) E[i] = u[RU_E + i];
    }
    R El[3];
    lower<R, FLAT>(mr, E, El);
    const R EM = 0.5 * (dot3(E, El) + dot3(cB, cBl)) * isg;
    R P[3];
    cross3(E, cB, P);
    const R den = u[RU_TAU] + u[RU_D] + sg * p - EM;
#pragma unroll
    for (int i = 0; i < 3; i++) r[1 + i] = vl[i] * den - (u[RU_S + i] - P[i]);
    const R num = u[RU_TAU] - u[RU_D] * (W - 1.0) - sg * p * (v2 * W * W) - EM;
    r[0] = (Gam - 1.0) * num * omv * isg - p;
    h[RH_RHO] = u[RU_D] * omv * W * isg;
    h[RH_P] = p;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        h[RH_V + i] = v[i];
        h[RH_EP + i] = E[i] * isg;
        h[RH_CE + i] = E[i];
    }
}

// lu = dh/du^T lh at the root x0: lu = h_u^T lh - r_u^T mu, r_x^T mu = h_x^T lh.
// False if r_x is singular there.
template <bool FLAT>
__device__ bool rec_vjp(const Met<double> &m, bool implicit, double Gam, const double u0[NRU],
                        const double x0[4], const double lh[NRH], double lu[NRU])
{
    double A[16], b[4], mu[4];
    {
        Dual<4> u[NRU], x[4], r[4], h[NRH];
        for (int k = 0; k < NRU; k++) u[k] = Dual<4>(u0[k]);
        for (int j = 0; j < 4; j++) x[j] = seed<4>(x0[j], j);
        rec_system<FLAT>(m, implicit, Gam, u, x, r, h);
        for (int i = 0; i < 4; i++)
            for (int j = 0; j < 4; j++) A[j * 4 + i] = r[i].d[j];   // r_x transposed
        for (int j = 0; j < 4; j++) {
            double s = 0.0;
            for (int o = 0; o < NRH; o++) s += h[o].d[j] * lh[o];
            b[j] = s;
        }
    }
    if (!solve4(A, b, mu)) return false;
    for (int g = 0; g < NRU; g += 4) {
        Dual<4> u[NRU], x[4], r[4], h[NRH];
        for (int k = 0; k < NRU; k++) u[k] = Dual<4>(u0[k]);
        for (int j = 0; j < 4; j++) u[g + j].d[j] = 1.0;
        for (int j = 0; j < 4; j++) x[j] = Dual<4>(x0[j]);
        rec_system<FLAT>(m, implicit, Gam, u, x, r, h);
        for (int j = 0; j < 4; j++) {
            double s = 0.0;
            for (int o = 0; o < NRH; o++) s += h[o].d[j] * lh[o];
            for (int i = 0; i < 4; i++) s -= r[i].d[j] * mu[i];
            lu[g + j] = s;
        }
    }
    return true;
}

// d cc / d D of the density-dependent conductivities (Eqs. sigma_evol,
// dynamo_sigma), as a factor of cc
__device__ __forceinline__ double dlogsigma_dD(const StepConst &K, double D)
{
    if (K.sigma_model == 2) return K.sigma_exp / D;
    if (K.sigma_model == 3) {
        const double t = 1.0 - K.D_atmo / D;
        return t > 0.0 ? 2.0 * K.D_atmo / (D * D * t) : 0.0;
    }
    return 0.0;
}

// Adjoint of one recovery at a cell.  P: its converged primitives; lamP the
// adjoint of P (14) and lamCE of the solved calE (3, implicit only).  Adds
// the adjoint of its conserved input to lamU and returns the adjoint of cc.
template <bool FLAT>
__device__ double rec_adjoint(const StepConst &K, const Met<double> &m, bool implicit,
                              double cc, const double u[NCO], const double P[NPR],
                              const double lamP[NPR], const double lamCE[3], double lamU[NCO],
                              int *bad)
{
    const double isg = FLAT ? 1.0 : m.isg;
    // fields the recovery passes through: calB, Phi, Psi, Q over sqrt(gamma)
#pragma unroll
    for (int a = 0; a < 3; a++) lamU[CO_BX + a] += lamP[PR_BX + a] * isg;
    lamU[CO_PSI] += lamP[PR_PSI] * isg;
    lamU[CO_PHI] += lamP[PR_PHI] * isg;
    lamU[CO_Q] += lamP[PR_Q] * isg;
    double lcc = 0.0;
    if (P[PR_RHO] < K.ro.atmo_floor) {
        // atmosphere: rho, p, v fixed; calE = calE*/(1 + cc) (implicit) or calE
        const double s = implicit ? 1.0 / (1.0 + cc) : 1.0;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const double lE = (implicit ? lamCE[a] : 0.0) + lamP[PR_EX + a] * isg;
            lamU[CO_EX + a] += lE * s;
            if (implicit) lcc -= lE * u[CO_EX + a] * s * s;
        }
        return lcc;
    }
    double u0[NRU], x0[4], lh[NRH], lu[NRU];
    u0[RU_D] = u[CO_D];
    u0[RU_TAU] = u[CO_TAU];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        u0[RU_S + a] = u[CO_SX + a];
        u0[RU_B + a] = u[CO_BX + a];
        u0[RU_E + a] = u[CO_EX + a];
    }
    u0[RU_CC] = implicit ? cc : 0.0;
    double v[3] = {P[PR_VX], P[PR_VY], P[PR_VZ]}, vl[3];
    lower<double, FLAT>(m, v, vl);
    x0[0] = P[PR_P];
    x0[1] = vl[0]; x0[2] = vl[1]; x0[3] = vl[2];
    lh[RH_RHO] = lamP[PR_RHO];
    lh[RH_P] = lamP[PR_P];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        lh[RH_V + a] = lamP[PR_VX + a];
        lh[RH_EP + a] = lamP[PR_EX + a];
        lh[RH_CE + a] = implicit ? lamCE[a] : 0.0;
    }
    if (!rec_vjp<FLAT>(m, implicit, K.ro.Gam, u0, x0, lh, lu)) {
        atomicOr(bad, 1);
        return 0.0;
    }
    lamU[CO_D] += lu[RU_D];
    lamU[CO_TAU] += lu[RU_TAU];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        lamU[CO_SX + a] += lu[RU_S + a];
        lamU[CO_BX + a] += lu[RU_B + a];
        lamU[CO_EX + a] += lu[RU_E + a];
    }
    return implicit ? lu[RU_CC] : 0.0;
}

// Adjoint of an implicit stage at a cell given the adjoints of its outputs:
// primitives lamP (from the explicit part that used them), current lamJ and
// the direct adjoint lamdR of Dt R.  Writes the adjoint of the stage input
// uin to lamU and returns dL/dlog(sigma0) of the cell.
template <bool FLAT>
__device__ double stage_adjoint(const StepConst &K, const Met<double> &m, const double *sig,
                                long long c, const double uin[NCO], const double P[NPR],
                                double lamP[NPR], const double lamJ[3], const double lamdR_in[3],
                                double lamU[NCO], int *bad)
{
    const double iad = K.idt / m.alpha;
    for (int f = 0; f < NCO; f++) lamU[f] = 0.0;
    double lamCE[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        // J = Q v - dR/(alpha dt)
        lamU[CO_Q] += lamJ[a] * P[PR_VX + a];
        lamP[PR_VX + a] += lamJ[a] * uin[CO_Q];
        const double ldR = lamdR_in[a] - lamJ[a] * iad;
        // dR = (calE - calE_in)/gamma
        lamCE[a] = ldR * K.igimex;
        lamU[CO_EX + a] -= ldR * K.igimex;
    }
    const double cc = K.gimex * K.dt * m.alpha * sigma_cell(K, sig, c, uin[CO_D]);
    const double lcc = rec_adjoint<FLAT>(K, m, true, cc, uin, P, lamP, lamCE, lamU, bad);
    // cc = gamma dt alpha sigma0 f(D): d/dlog sigma0 = cc, d/dD = cc dlog f/dD
    lamU[CO_D] += lcc * cc * dlogsigma_dD(K, uin[CO_D]);
    return lcc * cc;
}

// Fixed-order sum of the per-cell values v (padded layout) over the
// interior, one block: each thread sums a strided subset in order, then a
// shared-memory tree.  *out = the sum.
static __global__ void __launch_bounds__(1024)
k_adj_sum(const StepConst K, const double *__restrict__ v, double *out)
{
    __shared__ double part[1024];
    const Grid &G = K.G;
    double acc = 0.0;
    for (long long t = threadIdx.x; t < G.N; t += blockDim.x) {
        int i, j, k;
        interior_coords(G, t, i, j, k);
        acc += v[cell_at(G, i, j, k)];
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = part[0];
}

// ------------------------------------------------------------ kernels

// adjoint of the last recovery (calE fixed): lamP^N -> lamU^N
template <bool FLAT>
__global__ void __launch_bounds__(128)
k_adj_final(const StepConst K, const double *__restrict__ U, const double *__restrict__ P,
            const double *__restrict__ met, const double *__restrict__ lamPin, double *lamU,
            int *bad)
{
    const Grid &G = K.G;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= G.N) return;
    int i, j, k;
    interior_coords(G, t, i, j, k);
    const long long c = cell_at(G, i, j, k), S = G.S;
    Met<double> m;
    load_metric<FLAT>(met, S, c, m);
    double u[NCO], pr[NPR], lp[NPR], lu[NCO], lce[3] = {0, 0, 0};
    for (int f = 0; f < NCO; f++) {
        u[f] = U[f * S + c];
        lu[f] = 0.0;
    }
    for (int f = 0; f < NPR; f++) {
        pr[f] = P[f * S + c];
        lp[f] = lamPin[f * S + c];
    }
    rec_adjoint<FLAT>(K, m, false, 0.0, u, pr, lp, lce, lu, bad);
    for (int f = 0; f < NCO; f++) lamU[f * S + c] = lu[f];
}

// adjoint of the cell sources: lamP = scale (dS/dP)^T lamR (initialises lamP)
template <bool FLAT>
__global__ void __launch_bounds__(128)
k_adj_sources(const StepConst K, const double *__restrict__ P, const double *__restrict__ met,
              const double *__restrict__ lamR, double scale, double *lamP)
{
    const Grid &G = K.G;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= G.N) return;
    int i, j, k;
    interior_coords(G, t, i, j, k);
    const long long c = cell_at(G, i, j, k), S = G.S;
    double lr[NCO];
    for (int f = 0; f < NCO; f++) lr[f] = scale * lamR[f * S + c];
    constexpr int ND = 7;
    for (int g = 0; g < NPR; g += ND) {
        Dual<ND> pr[NPR], Sv[NCO];
        for (int f = 0; f < NPR; f++) pr[f] = Dual<ND>(P[f * S + c]);
        for (int q = 0; q < ND; q++) pr[g + q].d[q] = 1.0;
        if (FLAT)
            sources<true, Dual<ND>>(K, pr, met, c, Sv);
        else
            sources_curved<Dual<ND>>(K, pr, met, c, Sv);
        for (int q = 0; q < ND; q++) {
            double s = 0.0;
            for (int f = 0; f < NCO; f++) s += lr[f] * Sv[f].d[q];
            lamP[(g + q) * S + c] = s;
        }
    }
}

// Gradient of the WENO5 face value (Jiang-Shu weights, as reconstruct
// forms it) with respect to its five stencil values:
//   u = sum_k w_k q_k / sum_k w_k,  w_k = d_k / (eps + beta_k)^2,
//   du/ds = sum_k [omega_k dq_k/ds - 2 omega_k (q_k - u)/(eps + beta_k) dbeta_k/ds].
__device__ __forceinline__ void weno5_grad(double a, double b, double c, double d, double e,
                                           double g[5])
{
    const double eps = 1e-6, sixth = 1.0 / 6.0, k13 = 13.0 / 12.0;
    const double q0 = (2.0 * a - 7.0 * b + 11.0 * c) * sixth;
    const double q1 = (-b + 5.0 * c + 2.0 * d) * sixth;
    const double q2 = (2.0 * c + 5.0 * d - e) * sixth;
    const double t10 = a - 2.0 * b + c, t20 = a - 4.0 * b + 3.0 * c;
    const double t11 = b - 2.0 * c + d, t21 = b - d;
    const double t12 = c - 2.0 * d + e, t22 = 3.0 * c - 4.0 * d + e;
    const double b0 = k13 * t10 * t10 + 0.25 * t20 * t20;
    const double b1 = k13 * t11 * t11 + 0.25 * t21 * t21;
    const double b2 = k13 * t12 * t12 + 0.25 * t22 * t22;
    // the three 1/(eps + beta_k) from one division
    const double e0 = eps + b0, e1 = eps + b1, e2 = eps + b2;
    const double r = 1.0 / (e0 * e1 * e2);   // e_k >= eps: no underflow
    double i0 = r * (e1 * e2), i1 = r * (e0 * e2), i2 = r * (e0 * e1);
    if (!(r > 0.0)) {   // the product overflowed (extreme stencils)
        i0 = 1.0 / e0;
        i1 = 1.0 / e1;
        i2 = 1.0 / e2;
    }
    const double w0 = 0.1 * i0 * i0, w1 = 0.6 * i1 * i1, w2 = 0.3 * i2 * i2;
    const double iW = 1.0 / (w0 + w1 + w2);
    const double o0 = w0 * iW, o1 = w1 * iW, o2 = w2 * iW;
    const double u = o0 * q0 + o1 * q1 + o2 * q2;
    const double c0 = -2.0 * o0 * (q0 - u) * i0;
    const double c1 = -2.0 * o1 * (q1 - u) * i1;
    const double c2 = -2.0 * o2 * (q2 - u) * i2;
    // dbeta_k / d(its three points), times c_k
    const double p0 = 2.0 * k13 * t10 * c0, r0 = 0.5 * t20 * c0;
    const double p1 = 2.0 * k13 * t11 * c1, r1 = 0.5 * t21 * c1;
    const double p2 = 2.0 * k13 * t12 * c2, r2 = 0.5 * t22 * c2;
    g[0] = o0 * 2.0 * sixth + p0 + r0;
    g[1] = -o0 * 7.0 * sixth - o1 * sixth - 2.0 * p0 - 4.0 * r0 + p1 + r1;
    g[2] = o0 * 11.0 * sixth + o1 * 5.0 * sixth + o2 * 2.0 * sixth + p0 + 3.0 * r0 - 2.0 * p1 +
           p2 + 3.0 * r2;
    g[3] = o1 * 2.0 * sixth + o2 * 5.0 * sixth + p1 - r1 - 2.0 * p2 - 4.0 * r2;
    g[4] = -o2 * sixth + p2 + r2;
}

// gradient of the TVD slope of (um, u0, up): the selected candidate's
template <int RC>
__device__ __forceinline__ void tvd_slope_grad(double um, double u0, double up, double g[3])
{
    g[0] = g[1] = g[2] = 0.0;
    if (RC == RC_MINMOD) {
        const double x = u0 - um, y = up - u0;
        if (x * y <= 0.0) return;
        if (fabs(x) <= fabs(y)) { g[0] = -1.0; g[1] = 1.0; }
        else { g[1] = -1.0; g[2] = 1.0; }
        return;
    }
    const double a = 2.0 * (u0 - um), b = 0.5 * (up - um), c = 2.0 * (up - u0);
    int pick = -1;   // the argument mm3 returns: fmin(a, fmin(b, c)) or fmax(...)
    if (a > 0.0 && b > 0.0 && c > 0.0) {
        const int bc = c < b ? 2 : 1;
        const double vbc = bc == 2 ? c : b;
        pick = vbc < a ? bc : 0;
    } else if (a < 0.0 && b < 0.0 && c < 0.0) {
        const int bc = c > b ? 2 : 1;
        const double vbc = bc == 2 ? c : b;
        pick = vbc > a ? bc : 0;
    }
    if (pick == 0) { g[0] = -2.0; g[1] = 2.0; }
    if (pick == 1) { g[0] = -0.5; g[2] = 0.5; }
    if (pick == 2) { g[1] = -2.0; g[2] = 2.0; }
}

// d uL / d s[0..5] and d uR / d s[0..5] of reconstruct<double, RC>
template <int RC>
__device__ __forceinline__ void recon_grad(const double s[6], double dL[6], double dR[6])
{
    for (int o = 0; o < 6; o++) dL[o] = dR[o] = 0.0;
    if (RC == RC_WENO5) {
        double g[5];
        weno5_grad(s[0], s[1], s[2], s[3], s[4], g);
        for (int k = 0; k < 5; k++) dL[k] = g[k];
        weno5_grad(s[5], s[4], s[3], s[2], s[1], g);
        for (int k = 0; k < 5; k++) dR[5 - k] = g[k];
    } else {
        double g[3];
        tvd_slope_grad<RC>(s[1], s[2], s[3], g);
        dL[1] = 0.5 * g[0];
        dL[2] = 1.0 + 0.5 * g[1];
        dL[3] = 0.5 * g[2];
        tvd_slope_grad<RC>(s[2], s[3], s[4], g);
        dR[2] = -0.5 * g[0];
        dR[3] = 1.0 - 0.5 * g[1];
        dR[4] = -0.5 * g[2];
    }
}

// One side of a face, reverse mode written out from flux_accumulate:
// lam_k = d/dpr_k of sum_f lf_f (cF F_f + cU U_f) at the state pr (14
// primitives, then the charge-flux current J^D in slot 14).
template <bool FLAT, int D>
__device__ __forceinline__ void side_vjp(const double pr[NPR + 1], const Met<double> &m,
                                         double gfac, double cF, double cU, const double lf[NCO],
                                         double lam[NPR + 1])
{
    const double sg = FLAT ? 1.0 : m.sg, a = FLAT ? 1.0 : m.alpha;
    const double bD = FLAT ? 0.0 : m.beta[D];
    double wF[NCO], wU[NCO];
#pragma unroll
    for (int f = 0; f < NCO; f++) {
        wF[f] = lf[f] * cF;
        wU[f] = lf[f] * cU;
    }
    // forward values
    const double v[3] = {pr[PR_VX], pr[PR_VY], pr[PR_VZ]};
    const double E[3] = {pr[PR_EX], pr[PR_EY], pr[PR_EZ]};
    const double B[3] = {pr[PR_BX], pr[PR_BY], pr[PR_BZ]};
    double vl[3], El[3], Bl[3];
    lower<double, FLAT>(m, v, vl);
    lower<double, FLAT>(m, E, El);
    lower<double, FLAT>(m, B, Bl);
    const double rho = pr[PR_RHO];
    const double v2 = dot3(v, vl);
    const double W = rsqrt(1.0 - v2);   // as the FP64 forward forms it
    const double h = rho + gfac * pr[PR_P];
    const double hW2 = h * W * W;
    const double Dc = sg * rho * W;
    // adjoints of the intermediates
    const double lTau = wU[CO_TAU] - bD * wF[CO_TAU];
    double lS[3], lst[3], lv[3] = {0, 0, 0}, lvl[3], lE[3], lEl[3], lB[3], lBl[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const double gDi = FLAT ? (i == D ? 1.0 : 0.0) : m.gi[sym(D, i)];
        lS[i] = wU[CO_SX + i] - bD * wF[CO_SX + i] + wF[CO_TAU] * a * gDi;   // S, S^D
        lst[i] = wF[CO_SX + i] * a * sg;                                     // stress row
        lvl[i] = lEl[i] = lBl[i] = 0.0;
    }
    double lDc = wF[CO_D] * (a * v[D] - bD) + wU[CO_D] - wF[CO_TAU] * a * v[D] - lTau;
    lv[D] += (wF[CO_D] - wF[CO_TAU]) * a * Dc;
    double lhW2 = 0.0, lp = 0.0, lem = 0.0;
    lE[0] = lE[1] = lE[2] = lB[0] = lB[1] = lB[2] = 0.0;
    // st_i = hW2 v^D v_i - E^D E_i - B^D B_i + delta_iD (p + em)
#pragma unroll
    for (int i = 0; i < 3; i++) {
        lhW2 += lst[i] * v[D] * vl[i];
        lv[D] += lst[i] * hW2 * vl[i];
        lvl[i] += lst[i] * hW2 * v[D];
        lE[D] -= lst[i] * El[i];
        lEl[i] -= lst[i] * E[D];
        lB[D] -= lst[i] * Bl[i];
        lBl[i] -= lst[i] * B[D];
    }
    lp += lst[D];
    lem += lst[D];
    // S_i = sg (hW2 v_i + sg (E x B)_i)
    double lExB[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        lhW2 += lS[i] * sg * vl[i];
        lvl[i] += lS[i] * sg * hW2;
        lExB[i] = lS[i] * sg * sg;
    }
    // tau = sg (hW2 - p + em) - D
    lhW2 += lTau * sg;
    lp -= lTau * sg;
    lem += lTau * sg;
    // E x B
    {
        double t[3];
        cross3(B, lExB, t);
        for (int i = 0; i < 3; i++) lE[i] += t[i];
        cross3(lExB, E, t);
        for (int i = 0; i < 3; i++) lB[i] += t[i];
    }
    // calB^i, calE^i rows and the cleaning potentials
    double lPhi = wU[CO_PHI] - bD * wF[CO_PHI], lPsi = wU[CO_PSI] - bD * wF[CO_PSI];
    double leE[3], leB[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const double gid = FLAT ? (i == D ? 1.0 : 0.0) : m.gi[sym(i, D)];
        leE[i] = wF[CO_BX + i] * a;
        lPhi += wF[CO_BX + i] * a * gid;
        leB[i] = -wF[CO_EX + i] * a;
        lPsi += wF[CO_EX + i] * a * gid;
        lB[i] += (wU[CO_BX + i] - bD * wF[CO_BX + i]) * sg;
        lE[i] += (wU[CO_EX + i] - bD * wF[CO_EX + i]) * sg;
    }
    if (D == 0) {
        lEl[2] -= leE[1]; lEl[1] += leE[2]; lBl[2] -= leB[1]; lBl[1] += leB[2];
    } else if (D == 1) {
        lEl[2] += leE[0]; lEl[0] -= leE[2]; lBl[2] += leB[0]; lBl[0] -= leB[2];
    } else {
        lEl[1] -= leE[0]; lEl[0] += leE[1]; lBl[1] -= leB[0]; lBl[0] += leB[1];
    }
    lB[D] += wF[CO_PHI] * a * sg;
    lE[D] += wF[CO_PSI] * a * sg;
    // em = (E.E_lower + B.B_lower)/2
#pragma unroll
    for (int i = 0; i < 3; i++) {
        lE[i] += lem * El[i];
        lB[i] += lem * Bl[i];
    }
    // hW2 = h W^2, h = rho + gfac p, Dc = sg rho W, W = (1 - v.v_lower)^(-1/2)
    const double lh = lhW2 * W * W;
    const double lW = lhW2 * 2.0 * h * W + lDc * sg * rho;
    const double lv2 = lW * 0.5 * W * W * W;
    lam[PR_RHO] = lh + lDc * sg * W;
    lam[PR_P] = lp + lh * gfac;
    double t[3];
    lower<double, FLAT>(m, lvl, t);
#pragma unroll
    for (int i = 0; i < 3; i++) lam[PR_VX + i] = lv[i] + 2.0 * lv2 * vl[i] + t[i];
    lower<double, FLAT>(m, lEl, t);
#pragma unroll
    for (int i = 0; i < 3; i++) lam[PR_EX + i] = lE[i] + t[i];
    lower<double, FLAT>(m, lBl, t);
#pragma unroll
    for (int i = 0; i < 3; i++) lam[PR_BX + i] = lB[i] + t[i];
    lam[PR_PSI] = lPsi * sg;
    lam[PR_PHI] = lPhi * sg;
    const double lQc = wU[CO_Q] - bD * wF[CO_Q];
    lam[PR_Q] = lQc * sg;
    lam[NPR] = wF[CO_Q] * a;   // J^D
}

// Adjoint of the face fluxes of direction D (stage current in the charge
// flux): lambda_face = scale (lamR(cR) - lamR(cL))/dx_D from the flux
// difference, then through HLLE, the face physics of each side and the
// reconstruction (or the first-order fallback).  The contribution of the
// face to each of its six stencil cells (field f, slot o = cell iD - 3 + o)
// is stored at C[(o * 15 + f) S + face]; k_adj_gather sums them per cell.
enum { ADJ_NF = NPR + 1, ADJ_SLOTS = 6 };

template <bool FLAT, int RC, int D>
__global__ void __launch_bounds__(128)
k_adj_flux(const StepConst K, const double *__restrict__ P, const double *__restrict__ Jc,
           const double *__restrict__ met, const double *__restrict__ lamR, double scale,
           double *C)
{
    const Grid &G = K.G;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    int m0 = G.n[0] + (D == 0), m1 = G.n[1] + (D == 1);
    long long nf = (long long)m0 * m1 * (G.n[2] + (D == 2));
    if (t >= nf) return;
    const unsigned u = (unsigned)t, r = u / (unsigned)m0;
    int i = (int)(u - r * (unsigned)m0);
    int k = (int)(r / (unsigned)m1);
    int j = (int)(r - (unsigned)k * (unsigned)m1);
    const long long cR = cell_at(G, i, j, k);
    const long long s = dstride(G, D);
    const long long cL = cR - s;
    const long long S = G.S;

    double lf[NCO];
    bool any = false;
    const double w = scale * G.idx[D];
#pragma unroll
    for (int f = 0; f < NCO; f++) {
        lf[f] = w * (lamR[f * S + cR] - lamR[f * S + cL]);
        any = any || lf[f] != 0.0;
    }
    if (!any) {
        for (int q = 0; q < ADJ_SLOTS * ADJ_NF; q++) C[q * S + cR] = 0.0;
        return;
    }

    // primal face states (as the flux kernel forms them)
    double pL[NPR + 1], pR[NPR + 1];
#pragma unroll 1
    for (int f = 0; f <= NPR; f++) {
        const double *q = (f < NPR ? P + f * S : Jc + D * S) + cL;
        double st[6];
        for (int o = 0; o < 6; o++)
            st[o] = (RC == RC_WENO5 || (o > 0 && o < 5)) ? q[(o - 2) * s] : 0.0;
        reconstruct<double, RC>(st, pL[f], pR[f]);
    }
    Met<double> m;
    if (FLAT) {
        load_metric<true>(met, S, cR, m);
    } else {
        m.alpha = 0.5 * (met[M_ALPHA * S + cL] + met[M_ALPHA * S + cR]);
        for (int a = 0; a < 3; a++)
            m.beta[a] = 0.5 * (met[(M_BETA + a) * S + cL] + met[(M_BETA + a) * S + cR]);
        for (int a = 0; a < 6; a++)
            m.g[a] = 0.5 * (met[(M_GAMMA + a) * S + cL] + met[(M_GAMMA + a) * S + cR]);
        met_complete(m);
    }
    bool fb[2];
#pragma unroll
    for (int sd = 0; sd < 2; sd++) {
        double *q = sd == 0 ? pL : pR;
        double v[3] = {q[PR_VX], q[PR_VY], q[PR_VZ]}, vl[3];
        lower<double, FLAT>(m, v, vl);
        fb[sd] = !(q[PR_RHO] > 0.0) || !(q[PR_P] > 0.0) || !(dot3(v, vl) < 1.0);
        if (fb[sd]) {
            const long long cc = sd == 0 ? cL : cR;
            for (int f = 0; f < NPR; f++) q[f] = P[f * S + cc];
            q[NPR] = Jc[D * S + cc];
        }
    }
    double cFL, cFR, cUU;
    if (FLAT) {
        cFL = 0.5; cFR = 0.5; cUU = -0.5;
    } else {
        const double sq = sqrt(m.gi[sym(D, D)]);
        const double bs = m.beta[D] / m.alpha;
        double ap = sq - bs, am = -sq - bs;
        ap = ap > 0.0 ? ap : 0.0;
        am = am < 0.0 ? am : 0.0;
        const double inv = 1.0 / (ap - am);
        cFL = ap * inv; cFR = -am * inv; cUU = ap * am * inv;
    }
    double lamL[NPR + 1], lamRr[NPR + 1];
    side_vjp<FLAT, D>(pL, m, K.gfac, cFL, -cUU, lf, lamL);
    side_vjp<FLAT, D>(pR, m, K.gfac, cFR, cUU, lf, lamRr);

    // through the reconstruction to the six stencil cells
#pragma unroll 1
    for (int f = 0; f <= NPR; f++) {
        const double *q = (f < NPR ? P + f * S : Jc + D * S) + cL;
        double st[6], dL[6], dR[6], g[6];
        for (int o = 0; o < 6; o++)
            st[o] = (RC == RC_WENO5 || (o > 0 && o < 5)) ? q[(o - 2) * s] : 0.0;
        recon_grad<RC>(st, dL, dR);
        for (int o = 0; o < 6; o++)
            g[o] = (fb[0] ? 0.0 : lamL[f] * dL[o]) + (fb[1] ? 0.0 : lamRr[f] * dR[o]);
        if (fb[0]) g[2] += lamL[f];    // first order: the cell below the face
        if (fb[1]) g[3] += lamRr[f];   // the cell above
        for (int o = 0; o < 6; o++) C[(o * ADJ_NF + f) * S + cR] = g[o];
    }
}

// Sum of the stencil contributions of direction D's faces into every
// interior cell, in a fixed order: lamP (14 fields) and lamJ[D] +=.  A ghost
// position counts for the interior cell the boundary condition copies into
// it (periodic wrap; outflow: the boundary cell).
template <int D>
__global__ void __launch_bounds__(128)
k_adj_gather(const StepConst K, const double *__restrict__ C, double *lamP, double *lamJ)
{
    const Grid &G = K.G;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= G.N) return;
    int i, j, k;
    interior_coords(G, t, i, j, k);
    const long long c = cell_at(G, i, j, k), S = G.S, s = dstride(G, D);
    const int x = D == 0 ? i : (D == 1 ? j : k), n = G.n[D];
    const long long c0 = c - (long long)x * s;
    int img[4], ni = 0;
    img[ni++] = x;
    if (G.bc[D] == 0) {
        if (x - n >= -3) img[ni++] = x - n;
        if (x + n <= n + 2) img[ni++] = x + n;
    } else {
        if (x == 0) { img[ni++] = -1; img[ni++] = -2; img[ni++] = -3; }
        if (x == n - 1) { img[ni++] = n; img[ni++] = n + 1; img[ni++] = n + 2; }
    }
#pragma unroll 1
    for (int f = 0; f < ADJ_NF; f++) {
        double sum = 0.0;
        for (int m = 0; m < ni; m++)
            for (int o = 0; o < ADJ_SLOTS; o++) {
                const int face = img[m] + 3 - o;
                if (face >= 0 && face <= n) sum += C[(o * ADJ_NF + f) * S + c0 + face * s];
            }
        if (f < NPR) lamP[f * S + c] += sum;
        else lamJ[D * S + c] += sum;
    }
}

// Stage 2 and the final combination, per cell.  In: lamU = dL/dU^{n+1},
// lamP2 / lamJ2 from the adjoint of F(P2, J2) (with scale dt/2).  Out: the
// adjoint of F(P1, J1) (lamR1), of Dt R1 (lamdR1), the part of dL/dU^n
// found so far (lamUn), and the cell's dL/dlog sigma0 (added to lsigc[c]).
template <bool FLAT>
__global__ void __launch_bounds__(128)
k_adj_stage2(const StepConst K, const double *__restrict__ Us, const double *__restrict__ P2,
             const double *__restrict__ met, const double *__restrict__ sig,
             const double *__restrict__ lamU, const double *__restrict__ lamP2,
             const double *__restrict__ lamJ2, double *lamR1, double *lamdR1, double *lamUn,
             double *lsigc, int *bad)
{
    const Grid &G = K.G;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < G.N) {
        int i, j, k;
        interior_coords(G, t, i, j, k);
        const long long c = cell_at(G, i, j, k), S = G.S;
        Met<double> m;
        load_metric<FLAT>(met, S, c, m);
        double us[NCO], pr[NPR], lp[NPR], lj[3], ldr[3], lus[NCO];
        for (int f = 0; f < NCO; f++) us[f] = Us[f * S + c];
        for (int f = 0; f < NPR; f++) {
            pr[f] = P2[f * S + c];
            lp[f] = lamP2[f * S + c];
        }
        for (int a = 0; a < 3; a++) {
            lj[a] = lamJ2[a * S + c];
            ldr[a] = 0.5 * lamU[(CO_EX + a) * S + c];   // U^{n+1} holds (dR1 + dR2)/2
        }
        lsigc[c] += stage_adjoint<FLAT>(K, m, sig, c, us, pr, lp, lj, ldr, lus, bad);
        const double dt = K.dt, hdt = 0.5 * dt, a12 = 1.0 - 2.0 * K.gimex;
        for (int f = 0; f < NCO; f++) {
            const double l = lamU[f * S + c];
            lamR1[f * S + c] = hdt * l + dt * lus[f];
            lamUn[f * S + c] = l + lus[f];
        }
        for (int a = 0; a < 3; a++)
            lamdR1[a * S + c] = 0.5 * lamU[(CO_EX + a) * S + c] + a12 * lus[CO_EX + a];
    }
}

// Stage 1, per cell: completes lamUn = dL/dU^n.
template <bool FLAT>
__global__ void __launch_bounds__(128)
k_adj_stage1(const StepConst K, const double *__restrict__ U, const double *__restrict__ P1,
             const double *__restrict__ met, const double *__restrict__ sig,
             const double *__restrict__ lamP1, const double *__restrict__ lamJ1,
             const double *__restrict__ lamdR1, double *lamUn, double *lsigc, int *bad)
{
    const Grid &G = K.G;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < G.N) {
        int i, j, k;
        interior_coords(G, t, i, j, k);
        const long long c = cell_at(G, i, j, k), S = G.S;
        Met<double> m;
        load_metric<FLAT>(met, S, c, m);
        double u[NCO], pr[NPR], lp[NPR], lj[3], ldr[3], lu[NCO];
        for (int f = 0; f < NCO; f++) u[f] = U[f * S + c];
        for (int f = 0; f < NPR; f++) {
            pr[f] = P1[f * S + c];
            lp[f] = lamP1[f * S + c];
        }
        for (int a = 0; a < 3; a++) {
            lj[a] = lamJ1[a * S + c];
            ldr[a] = lamdR1[a * S + c];
        }
        lsigc[c] += stage_adjoint<FLAT>(K, m, sig, c, u, pr, lp, lj, ldr, lu, bad);
        for (int f = 0; f < NCO; f++) lamUn[f * S + c] += lu[f];
    }
}

// cells whose last recovery reset them to the atmosphere: U^{n+1} holds
// fixed D, S_i, tau there, so no derivative flows back through those rows
static __global__ void __launch_bounds__(128)
k_adj_reset_mask(const StepConst K, const double *__restrict__ Pnext, double *lamU)
{
    const Grid &G = K.G;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= G.N) return;
    int i, j, k;
    interior_coords(G, t, i, j, k);
    const long long c = cell_at(G, i, j, k), S = G.S;
    if (!(Pnext[PR_RHO * S + c] < K.ro.atmo_floor)) return;
    lamU[CO_D * S + c] = 0.0;
    lamU[CO_TAU * S + c] = 0.0;
    for (int a = 0; a < 3; a++) lamU[(CO_SX + a) * S + c] = 0.0;
}

// adjoint of U^0 = prim2con(P^0): lamP0 (interior, field-major) = dU/dP^T lamU
template <bool FLAT>
__global__ void __launch_bounds__(128)
k_adj_prim2con(const StepConst K, const double *__restrict__ P, const double *__restrict__ met,
               const double *__restrict__ lamU, double *lamP0)
{
    const Grid &G = K.G;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= G.N) return;
    int i, j, k;
    interior_coords(G, t, i, j, k);
    const long long c = cell_at(G, i, j, k), S = G.S;
    Met<double> m;
    load_metric<FLAT>(met, S, c, m);
    constexpr int ND = 7;
    const Met<Dual<ND>> md = met_cast<Dual<ND>>(m);
    double lu[NCO];
    for (int f = 0; f < NCO; f++) lu[f] = lamU[f * S + c];
    for (int g = 0; g < NPR; g += ND) {
        Dual<ND> pr[NPR], U[NCO];
        for (int f = 0; f < NPR; f++) pr[f] = Dual<ND>(P[f * S + c]);
        for (int q = 0; q < ND; q++) pr[g + q].d[q] = 1.0;
        prim_to_cons<Dual<ND>, FLAT>(pr, md, Dual<ND>(K.gfac), U);
        for (int q = 0; q < ND; q++) {
            double s = 0.0;
            for (int f = 0; f < NCO; f++) s += lu[f] * U[f].d[q];
            lamP0[(g + q) * G.N + t] = s;
        }
    }
}

} // namespace rmhd
