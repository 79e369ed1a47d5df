// kernels.cuh -- grid kernels of one IMEX-SSP2(2,2,2) step (arXiv:2510.18968,
// Sec. III.A Table imex and Eq. IMEX3), FP64 state.
//
// Layout in HBM: every field is a padded structure-of-arrays block with 3
// ghost layers in each active direction (0 in an inactive one), x fastest;
// field f of a buffer starts at f * S.  Conserved U^n, the two primitive
// ping-pong buffers, the stage accumulator V, the stiff increments and the
// per-direction face fluxes all share that layout, so a cell (or the face on
// its low side) has the same offset in every array.
//
// Per step (one thread per cell or face, grid-stride free 1D launches):
//   stage1  U^n, P^n          -> P1 (in place), dR1 = Dt R[U1], J1   (recovery)
//   ghosts  P1, J1
//   flux_d  P1, J1            -> F_d at every face, d = x, y, z      (recon+HLLE)
//   stage2  U^n, P1, F, dR1   -> P2, V = U^n + dt/2 F[U1] + dt/2 (R1 + R2), J2
//   ghosts  P2, J2
//   flux_d  P2, J2            -> F_d
//   final   V, P2, F          -> U^{n+1} = V + dt/2 F[U2], P^{n+1}   (recovery)
//   ghosts  P^{n+1}
#pragma once
#include "physics.cuh"
#include "recovery.cuh"

namespace rmhd {

struct Grid {
    int n[3], g[3];
    int px, pxy;          // padded pitches
    long long S;          // padded cells (field stride)
    long long N;          // interior cells
    double idx[3];        // 1 / dx
    int bc[3];
};

struct StepConst {
    Grid G;
    double dt, gimex;     // dt, gamma of Table imex
    double gfac;          // Gamma / (Gamma - 1)
    double kappa;
    int sigma_model;
    double sigma0, sigma_exp, D_atmo;
    int qflux;            // 0 stage current, 1 Ohm's law at faces
    RecOpts ro;
};

// metric fields: alpha, beta^x..z, gamma_xx..zz, K_xx..zz
enum { M_ALPHA = 0, M_BETA = 1, M_GAMMA = 4, M_K = 10, NMET = 16 };

enum { ST_ITERS = 0, ST_FALLBACK, ST_FAIL, ST_FLOOR, ST_MAXIT, ST_NAN, ST_CALLS, NSTAT };

__device__ __forceinline__ long long cell_at(const Grid &G, int i, int j, int k)
{
    return (long long)(k + G.g[2]) * G.pxy + (long long)(j + G.g[1]) * G.px + (i + G.g[0]);
}

__device__ __forceinline__ long long dstride(const Grid &G, int d)
{
    return d == 0 ? 1LL : (d == 1 ? (long long)G.px : (long long)G.pxy);
}

__device__ __forceinline__ void interior_coords(const Grid &G, long long t, int &i, int &j,
                                                int &k)
{
    i = (int)(t % G.n[0]);
    long long r = t / G.n[0];
    j = (int)(r % G.n[1]);
    k = (int)(r / G.n[1]);
}

template <bool FLAT>
__device__ __forceinline__ void load_metric(const double *__restrict__ met, long long S,
                                            long long c, Met<double> &m)
{
    if (FLAT) {
        m.alpha = 1.0;
        m.beta[0] = m.beta[1] = m.beta[2] = 0.0;
        m.g[0] = m.g[3] = m.g[5] = 1.0;
        m.g[1] = m.g[2] = m.g[4] = 0.0;
        m.gi[0] = m.gi[3] = m.gi[5] = 1.0;
        m.gi[1] = m.gi[2] = m.gi[4] = 0.0;
        m.sg = m.isg = 1.0;
        return;
    }
    m.alpha = met[M_ALPHA * S + c];
    for (int a = 0; a < 3; a++) m.beta[a] = met[(M_BETA + a) * S + c];
    for (int a = 0; a < 6; a++) m.g[a] = met[(M_GAMMA + a) * S + c];
    met_complete(m);
}

// conductivity of a cell from its conserved D (models of Sec. IV)
__device__ __forceinline__ double sigma_cell(const StepConst &K, const double *sig, long long c,
                                             double D)
{
    switch (K.sigma_model) {
    case 1: return K.sigma0 * sig[c];
    case 2: return K.sigma0 * pow(D, K.sigma_exp);
    case 3: {
        double t = 1.0 - K.D_atmo / D;
        t = t > 0.0 ? t : 0.0;
        return K.sigma0 * t * t;
    }
    default: return K.sigma0;
    }
}

// warp-aggregated recovery statistics
__device__ __forceinline__ void record_stats(unsigned long long *st, bool active, int status,
                                             int iters)
{
    const unsigned full = 0xffffffffu;
    unsigned it = active ? (unsigned)iters : 0u;
    unsigned fb = active && (status == 1 || status == 4);
    unsigned fl = active && status == 2, fr = active && status == 3;
    unsigned ca = active ? 1u : 0u;
    unsigned s_it = __reduce_add_sync(full, it);
    unsigned s_fb = __reduce_add_sync(full, fb);
    unsigned s_fl = __reduce_add_sync(full, fl);
    unsigned s_fr = __reduce_add_sync(full, fr);
    unsigned s_ca = __reduce_add_sync(full, ca);
    unsigned m_it = __reduce_max_sync(full, it);
    if ((threadIdx.x & 31) == 0) {
        if (s_it) atomicAdd(&st[ST_ITERS], (unsigned long long)s_it);
        if (s_fb) atomicAdd(&st[ST_FALLBACK], (unsigned long long)s_fb);
        if (s_fl) atomicAdd(&st[ST_FAIL], (unsigned long long)s_fl);
        if (s_fr) atomicAdd(&st[ST_FLOOR], (unsigned long long)s_fr);
        if (s_ca) atomicAdd(&st[ST_CALLS], (unsigned long long)s_ca);
        if (m_it) atomicMax(&st[ST_MAXIT], (unsigned long long)m_it);
    }
}

// ---------------------------------------------------------------- set-up

// interior SoA (14 x N) <-> padded SoA (nf x S)
__global__ void k_scatter(const StepConst K, const double *__restrict__ src, double *dst,
                          int nf)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= K.G.N) return;
    int i, j, k;
    interior_coords(K.G, t, i, j, k);
    long long c = cell_at(K.G, i, j, k);
    for (int f = 0; f < nf; f++) dst[f * K.G.S + c] = src[f * K.G.N + t];
}

__global__ void k_gather(const StepConst K, const double *__restrict__ src, double *dst, int nf)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= K.G.N) return;
    int i, j, k;
    interior_coords(K.G, t, i, j, k);
    long long c = cell_at(K.G, i, j, k);
    for (int f = 0; f < nf; f++) dst[f * K.G.N + t] = src[f * K.G.S + c];
}

// Ghost layers of direction blockIdx.y's active dims: periodic wrap or copy of
// the nearest interior cell (Sec. IV: Neumann/outflow).  Only the slabs
// across each face are filled; edge and corner ghosts are never read.
__global__ void k_ghosts(const StepConst K, double *buf, int nf, int d0)
{
    const Grid &G = K.G;
    const int d = d0 + blockIdx.y;
    if (G.g[d] == 0) return;
    const int a = (d + 1) % 3, b = (d + 2) % 3;
    long long per_side = (long long)G.g[d] * G.n[a] * G.n[b];
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= 2 * per_side) return;
    int side = (int)(t / per_side);
    long long r = t % per_side;
    int layer = (int)(r % G.g[d]);
    r /= G.g[d];
    int ca = (int)(r % G.n[a]);
    int cb = (int)(r / G.n[a]);
    int dst_d = side == 0 ? -1 - layer : G.n[d] + layer;
    int src_d;
    if (G.bc[d] == 0)
        src_d = side == 0 ? G.n[d] - 1 - layer : layer;
    else
        src_d = side == 0 ? 0 : G.n[d] - 1;
    int cd[3], cs[3];
    cd[d] = dst_d; cs[d] = src_d;
    cd[a] = cs[a] = ca;
    cd[b] = cs[b] = cb;
    long long dc = cell_at(G, cd[0], cd[1], cd[2]);
    long long sc = cell_at(G, cs[0], cs[1], cs[2]);
    for (int f = 0; f < nf; f++) buf[f * G.S + dc] = buf[f * G.S + sc];
}

// U = prim->con(P) over the interior; flags unphysical input
template <bool FLAT>
__global__ void k_prim2con(const StepConst K, const double *__restrict__ P,
                           const double *__restrict__ met, double *U, int *bad)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= K.G.N) return;
    int i, j, k;
    interior_coords(K.G, t, i, j, k);
    long long c = cell_at(K.G, i, j, k);
    Met<double> m;
    load_metric<FLAT>(met, K.G.S, c, m);
    double pr[NPR], u[NCO];
    bool ok = true;
    for (int f = 0; f < NPR; f++) {
        pr[f] = P[f * K.G.S + c];
        ok = ok && isfinite(pr[f]);
    }
    double v[3] = {pr[PR_VX], pr[PR_VY], pr[PR_VZ]}, vl[3];
    lower<double, FLAT>(m, v, vl);
    ok = ok && pr[PR_RHO] > 0.0 && pr[PR_P] >= 0.0 && dot3(v, vl) < 1.0;
    if (!ok) {
        atomicOr(bad, 1);
        return;
    }
    prim_to_cons<double, FLAT>(pr, m, K.gfac, u);
    for (int f = 0; f < NCO; f++) U[f * K.G.S + c] = u[f];
}

// metric sanity: alpha > 0, gamma_ij positive definite (leading minors)
__global__ void k_check_metric(const StepConst K, const double *__restrict__ met, int *bad)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= K.G.N) return;
    int i, j, k;
    interior_coords(K.G, t, i, j, k);
    long long c = cell_at(K.G, i, j, k);
    double g[6];
    for (int a = 0; a < 6; a++) g[a] = met[(M_GAMMA + a) * K.G.S + c];
    double m1 = g[0], m2 = g[0] * g[3] - g[1] * g[1];
    double det = g[0] * (g[3] * g[5] - g[4] * g[4]) - g[1] * (g[1] * g[5] - g[4] * g[2]) +
                 g[2] * (g[1] * g[4] - g[3] * g[2]);
    double al = met[M_ALPHA * K.G.S + c];
    bool ok = al > 0.0 && m1 > 0.0 && m2 > 0.0 && det > 0.0 && isfinite(det);
    for (int a = 0; a < NMET; a++) ok = ok && isfinite(met[a * K.G.S + c]);
    if (!ok) atomicOr(bad, 1);
}

__global__ void k_check_finite(long long n, const double *__restrict__ a, int *bad)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < n && !isfinite(a[t])) atomicOr(bad, 1);
}

// ---------------------------------------------------------------- stencil

// Face flux in direction D for the face on the low side of cell (i,j,k)
// (between cells i-1 and i along D): reconstruct the 14 primitives (and the
// stage current J^D when K.qflux == 0), fall back to first order on an
// unphysical side, mean face metric and conductivity, HLLE (Sec. III).
template <class T, bool FLAT, int RC, int D>
__global__ void __launch_bounds__(128) k_flux(const StepConst K, const double *__restrict__ P,
                                              const double *__restrict__ Jc,
                                              const double *__restrict__ met,
                                              const double *__restrict__ sig, double *F)
{
    const Grid &G = K.G;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    int m0 = G.n[0] + (D == 0), m1 = G.n[1] + (D == 1);
    long long nf = (long long)m0 * m1 * (G.n[2] + (D == 2));
    if (t >= nf) return;
    int i = (int)(t % m0);
    long long r = t / m0;
    int j = (int)(r % m1);
    int k = (int)(r / m1);
    const long long cR = cell_at(G, i, j, k);
    const long long s = dstride(G, D);
    const long long cL = cR - s;
    const long long S = G.S;

    T pL[NPR], pR[NPR];
#pragma unroll
    for (int f = 0; f < NPR; f++) {
        const double *q = P + f * S + cL;
        T st[6];
        if (RC == RC_WENO5) {
#pragma unroll
            for (int o = 0; o < 6; o++) st[o] = (T)q[(o - 2) * s];
        } else {
#pragma unroll
            for (int o = 1; o < 5; o++) st[o] = (T)q[(o - 2) * s];
            st[0] = st[5] = T(0);
        }
        reconstruct<T, RC>(st, pL[f], pR[f]);
    }
    T JL = T(0), JR = T(0);
    const bool useJ = K.qflux == 0;
    if (useJ) {
        const double *q = Jc + D * S + cL;
        T st[6];
        if (RC == RC_WENO5) {
#pragma unroll
            for (int o = 0; o < 6; o++) st[o] = (T)q[(o - 2) * s];
        } else {
#pragma unroll
            for (int o = 1; o < 5; o++) st[o] = (T)q[(o - 2) * s];
            st[0] = st[5] = T(0);
        }
        reconstruct<T, RC>(st, JL, JR);
    }
    // face metric: mean of the two cells
    Met<T> m;
    if (FLAT) {
        m.alpha = T(1);
        m.beta[0] = m.beta[1] = m.beta[2] = T(0);
        m.g[0] = m.g[3] = m.g[5] = T(1);
        m.g[1] = m.g[2] = m.g[4] = T(0);
        m.gi[0] = m.gi[3] = m.gi[5] = T(1);
        m.gi[1] = m.gi[2] = m.gi[4] = T(0);
        m.sg = m.isg = T(1);
    } else {
        m.alpha = (T)(0.5 * (met[M_ALPHA * S + cL] + met[M_ALPHA * S + cR]));
        for (int a = 0; a < 3; a++)
            m.beta[a] = (T)(0.5 * (met[(M_BETA + a) * S + cL] + met[(M_BETA + a) * S + cR]));
        for (int a = 0; a < 6; a++)
            m.g[a] = (T)(0.5 * (met[(M_GAMMA + a) * S + cL] + met[(M_GAMMA + a) * S + cR]));
        met_complete(m);
    }
    // first-order fallback on an unphysical reconstructed side
#pragma unroll
    for (int sd = 0; sd < 2; sd++) {
        T *q = sd == 0 ? pL : pR;
        T v[3] = {q[PR_VX], q[PR_VY], q[PR_VZ]}, vl[3];
        lower<T, FLAT>(m, v, vl);
        if (!(q[PR_RHO] > T(0)) || !(q[PR_P] > T(0)) || !(dot3(v, vl) < T(1))) {
            const long long cc = sd == 0 ? cL : cR;
#pragma unroll
            for (int f = 0; f < NPR; f++) q[f] = (T)P[f * S + cc];
            if (useJ) {
                if (sd == 0) JL = (T)Jc[D * S + cc];
                else JR = (T)Jc[D * S + cc];
            }
        }
    }
    T sigma = (T)K.sigma0;
    if (K.sigma_model == 1) {
        sigma = (T)(K.sigma0 * 0.5 * (sig[cL] + sig[cR]));
    } else if (K.sigma_model >= 2) {
        // D of each cell from its primitives
        double sgm = 0.0;
        for (int sd = 0; sd < 2; sd++) {
            const long long cc = sd == 0 ? cL : cR;
            Met<double> mc;
            load_metric<FLAT>(met, S, cc, mc);
            double v[3] = {P[PR_VX * S + cc], P[PR_VY * S + cc], P[PR_VZ * S + cc]}, vl[3];
            lower<double, FLAT>(mc, v, vl);
            double Dc = mc.sg * P[PR_RHO * S + cc] / sqrt(1.0 - dot3(v, vl));
            sgm += 0.5 * sigma_cell(K, sig, cc, Dc);
        }
        sigma = (T)sgm;
    }
    // HLLE: F = cL F_L + cR F_R + cU (U_R - U_L)
    T cFL, cFR, cUU;
    if (FLAT) {
        cFL = T(0.5); cFR = T(0.5); cUU = T(-0.5);
    } else {
        const T sq = sqrt(m.gi[sym(D, D)]);
        const T bs = m.beta[D] / m.alpha;
        T ap = sq - bs, am = -sq - bs;
        ap = ap > T(0) ? ap : T(0);
        am = am < T(0) ? am : T(0);
        const T inv = T(1) / (ap - am);
        cFL = ap * inv; cFR = -am * inv; cUU = ap * am * inv;
    }
    const T gfac = (T)K.gfac;
    T acc[NCO];
#pragma unroll
    for (int f = 0; f < NCO; f++) acc[f] = T(0);
    flux_accumulate<T, FLAT, D>(pL, m, sigma, gfac, useJ, JL, cFL, -cUU, acc);
    flux_accumulate<T, FLAT, D>(pR, m, sigma, gfac, useJ, JR, cFR, cUU, acc);
#pragma unroll
    for (int f = 0; f < NCO; f++) F[f * S + cR] = (double)acc[f];
}

// Source vector of Eq. GRRMHD_flux_form without the stiff part of -alpha J
// (Sec. III.A split), at a cell with primitives pr.  Metric derivatives:
// second-order central differences of the cell-centred metric.
template <bool FLAT>
__device__ __forceinline__ void sources(const StepConst &K, const double pr[NPR],
                                        const double *__restrict__ met, long long c,
                                        double Sv[NCO])
{
    const double kap = K.kappa;
    if (FLAT) {
        // only -Q v^i (E), -kappa Phi, Q - kappa Psi survive in flat space
        for (int f = 0; f < NCO; f++) Sv[f] = 0.0;
        const double Q = pr[PR_Q];
        for (int a = 0; a < 3; a++) Sv[CO_EX + a] = -Q * pr[PR_VX + a];
        Sv[CO_PHI] = -kap * pr[PR_PHI];
        Sv[CO_PSI] = Q - kap * pr[PR_PSI];
        return;
    }
    const Grid &G = K.G;
    const long long S = G.S;
    Met<double> m;
    load_metric<false>(met, S, c, m);
    double U[NCO];
    prim_to_cons<double, false>(pr, m, K.gfac, U);
    double da[3], db[3][3], dg[3][6];
    for (int d = 0; d < 3; d++) {
        if (G.g[d] == 0) {
            da[d] = 0.0;
            for (int a = 0; a < 3; a++) db[d][a] = 0.0;
            for (int a = 0; a < 6; a++) dg[d][a] = 0.0;
            continue;
        }
        const long long s = dstride(G, d);
        const double h = 0.5 * G.idx[d];
        da[d] = (met[M_ALPHA * S + c + s] - met[M_ALPHA * S + c - s]) * h;
        for (int a = 0; a < 3; a++)
            db[d][a] = (met[(M_BETA + a) * S + c + s] - met[(M_BETA + a) * S + c - s]) * h;
        for (int a = 0; a < 6; a++)
            dg[d][a] = (met[(M_GAMMA + a) * S + c + s] - met[(M_GAMMA + a) * S + c - s]) * h;
    }
    double Kij[6];
    for (int a = 0; a < 6; a++) Kij[a] = met[(M_K + a) * S + c];
    const double *gi = m.gi;
    const double Ktr = gi[0] * Kij[0] + gi[3] * Kij[3] + gi[5] * Kij[5] +
                       2.0 * (gi[1] * Kij[1] + gi[2] * Kij[2] + gi[4] * Kij[4]);
    // w_l = 1/2 gamma^{bc} (2 d_b gamma_lc - d_l gamma_bc); gamma^{bc} Gamma^a_bc = gamma^{al} w_l
    double w[3];
    for (int l = 0; l < 3; l++) {
        double s = 0.0;
        for (int b = 0; b < 3; b++)
            for (int cc = 0; cc < 3; cc++)
                s += gi[sym(b, cc)] * (2.0 * dg[b][sym(l, cc)] - dg[l][sym(b, cc)]);
        w[l] = 0.5 * s;
    }
    double v[3] = {pr[PR_VX], pr[PR_VY], pr[PR_VZ]};
    double E[3] = {pr[PR_EX], pr[PR_EY], pr[PR_EZ]};
    double B[3] = {pr[PR_BX], pr[PR_BY], pr[PR_BZ]};
    double vl[3], El[3], Bl[3];
    lower<double, false>(m, v, vl);
    lower<double, false>(m, E, El);
    lower<double, false>(m, B, Bl);
    const double W2 = 1.0 / (1.0 - dot3(v, vl));
    const double hW2 = (pr[PR_RHO] + K.gfac * pr[PR_P]) * W2;
    const double pem = pr[PR_P] + 0.5 * (dot3(E, El) + dot3(B, Bl));
    double Sup[6];   // undensitised stress, indices up
    for (int a = 0; a < 3; a++)
        for (int b = a; b < 3; b++)
            Sup[sym(a, b)] = hW2 * v[a] * v[b] + gi[sym(a, b)] * pem - E[a] * E[b] - B[a] * B[b];
    const double al = m.alpha, sg = m.sg;
    double Su[3];
    double Sl[3] = {U[CO_SX], U[CO_SY], U[CO_SZ]};
    raise<double, false>(m, Sl, Su);
    for (int a = 0; a < 3; a++) {
        double s = 0.0;
        for (int b = 0; b < 3; b++)
            for (int cc = 0; cc < 3; cc++) s += Sup[sym(b, cc)] * dg[a][sym(b, cc)];
        s *= 0.5 * al * sg;
        for (int b = 0; b < 3; b++) s += Sl[b] * db[a][b];
        s -= (U[CO_TAU] + U[CO_D]) * da[a];
        Sv[CO_SX + a] = s;
    }
    {
        double s = Sup[0] * Kij[0] + Sup[3] * Kij[3] + Sup[5] * Kij[5] +
                   2.0 * (Sup[1] * Kij[1] + Sup[2] * Kij[2] + Sup[4] * Kij[4]);
        s *= al * sg;
        for (int a = 0; a < 3; a++) s -= Su[a] * da[a];
        Sv[CO_TAU] = s;
    }
    for (int a = 0; a < 3; a++) {
        double G1 = gi[sym(a, 0)] * da[0] + gi[sym(a, 1)] * da[1] + gi[sym(a, 2)] * da[2];
        double G2 = gi[sym(a, 0)] * w[0] + gi[sym(a, 1)] * w[1] + gi[sym(a, 2)] * w[2];
        double geo = G1 - al * G2;
        double sB = 0.0, sE = 0.0;
        for (int b = 0; b < 3; b++) {
            sB -= U[CO_BX + b] * db[b][a];
            sE -= U[CO_EX + b] * db[b][a];
        }
        Sv[CO_BX + a] = sB + U[CO_PHI] * geo;
        Sv[CO_EX + a] = sE + U[CO_PSI] * geo - al * U[CO_Q] * v[a];
    }
    double Bda = 0.0, Eda = 0.0;
    for (int b = 0; b < 3; b++) {
        Bda += U[CO_BX + b] * da[b];
        Eda += U[CO_EX + b] * da[b];
    }
    Sv[CO_PHI] = -al * U[CO_PHI] * Ktr + Bda - al * kap * U[CO_PHI];
    Sv[CO_PSI] = -al * U[CO_PSI] * Ktr + Eda + al * U[CO_Q] - al * kap * U[CO_PSI];
    Sv[CO_D] = 0.0;
    Sv[CO_Q] = 0.0;
}

// explicit right-hand side F(U) at an interior cell from the face fluxes
template <bool FLAT>
__device__ __forceinline__ void rhs_cell(const StepConst &K, const double pr[NPR],
                                         const double *__restrict__ met,
                                         const double *__restrict__ Fx,
                                         const double *__restrict__ Fy,
                                         const double *__restrict__ Fz, long long c,
                                         double r[NCO])
{
    sources<FLAT>(K, pr, met, c, r);
    const Grid &G = K.G;
    const double *Fd[3] = {Fx, Fy, Fz};
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if (G.g[d] == 0) continue;
        const long long s = dstride(G, d);
        const double ih = G.idx[d];
        const double *F = Fd[d];
#pragma unroll
        for (int f = 0; f < NCO; f++) r[f] -= (F[f * G.S + c + s] - F[f * G.S + c]) * ih;
    }
}

// ---------------------------------------------------------------- stages

// Stage 1 (purely implicit): recovery of U^n with calE solved, guess P^n.
template <bool FLAT>
__global__ void __launch_bounds__(128)
k_stage1(const StepConst K, const double *__restrict__ U, double *P, double *dR1, double *J1,
         const double *__restrict__ met, const double *__restrict__ sig,
         unsigned long long *stats)
{
    const Grid &G = K.G;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const bool active = t < G.N;
    int status = 0, iters = 0;
    if (active) {
        int i, j, k;
        interior_coords(G, t, i, j, k);
        const long long c = cell_at(G, i, j, k), S = G.S;
        Met<double> m;
        load_metric<FLAT>(met, S, c, m);
        RecIn in;
        in.D = U[CO_D * S + c];
        in.tau = U[CO_TAU * S + c];
        for (int a = 0; a < 3; a++) {
            in.S[a] = U[(CO_SX + a) * S + c];
            in.cB[a] = U[(CO_BX + a) * S + c];
            in.cE0[a] = U[(CO_EX + a) * S + c];
        }
        const double Phi = U[CO_PHI * S + c], Psi = U[CO_PSI * S + c], Q = U[CO_Q * S + c];
        const double sigma = sigma_cell(K, sig, c, in.D);
        const double cc = K.gimex * K.dt * m.alpha * sigma;
        const double gp = P[PR_P * S + c];
        const double gv[3] = {P[PR_VX * S + c], P[PR_VY * S + c], P[PR_VZ * S + c]};
        double pr[NPR], E[3];
        status = recover<FLAT>(in, m, K.ro, true, cc, gp, gv, Phi, Psi, Q, pr, E, iters);
        for (int f = 0; f < NPR; f++) P[f * S + c] = pr[f];
        const double ig = 1.0 / K.gimex;
        const double iad = 1.0 / (m.alpha * K.dt);
        for (int a = 0; a < 3; a++) {
            const double r = (E[a] - in.cE0[a]) * ig;
            dR1[a * S + c] = r;
            // stage current J = Q v - Dt R / (alpha Dt)
            J1[a * S + c] = Q * pr[PR_VX + a] - r * iad;
        }
    }
    record_stats(stats, active, status, iters);
}

// Stage 2: U* = U^n + dt F[U1] + (1-2gamma) Dt R1 on calE; implicit recovery
// (guess P1); V = U^n + dt/2 F[U1] + dt/2 (R1 + R2) (Eq. IMEX3 minus F[U2]).
template <bool FLAT>
__global__ void __launch_bounds__(128)
k_stage2(const StepConst K, const double *__restrict__ U, const double *__restrict__ P1,
         const double *__restrict__ Fx, const double *__restrict__ Fy,
         const double *__restrict__ Fz, const double *__restrict__ dR1,
         const double *__restrict__ met, const double *__restrict__ sig, double *P2,
         double *V, double *J2, unsigned long long *stats)
{
    const Grid &G = K.G;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const bool active = t < G.N;
    int status = 0, iters = 0;
    if (active) {
        int i, j, k;
        interior_coords(G, t, i, j, k);
        const long long c = cell_at(G, i, j, k), S = G.S;
        double pr[NPR];
        for (int f = 0; f < NPR; f++) pr[f] = P1[f * S + c];
        double r[NCO];
        rhs_cell<FLAT>(K, pr, met, Fx, Fy, Fz, c, r);
        const double dt = K.dt, hdt = 0.5 * dt;
        double us[NCO];
        for (int f = 0; f < NCO; f++) {
            const double u = U[f * S + c];
            us[f] = u + dt * r[f];
            V[f * S + c] = u + hdt * r[f];
        }
        double r1[3];
        for (int a = 0; a < 3; a++) {
            r1[a] = dR1[a * S + c];
            us[CO_EX + a] += (1.0 - 2.0 * K.gimex) * r1[a];
        }
        Met<double> m;
        load_metric<FLAT>(met, S, c, m);
        RecIn in;
        in.D = us[CO_D];
        in.tau = us[CO_TAU];
        for (int a = 0; a < 3; a++) {
            in.S[a] = us[CO_SX + a];
            in.cB[a] = us[CO_BX + a];
            in.cE0[a] = us[CO_EX + a];
        }
        const double sigma = sigma_cell(K, sig, c, in.D);
        const double cc = K.gimex * dt * m.alpha * sigma;
        const double gv[3] = {pr[PR_VX], pr[PR_VY], pr[PR_VZ]};
        double p2[NPR], E[3];
        status = recover<FLAT>(in, m, K.ro, true, cc, pr[PR_P], gv, us[CO_PHI], us[CO_PSI],
                               us[CO_Q], p2, E, iters);
        for (int f = 0; f < NPR; f++) P2[f * S + c] = p2[f];
        const double ig = 1.0 / K.gimex;
        const double iad = 1.0 / (m.alpha * dt);
        for (int a = 0; a < 3; a++) {
            const double r2 = (E[a] - in.cE0[a]) * ig;
            V[(CO_EX + a) * S + c] += 0.5 * (r1[a] + r2);
            J2[a * S + c] = us[CO_Q] * p2[PR_VX + a] - r2 * iad;
        }
    }
    record_stats(stats, active, status, iters);
}

// Final: U^{n+1} = V + dt/2 F[U2]; recovery with calE fixed (guess P2).
template <bool FLAT>
__global__ void __launch_bounds__(128)
k_final(const StepConst K, const double *__restrict__ Vb, const double *__restrict__ P2,
        const double *__restrict__ Fx, const double *__restrict__ Fy,
        const double *__restrict__ Fz, const double *__restrict__ met, double *U, double *P,
        unsigned long long *stats)
{
    const Grid &G = K.G;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const bool active = t < G.N;
    int status = 0, iters = 0;
    if (active) {
        int i, j, k;
        interior_coords(G, t, i, j, k);
        const long long c = cell_at(G, i, j, k), S = G.S;
        double pr[NPR];
        for (int f = 0; f < NPR; f++) pr[f] = P2[f * S + c];
        double r[NCO];
        rhs_cell<FLAT>(K, pr, met, Fx, Fy, Fz, c, r);
        const double hdt = 0.5 * K.dt;
        double un[NCO];
        bool finite = true;
        for (int f = 0; f < NCO; f++) {
            un[f] = Vb[f * S + c] + hdt * r[f];
            finite = finite && isfinite(un[f]);
        }
        if (!finite) atomicOr((unsigned long long *)&stats[ST_NAN], 1ULL);
        Met<double> m;
        load_metric<FLAT>(met, S, c, m);
        RecIn in;
        in.D = un[CO_D];
        in.tau = un[CO_TAU];
        for (int a = 0; a < 3; a++) {
            in.S[a] = un[CO_SX + a];
            in.cB[a] = un[CO_BX + a];
            in.cE0[a] = un[CO_EX + a];
        }
        const double gv[3] = {pr[PR_VX], pr[PR_VY], pr[PR_VZ]};
        double pn[NPR], E[3];
        status = recover<FLAT>(in, m, K.ro, false, 0.0, pr[PR_P], gv, un[CO_PHI], un[CO_PSI],
                               un[CO_Q], pn, E, iters);
        if (status == 2 || status == 3) {
            double u2[NCO];
            prim_to_cons<double, FLAT>(pn, m, K.gfac, u2);
            un[CO_D] = u2[CO_D];
            un[CO_TAU] = u2[CO_TAU];
            for (int a = 0; a < 3; a++) un[CO_SX + a] = u2[CO_SX + a];
        }
        for (int f = 0; f < NCO; f++) U[f * S + c] = un[f];
        for (int f = 0; f < NPR; f++) P[f * S + c] = pn[f];
    }
    record_stats(stats, active, status, iters);
}

// explicit right-hand side only (testing entry point)
template <bool FLAT>
__global__ void k_rhs(const StepConst K, const double *__restrict__ P,
                      const double *__restrict__ Fx, const double *__restrict__ Fy,
                      const double *__restrict__ Fz, const double *__restrict__ met,
                      double *out)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= K.G.N) return;
    int i, j, k;
    interior_coords(K.G, t, i, j, k);
    const long long c = cell_at(K.G, i, j, k), S = K.G.S;
    double pr[NPR], r[NCO];
    for (int f = 0; f < NPR; f++) pr[f] = P[f * S + c];
    rhs_cell<FLAT>(K, pr, met, Fx, Fy, Fz, c, r);
    for (int f = 0; f < NCO; f++) out[f * K.G.N + t] = r[f];
}

// pointwise recovery on independent points (testing entry point)
__global__ void __launch_bounds__(128)
k_recover_points(const RecOpts ro, int npts, const double *__restrict__ cons,
                 const double *__restrict__ guess, const double *__restrict__ alpha,
                 const double *__restrict__ gam, const double *__restrict__ sigma, int implicit,
                 double c, double gfac, double *prim, double *cons_out, int *iters, int *status)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npts) return;
    Met<double> m;
    m.alpha = alpha[t];
    m.beta[0] = m.beta[1] = m.beta[2] = 0.0;
    for (int a = 0; a < 6; a++) m.g[a] = gam[a * npts + t];
    met_complete(m);
    RecIn in;
    in.D = cons[CO_D * npts + t];
    in.tau = cons[CO_TAU * npts + t];
    for (int a = 0; a < 3; a++) {
        in.S[a] = cons[(CO_SX + a) * npts + t];
        in.cB[a] = cons[(CO_BX + a) * npts + t];
        in.cE0[a] = cons[(CO_EX + a) * npts + t];
    }
    const double gv[3] = {guess[PR_VX * npts + t], guess[PR_VY * npts + t],
                          guess[PR_VZ * npts + t]};
    double pr[NPR], E[3];
    int it = 0;
    const double cc = implicit ? c * m.alpha * sigma[t] : 0.0;
    int st = recover<false>(in, m, ro, implicit != 0, cc, guess[PR_P * npts + t], gv,
                            cons[CO_PHI * npts + t], cons[CO_PSI * npts + t],
                            cons[CO_Q * npts + t], pr, E, it);
    double u[NCO];
    for (int f = 0; f < NCO; f++) u[f] = cons[f * npts + t];
    for (int a = 0; a < 3; a++) u[CO_EX + a] = E[a];
    if (st == 2 || st == 3) {
        double u2[NCO];
        prim_to_cons<double, false>(pr, m, gfac, u2);
        u[CO_D] = u2[CO_D];
        u[CO_TAU] = u2[CO_TAU];
        for (int a = 0; a < 3; a++) u[CO_SX + a] = u2[CO_SX + a];
    }
    for (int f = 0; f < NPR; f++) prim[f * npts + t] = pr[f];
    for (int f = 0; f < NCO; f++) cons_out[f * npts + t] = u[f];
    iters[t] = it;
    status[t] = st;
}

} // namespace rmhd
