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
// The explicit part (primitives read by the stencil, stage currents, face
// fluxes, right-hand side) is stored and computed in T: double on the FP64
// path, float on the mixed path.  U^n, V, U^{n+1}, the stiff increments and
// the recovery are FP64 on both; the recovery guess (p, v^i) is kept in FP64
// in G (on the FP64 path G aliases fields 1..4 of the primitive buffer).
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
#include "tma.cuh"

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
    double idt, igimex;   // 1/dt, 1/gamma
    double gfac;          // Gamma / (Gamma - 1)
    double kappa;
    int sigma_model;
    double sigma0, sigma_exp, D_atmo;
    int qflux;            // 0 stage current, 1 Ohm's law at faces, 2 Gauss's law
    RecOpts ro;
    float sigma0f, gfacf; // FP32 copies for the FP32 stencil (no FP64 conversions)
    float kappaf, idxf[3];
};

// a constant of StepConst in the stencil's type
template <class T> __device__ __forceinline__ T kc(double d, float f)
{
    if (sizeof(T) == sizeof(float)) return (T)f;
    return (T)d;
}

// metric fields: alpha, beta^x..z, gamma_xx..zz, K_xx..zz
enum { M_ALPHA = 0, M_BETA = 1, M_GAMMA = 4, M_K = 10, NMET = 16 };

// ST_TILE: a stencil tile load did not complete within its wait bound
enum { ST_ITERS = 0, ST_FALLBACK, ST_FAIL, ST_FLOOR, ST_MAXIT, ST_NAN, ST_CALLS, ST_TILE, NSTAT };

__device__ __forceinline__ long long cell_at(const Grid &G, int i, int j, int k)
{
    return (long long)(k + G.g[2]) * G.pxy + (long long)(j + G.g[1]) * G.px + (i + G.g[0]);
}

__device__ __forceinline__ long long dstride(const Grid &G, int d)
{
    return d == 0 ? 1LL : (d == 1 ? (long long)G.px : (long long)G.pxy);
}

// linear interior index -> (i, j, k); 32-bit arithmetic (the library
// rejects grids of 2^31 cells or more), which the GPU divides far faster
// than 64-bit integers
__device__ __forceinline__ void interior_coords(const Grid &G, long long t, int &i, int &j,
                                                int &k)
{
    const unsigned u = (unsigned)t, nx = (unsigned)G.n[0], ny = (unsigned)G.n[1];
    const unsigned r = u / nx;
    i = (int)(u - r * nx);
    k = (int)(r / ny);
    j = (int)(r - (unsigned)k * ny);
}

// Cells of the recovery kernels are handed out in bricks of 32 (4 x 4 x 2,
// or 8 x 4 in 2D, a row in 1D), so that a warp holds neighbouring cells:
// cells that need more recovery iterations cluster in space, and a brick
// mixes fewer of them with one-iteration cells than a 32-cell row does.
struct Bricks {
    int bx, by, bz;       // brick extents (bx * by * bz = 32)
    int nbx, nby;         // bricks along x, y
    long long threads;    // 32 x number of bricks
};

__host__ __device__ inline Bricks make_bricks(const int n[3])
{
    Bricks b;
    int e[3] = {1, 1, 1};
    const int nact = (n[0] > 1) + (n[1] > 1) + (n[2] > 1);
    if (nact == 3) {
        e[0] = 4; e[1] = 4; e[2] = 2;
    } else if (nact == 2) {
        int first = 1;   // the first active axis takes 8, the second 4
        for (int d = 0; d < 3; d++)
            if (n[d] > 1) { e[d] = first ? 8 : 4; first = 0; }
    } else {
        for (int d = 0; d < 3; d++)
            if (n[d] > 1) e[d] = 32;
        if (nact == 0) e[0] = 32;
    }
    b.bx = e[0]; b.by = e[1]; b.bz = e[2];
    b.nbx = (n[0] + b.bx - 1) / b.bx;
    b.nby = (n[1] + b.by - 1) / b.by;
    const long long nbz = (n[2] + b.bz - 1) / b.bz;
    b.threads = 32LL * b.nbx * b.nby * nbz;
    return b;
}

// brick thread t -> interior cell (i, j, k); false if outside the grid
__device__ __forceinline__ bool brick_coords(const Grid &G, const Bricks &b, long long t, int &i,
                                             int &j, int &k)
{
    const unsigned u = (unsigned)t, br = u >> 5, l = u & 31u;
    const unsigned qx = br % (unsigned)b.nbx, r = br / (unsigned)b.nbx;
    const unsigned qy = r % (unsigned)b.nby, qz = r / (unsigned)b.nby;
    const unsigned lx = l % (unsigned)b.bx, ly = (l / (unsigned)b.bx) % (unsigned)b.by;
    const unsigned lz = l / (unsigned)(b.bx * b.by);
    i = (int)(qx * b.bx + lx);
    j = (int)(qy * b.by + ly);
    k = (int)(qz * b.bz + lz);
    return t < b.threads && i < G.n[0] && j < G.n[1] && k < G.n[2];
}

// linear interior index of (i, j, k), x fastest
__device__ __forceinline__ long long interior_index(const Grid &G, int i, int j, int k)
{
    return ((long long)k * G.n[1] + j) * G.n[0] + i;
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
// (call = false: only the iterations of a recovery finished by a later pass)
__device__ __forceinline__ void record_stats(unsigned long long *st, bool active, int status,
                                             int iters, bool call = true)
{
    const unsigned full = 0xffffffffu;
    unsigned it = active ? (unsigned)iters : 0u;
    active = active && call;
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

// interior SoA (nf x N, FP64) <-> padded SoA (nf x S)
template <class T>
__global__ void k_scatter(const StepConst K, const double *__restrict__ src, T *dst, int nf)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= K.G.N) return;
    int i, j, k;
    interior_coords(K.G, t, i, j, k);
    long long c = cell_at(K.G, i, j, k);
    for (int f = 0; f < nf; f++) dst[f * K.G.S + c] = (T)src[f * K.G.N + t];
}

static __global__ void k_gather(const StepConst K, const double *__restrict__ src, double *dst, int nf)
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
template <class T> __global__ void k_ghosts(const StepConst K, T *buf, int nf, int d0)
{
    const Grid &G = K.G;
    const int d = d0 + blockIdx.y;
    if (G.g[d] == 0) return;
    const int a = (d + 1) % 3, b = (d + 2) % 3;
    const unsigned per_side = (unsigned)G.g[d] * G.n[a] * G.n[b];
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * per_side) return;
    const int side = t >= per_side;
    unsigned r = t - (side ? per_side : 0u);
    const int layer = (int)(r % (unsigned)G.g[d]);
    r /= (unsigned)G.g[d];
    const int ca = (int)(r % (unsigned)G.n[a]);
    const int cb = (int)(r / (unsigned)G.n[a]);
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

// Charge from Gauss's law (RMHD_QFLUX_GAUSS, the variant of Sec. IV.E):
// calQ = d_i (sqrt(gamma) E^i) by 2nd-order central differences over the
// stage primitives, whose ghosts hold the boundary condition; q = calQ /
// sqrt(gamma) into P, and calQ into U when U is given (end of the step).
template <bool FLAT, class T>
__global__ void __launch_bounds__(128) k_gauss(const StepConst K, T *P,
                                               const double *__restrict__ met, double *U)
{
    const Grid &G = K.G;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= G.N) return;
    int i, j, k;
    interior_coords(G, t, i, j, k);
    const long long c = cell_at(G, i, j, k);
    const long long stride[3] = {1, G.px, G.pxy};
    double Q = 0.0;
    for (int d = 0; d < 3; d++) {
        if (!G.g[d]) continue;
        const long long cp = c + stride[d], cm = c - stride[d];
        double sp = 1.0, sm = 1.0;
        if (!FLAT) {
            Met<double> mp, mm;
            load_metric<false>(met, G.S, cp, mp);
            load_metric<false>(met, G.S, cm, mm);
            sp = mp.sg;
            sm = mm.sg;
        }
        const double ep = sp * (double)P[(PR_EX + d) * G.S + cp];
        const double em = sm * (double)P[(PR_EX + d) * G.S + cm];
        Q += (ep - em) * (0.5 * G.idx[d]);
    }
    double sg = 1.0;
    if (!FLAT) {
        Met<double> m;
        load_metric<false>(met, G.S, c, m);
        sg = m.sg;
    }
    P[PR_Q * G.S + c] = (T)(Q / sg);
    if (U) U[CO_Q * G.S + c] = Q;
}

// interior FP64 primitives -> padded primitives in T and the FP64 guess G
template <class T>
__global__ void k_scatter_prims(const StepConst K, const double *__restrict__ src, T *P,
                                double *Gs)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= K.G.N) return;
    int i, j, k;
    interior_coords(K.G, t, i, j, k);
    long long c = cell_at(K.G, i, j, k);
    for (int f = 0; f < NPR; f++) P[f * K.G.S + c] = (T)src[f * K.G.N + t];
    for (int f = 0; f < 4; f++) Gs[f * K.G.S + c] = src[(PR_P + f) * K.G.N + t];
}

// padded primitives (T) with p, v^i from G -> interior FP64
template <class T>
__global__ void k_gather_prims(const StepConst K, const T *__restrict__ P,
                               const double *__restrict__ Gs, double *dst)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= K.G.N) return;
    int i, j, k;
    interior_coords(K.G, t, i, j, k);
    long long c = cell_at(K.G, i, j, k);
    for (int f = 0; f < NPR; f++) dst[f * K.G.N + t] = (double)P[f * K.G.S + c];
    for (int f = 0; f < 4; f++) dst[(PR_P + f) * K.G.N + t] = Gs[f * K.G.S + c];
}

// U = prim->con of interior FP64 primitives src; flags unphysical input
template <bool FLAT>
__global__ void k_prim2con(const StepConst K, const double *__restrict__ src,
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
        pr[f] = src[f * K.G.N + t];
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
static __global__ void k_check_metric(const StepConst K, const double *__restrict__ met, int *bad)
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

static __global__ void k_check_finite(long long n, const double *__restrict__ a, int *bad)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < n && !isfinite(a[t])) atomicOr(bad, 1);
}

// ---------------------------------------------------------------- stencil

// Face flux in direction D for the face on the low side of cell (i,j,k)
// (between cells i-1 and i along D): reconstruct the 14 primitives (and the
// stage current J^D unless K.qflux == 1), fall back to first order on an
// unphysical side, mean face metric and conductivity, HLLE (Sec. III).
template <class T, bool FLAT, int RC, int D>
__global__ void __launch_bounds__(128) k_flux(const StepConst K, const T *__restrict__ P,
                                              const T *__restrict__ Jc,
                                              const double *__restrict__ met,
                                              const double *__restrict__ sig, T *F)
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

    T pL[NPR], pR[NPR];
#pragma unroll
    for (int f = 0; f < NPR; f++) {
        const T *q = P + f * S + cL;
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
    const bool useJ = K.qflux != 1;   // mode 2: Q row overwritten later
    if (useJ) {
        const T *q = Jc + D * S + cL;
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
    T sigma = kc<T>(K.sigma0, K.sigma0f);
    if (K.sigma_model == 1) {
        sigma = (T)(K.sigma0 * 0.5 * (sig[cL] + sig[cR]));
    } else if (K.sigma_model >= 2) {
        // D of each cell from its primitives
        double sgm = 0.0;
        for (int sd = 0; sd < 2; sd++) {
            const long long cc = sd == 0 ? cL : cR;
            Met<double> mc;
            load_metric<FLAT>(met, S, cc, mc);
            double v[3] = {(double)P[PR_VX * S + cc], (double)P[PR_VY * S + cc],
                           (double)P[PR_VZ * S + cc]}, vl[3];
            lower<double, FLAT>(mc, v, vl);
            double Dc = mc.sg * (double)P[PR_RHO * S + cc] / sqrt(1.0 - dot3(v, vl));
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
    const T gfac = kc<T>(K.gfac, K.gfacf);
    T acc[NCO];
#pragma unroll
    for (int f = 0; f < NCO; f++) acc[f] = T(0);
    ArrAcc<T> aa{acc};
    flux_accumulate<T, FLAT, D>(pL, m, sigma, gfac, useJ, JL, cFL, -cUU, aa);
    flux_accumulate<T, FLAT, D>(pR, m, sigma, gfac, useJ, JR, cFR, cUU, aa);
#pragma unroll
    for (int f = 0; f < NCO; f++) F[f * S + cR] = acc[f];
}

// Face fluxes of direction D in FP32 with the stencil staged in shared
// memory (the mixed path).  Same arithmetic as k_flux, face for face.
// D = 0: a block takes 128 consecutive faces of one x row (the row's last
// block also its face n) and stages their cells, 128 + 6, of the 15 fields
// (14 primitives, J^D); D = 1, 2: a
// block takes 32 (x) x 16 (along D) faces (the last along D also its face
// n) and stages 32 x 22 cells; every thread computes four or five faces
// along D.  Coalesced loads all in flight at
// once, then the stencil reads come from shared memory.
// With tma != 0 the staged cells arrive by two bulk tensor copies (the 14
// primitive fields, then J^D), completion on an mbarrier: D = 0 the row's
// cells x0-3 .. x0+132 (boxes of 136 starting at the 4-aligned padded x0);
// D > 0 boxes of 36 x 22 cells (x0-3 .. x0+32 by d0-3 .. d0+18).
template <bool FLAT, int RC, int D>
__global__ void __launch_bounds__(128)
k_flux_tile(const StepConst K, const float *__restrict__ P, const float *__restrict__ Jc,
            const double *__restrict__ met, const double *__restrict__ sig, float *F,
            const __grid_constant__ CUtensorMap tmP, const __grid_constant__ CUtensorMap tmJ,
            int tma, unsigned long long *stats)
{
    constexpr int TX = D == 0 ? 128 : 32;   // faces (D = 0) or cells (D > 0) along x
    constexpr int TD = D == 0 ? 1 : 16;     // faces along D (D > 0)
    // D = 0: the row's last block takes 129 faces; rows of 136 (a multiple of
    // 4 floats, as a tile copy needs)
    // D > 0: rows of 36 floats starting 3 cells before x0 (a 4-aligned
    // padded x), cell x0 + t at column t + 3
    constexpr int LX = D == 0 ? TX + 8 : TX + 4;
    constexpr int XO = D == 0 ? 0 : 3;
    constexpr int LD = D == 0 ? 1 : TD + 6;   // D > 0: the last block along D takes 17
    constexpr int NF = NPR + 1;
    constexpr int FSTRIDE = LD * LX;
    constexpr int JOFF = (NPR * FSTRIDE + 31) / 32 * 32;   // J^D block, 128-byte aligned
    __shared__ __align__(128) float sm[JOFF + FSTRIDE];
    __shared__ __align__(8) uint64_t bar;
    auto foff = [&](int f) -> int { return f < NPR ? f * FSTRIDE : JOFF; };
    const Grid &G = K.G;
    const long long S = G.S;
    const long long s = dstride(G, D);
    const bool useJ = K.qflux != 1;   // mode 2: Q row overwritten later
    // tile origin: x0 (faces or cells), d0 (faces along D), fixed coordinates
    int x0, d0, c1, c2;
    int x_end = 0;   // D = 0: faces x0 .. x_end - 1 of the row (the last block also takes face n)
    if (D == 0) {
        x0 = blockIdx.x * TX; d0 = 0; c1 = blockIdx.y; c2 = blockIdx.z;
        x_end = blockIdx.x + 1 == gridDim.x ? G.n[0] + 1 : x0 + TX;
    } else if (D == 1) {
        x0 = blockIdx.x * TX; d0 = blockIdx.y * TD; c1 = 0; c2 = blockIdx.z;
    } else {
        x0 = blockIdx.x * TX; d0 = blockIdx.z * TD; c1 = blockIdx.y; c2 = 0;
    }
    // D > 0: faces d0 .. d_end - 1 along D (the last block also takes face n)
    const int d_end = D == 0 ? 0
                    : ((D == 1 ? blockIdx.y + 1 == gridDim.y : blockIdx.z + 1 == gridDim.z)
                           ? G.n[D] + 1 : d0 + TD);
    // stage: cells x0-3 .. x0+TX+1 of the row (D = 0), or x0..x0+TX-1 by
    // d0-3 .. d0+TD+1 along D; only cells inside the padded grid
    const int nf_stage = useJ ? NF : NPR;
    if (tma) {
        if (threadIdx.x == 0) mbar_init(&bar, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            mbar_expect_tx(&bar, 4u * FSTRIDE * (NPR + (useJ ? 1 : 0)));
            // padded coordinates: x of cell x0-3 is x0 (3 ghost cells); along
            // D > 0 the first staged cell d0-3 is at d0
            const int cy = D == 1 ? d0 : c1 + G.g[1];
            const int cz = D == 2 ? d0 : c2 + G.g[2];
            tma_load_4d(sm, &tmP, x0, cy, cz, 0, &bar);
            if (useJ) tma_load_3d(sm + JOFF, &tmJ, x0, cy, cz, &bar);
        }
        // the block gives up together if any thread's bounded wait ran out
        const bool arrived = mbar_wait(&bar, 0, TILE_WAIT_POLLS);
        if (__syncthreads_or(!arrived)) {
            if (threadIdx.x == 0) atomicOr(&stats[ST_TILE], 1ULL);
            if (!arrived) mbar_wait(&bar, 0, TILE_WAIT_POLLS);   // let copies in flight land
            return;
        }
    }
    for (int idx = threadIdx.x; idx < (tma ? 0 : LD * (LX - XO)); idx += blockDim.x) {
        const int dl = idx / (LX - XO), xl = idx - dl * (LX - XO);
        int ci, cj, ck;
        bool ok;
        if (D == 0) {
            ci = x0 - 3 + xl; cj = c1; ck = c2;
            ok = ci <= G.n[0] + 2;
        } else if (D == 1) {
            ci = x0 + xl; cj = d0 - 3 + dl; ck = c2;
            ok = ci < G.n[0] && cj <= G.n[1] + 2;
        } else {
            ci = x0 + xl; cj = c1; ck = d0 - 3 + dl;
            ok = ci < G.n[0] && ck <= G.n[2] + 2;
        }
        if (!ok) continue;
        const long long c = cell_at(G, ci, cj, ck);
        for (int f = 0; f < nf_stage; f++)
            sm[foff(f) + dl * LX + xl + XO] = f < NPR ? P[f * S + c] : Jc[D * S + c];
    }
    __syncthreads();

    const int ty = D == 0 ? 0 : (threadIdx.x >> 5);
    constexpr int PER = D == 0 ? 2 : TD / 4 + 1;
    const float gfac = K.gfacf;
#pragma unroll 1
    for (int r = 0; r < PER; r++) {
        const int dloc = D == 0 ? 0 : ty + 4 * r;
        const int tx = D == 0 ? threadIdx.x + TX * r : (threadIdx.x & 31);
        int fi, fj, fk;   // face = low side of cell (fi, fj, fk)
        if (D == 0) {
            fi = x0 + tx; fj = c1; fk = c2;
            if (fi >= x_end) break;
        } else if (D == 1) {
            fi = x0 + tx; fj = d0 + dloc; fk = c2;
            if (fi >= G.n[0] || fj >= d_end) break;
        } else {
            fi = x0 + tx; fj = c1; fk = d0 + dloc;
            if (fi >= G.n[0] || fk >= d_end) break;
        }
        const long long cR = cell_at(G, fi, fj, fk);
        const long long cL = cR - s;
        // stencil o = 0..5: cells (face - 3 + o) along D
        auto at = [&](int f, int o) -> float {
            return D == 0 ? sm[foff(f) + tx + o] : sm[foff(f) + (dloc + o) * LX + tx + XO];
        };
        float pL[NPR], pR[NPR];
#pragma unroll
        for (int f = 0; f < NPR; f++) {
            float st[6];
            if (RC == RC_WENO5) {
#pragma unroll
                for (int o = 0; o < 6; o++) st[o] = at(f, o);
            } else {
#pragma unroll
                for (int o = 1; o < 5; o++) st[o] = at(f, o);
                st[0] = st[5] = 0.f;
            }
            reconstruct<float, RC>(st, pL[f], pR[f]);
        }
        float JL = 0.f, JR = 0.f;
        if (useJ) {
            float st[6];
            if (RC == RC_WENO5) {
#pragma unroll
                for (int o = 0; o < 6; o++) st[o] = at(NPR, o);
            } else {
#pragma unroll
                for (int o = 1; o < 5; o++) st[o] = at(NPR, o);
                st[0] = st[5] = 0.f;
            }
            reconstruct<float, RC>(st, JL, JR);
        }
        Met<float> m;
        if (FLAT) {
            m.alpha = 1.f;
            m.beta[0] = m.beta[1] = m.beta[2] = 0.f;
            m.g[0] = m.g[3] = m.g[5] = 1.f;
            m.g[1] = m.g[2] = m.g[4] = 0.f;
            m.gi[0] = m.gi[3] = m.gi[5] = 1.f;
            m.gi[1] = m.gi[2] = m.gi[4] = 0.f;
            m.sg = m.isg = 1.f;
        } else {
            m.alpha = (float)(0.5 * (met[M_ALPHA * S + cL] + met[M_ALPHA * S + cR]));
            for (int a = 0; a < 3; a++)
                m.beta[a] = (float)(0.5 * (met[(M_BETA + a) * S + cL] + met[(M_BETA + a) * S + cR]));
            for (int a = 0; a < 6; a++)
                m.g[a] = (float)(0.5 * (met[(M_GAMMA + a) * S + cL] + met[(M_GAMMA + a) * S + cR]));
            met_complete(m);
        }
#pragma unroll
        for (int sd = 0; sd < 2; sd++) {
            float *q = sd == 0 ? pL : pR;
            float v[3] = {q[PR_VX], q[PR_VY], q[PR_VZ]}, vl[3];
            lower<float, FLAT>(m, v, vl);
            if (!(q[PR_RHO] > 0.f) || !(q[PR_P] > 0.f) || !(dot3(v, vl) < 1.f)) {
                const int o = sd == 0 ? 2 : 3;
#pragma unroll
                for (int f = 0; f < NPR; f++) q[f] = at(f, o);
                if (useJ) {
                    if (sd == 0) JL = at(NPR, o);
                    else JR = at(NPR, o);
                }
            }
        }
        float sigma = K.sigma0f;
        if (K.sigma_model == 1) {
            sigma = (float)(K.sigma0 * 0.5 * (sig[cL] + sig[cR]));
        } else if (K.sigma_model >= 2) {
            double sgm = 0.0;
            for (int sd = 0; sd < 2; sd++) {
                const long long cc = sd == 0 ? cL : cR;
                Met<double> mc;
                load_metric<FLAT>(met, S, cc, mc);
                double v[3] = {(double)P[PR_VX * S + cc], (double)P[PR_VY * S + cc],
                               (double)P[PR_VZ * S + cc]}, vl[3];
                lower<double, FLAT>(mc, v, vl);
                double Dc = mc.sg * (double)P[PR_RHO * S + cc] / sqrt(1.0 - dot3(v, vl));
                sgm += 0.5 * sigma_cell(K, sig, cc, Dc);
            }
            sigma = (float)sgm;
        }
        float cFL, cFR, cUU;
        if (FLAT) {
            cFL = 0.5f; cFR = 0.5f; cUU = -0.5f;
        } else {
            const float sq = sqrt(m.gi[sym(D, D)]);
            const float bs = m.beta[D] / m.alpha;
            float ap = sq - bs, am = -sq - bs;
            ap = ap > 0.f ? ap : 0.f;
            am = am < 0.f ? am : 0.f;
            const float inv = 1.f / (ap - am);
            cFL = ap * inv; cFR = -am * inv; cUU = ap * am * inv;
        }
        float acc[NCO];
#pragma unroll
        for (int f = 0; f < NCO; f++) acc[f] = 0.f;
        ArrAcc<float> aa{acc};
        flux_accumulate<float, FLAT, D>(pL, m, sigma, gfac, useJ, JL, cFL, -cUU, aa);
        flux_accumulate<float, FLAT, D>(pR, m, sigma, gfac, useJ, JR, cFR, cUU, aa);
#pragma unroll
        for (int f = 0; f < NCO; f++) F[f * S + cR] = acc[f];
    }
}

// FP32 face fluxes along y or z (D > 0) for the TVD reconstructions,
// walking: lane t of a warp owns the line x = x0 + t along D and the
// block's four warps walk consecutive runs of FW faces along it, so that
// loads and flux stores stay coalesced along x.  The block's cells (15
// fields: primitives and J^D) with their halo are staged in shared memory,
// [field][position along D][lane] with a row pitch of 33 words.  Each cell
// is reconstructed once (one slope for its states at the face below and
// above, same arithmetic as reconstruct()); a face takes the upper state of
// the cell below, carried in registers from the previous face, and the
// lower state of the cell above.  The last block along D also takes face
// n_D (its last warp walks one face more).
constexpr int FW = 3;          // faces per warp run
constexpr int FB = 4 * FW;     // faces per block along D (the last block: one more)

// TVD states of the cell s[1] (stencil s[0..2]) at its lower (uM) and
// upper (uP) faces from one slope, the arithmetic of reconstruct()
template <class T, int RC>
__device__ __forceinline__ void recon_cell(const T s[3], T &uM, T &uP)
{
    const T sl = tvd_slope<T, RC>(s[0], s[1], s[2]);
    uP = s[1] + T(0.5) * sl;
    uM = s[1] - T(0.5) * sl;
}

// Staging by TMA (tma != 0): one bulk tensor copy of the 14 primitive fields
// and one of J^D, boxes of 36 (x) by LD (along D) cells starting at the
// 4-aligned x of the padded grid three cells before the block's first line,
// so line t sits at column t + 3 of a 36-float row; completion on an
// mbarrier.  Otherwise the threads stage the same rows with plain loads.
constexpr int WALK_PITCH = 36;
constexpr int WALK_LD = FB + 7;                                   // cells f0-3 .. f0+FB+3
constexpr int WALK_JOFF = (NPR * WALK_LD * WALK_PITCH + 31) / 32 * 32;   // J rows, 128-byte aligned
constexpr int WALK_SMEM = WALK_JOFF + WALK_LD * WALK_PITCH;

template <bool FLAT, int RC, int D>
__global__ void __launch_bounds__(128, 6)
k_flux_walk(const StepConst K, const float *__restrict__ P, const float *__restrict__ Jc,
            const double *__restrict__ met, const double *__restrict__ sig, float *F,
            const __grid_constant__ CUtensorMap tmP, const __grid_constant__ CUtensorMap tmJ,
            int tma, unsigned long long *stats)
{
    static_assert(D > 0 && RC != RC_WENO5, "TVD faces along y and z only (else k_flux_tile)");
    constexpr int NF = NPR + 1;
    constexpr int LD = WALK_LD;
    constexpr int PITCH = WALK_PITCH;
    __shared__ __align__(128) float sm[WALK_SMEM];
    __shared__ __align__(8) uint64_t bar;
    const Grid &G = K.G;
    const long long S = G.S;
    const long long s = dstride(G, D);
    const bool useJ = K.qflux != 1;   // mode 2: Q row overwritten later
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // block origin: first face f0 along D, first line x0 = t0, the remaining
    // coordinate c2 (z for D = 1, y for D = 2)
    int f0, t0, c2;
    bool last;
    if (D == 1) {
        f0 = blockIdx.y * FB; t0 = blockIdx.x * 32; c2 = blockIdx.z;
        last = blockIdx.y + 1 == gridDim.y;
    } else {
        f0 = blockIdx.z * FB; t0 = blockIdx.x * 32; c2 = blockIdx.y;
        last = blockIdx.z + 1 == gridDim.z;
    }
    const int nD = G.n[D], nT = G.n[0];
    const int f_end = last ? nD + 1 : f0 + FB;      // faces f0 .. f_end-1
    // cell of line t, position d along D (d = 0: cell f0-3)
    auto cell = [&](int t, int d) -> long long {
        const int a = f0 - 3 + d, b = t0 + t;
        if (D == 1) return cell_at(G, b, a, c2);
        return cell_at(G, b, c2, a);
    };
    // row of field f at position d (cell f0-3+d along D); line t at t + 3
    auto row = [&](int f, int d) -> int {
        return (f < NPR ? (f * LD + d) * PITCH : WALK_JOFF + d * PITCH) + 3;
    };
    if (tma) {
        if (threadIdx.x == 0) mbar_init(&bar, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned bytes = 4u * PITCH * LD * (NPR + (useJ ? 1 : 0));
            mbar_expect_tx(&bar, bytes);
            // padded coordinates: x of line -3 is t0 (3 ghost cells), the
            // first cell along D (f0 - 3) is at f0, the fixed one at c2 + g
            const int cy = D == 1 ? f0 : c2 + G.g[1];
            const int cz = D == 1 ? c2 + G.g[2] : f0;
            tma_load_4d(sm, &tmP, t0, cy, cz, 0, &bar);
            if (useJ) tma_load_3d(sm + WALK_JOFF, &tmJ, t0, cy, cz, &bar);
        }
        // the block gives up together if any thread's bounded wait ran out
        const bool arrived = mbar_wait(&bar, 0, TILE_WAIT_POLLS);
        if (__syncthreads_or(!arrived)) {
            if (threadIdx.x == 0) atomicOr(&stats[ST_TILE], 1ULL);
            if (!arrived) mbar_wait(&bar, 0, TILE_WAIT_POLLS);   // let copies in flight land
            return;
        }
    } else {
        // stage cells f0-3 .. f_end+1 along D of the block's lines (x fastest)
        const int nd_stage = f_end + 2 - (f0 - 3);
        const int nf_stage = useJ ? NF : NPR;
        for (int idx = threadIdx.x; idx < 32 * nd_stage; idx += blockDim.x) {
            const int d = idx >> 5, t = idx & 31;
            if (t0 + t >= nT) continue;
            const long long c = cell(t, d);
            for (int f = 0; f < nf_stage; f++)
                sm[row(f, d) + t] = f < NPR ? P[f * S + c] : Jc[D * S + c];
        }
        __syncthreads();
    }
    auto at = [&](int f, int d) -> float { return sm[row(f, d) + lane]; };

    // this warp's faces fs .. fe-1 (the last warp takes the rest of the block)
    const int fs = f0 + w * FW;
    const int fe = w == 3 ? f_end : min(fs + FW, f_end);
    if (t0 + lane >= nT || fs >= fe) return;
    const float gfac = K.gfacf;
    // upper states of the cell below the first face, then the walk
    float up[NF];
    {
        const int d = fs - 1 - (f0 - 3);
#pragma unroll
        for (int f = 0; f < NF; f++) {
            if (f == NPR && !useJ) { up[f] = 0.f; continue; }
            const float st[3] = {at(f, d - 1), at(f, d), at(f, d + 1)};
            float um;
            recon_cell<float, RC>(st, um, up[f]);
        }
    }
#pragma unroll 1
    for (int fi = fs; fi < fe; fi++) {
        const int dR = fi - (f0 - 3);          // the cell above the face
        float pL[NPR], pR[NPR], upn[NF];
        float JL = up[NPR], JR = 0.f;
#pragma unroll
        for (int f = 0; f < NF; f++) {
            if (f == NPR && !useJ) { upn[f] = 0.f; continue; }
            const float st[3] = {at(f, dR - 1), at(f, dR), at(f, dR + 1)};
            float um;
            recon_cell<float, RC>(st, um, upn[f]);
            if (f < NPR) { pL[f] = up[f]; pR[f] = um; }
            else JR = um;
        }
        const long long cR = cell(lane, dR), cL = cR - s;
        Met<float> m;
        if (FLAT) {
            m.alpha = 1.f;
            m.beta[0] = m.beta[1] = m.beta[2] = 0.f;
            m.g[0] = m.g[3] = m.g[5] = 1.f;
            m.g[1] = m.g[2] = m.g[4] = 0.f;
            m.gi[0] = m.gi[3] = m.gi[5] = 1.f;
            m.gi[1] = m.gi[2] = m.gi[4] = 0.f;
            m.sg = m.isg = 1.f;
        } else {
            m.alpha = (float)(0.5 * (met[M_ALPHA * S + cL] + met[M_ALPHA * S + cR]));
            for (int a = 0; a < 3; a++)
                m.beta[a] = (float)(0.5 * (met[(M_BETA + a) * S + cL] + met[(M_BETA + a) * S + cR]));
            for (int a = 0; a < 6; a++)
                m.g[a] = (float)(0.5 * (met[(M_GAMMA + a) * S + cL] + met[(M_GAMMA + a) * S + cR]));
            met_complete(m);
        }
        // a face state with rho <= 0, p <= 0 or v^2 >= 1 falls back to its
        // cell's values (all fields)
#pragma unroll
        for (int sd = 0; sd < 2; sd++) {
            float *q = sd == 0 ? pL : pR;
            float v[3] = {q[PR_VX], q[PR_VY], q[PR_VZ]}, vl[3];
            lower<float, FLAT>(m, v, vl);
            if (!(q[PR_RHO] > 0.f) || !(q[PR_P] > 0.f) || !(dot3(v, vl) < 1.f)) {
                const int d = sd == 0 ? dR - 1 : dR;
#pragma unroll
                for (int f = 0; f < NPR; f++) q[f] = at(f, d);
                if (useJ) {
                    if (sd == 0) JL = at(NPR, d);
                    else JR = at(NPR, d);
                }
            }
        }
        float sigma = K.sigma0f;
        if (K.sigma_model == 1) {
            sigma = (float)(K.sigma0 * 0.5 * (sig[cL] + sig[cR]));
        } else if (K.sigma_model >= 2) {
            double sgm = 0.0;
            for (int sd = 0; sd < 2; sd++) {
                const long long cc = sd == 0 ? cL : cR;
                Met<double> mc;
                load_metric<FLAT>(met, S, cc, mc);
                double v[3] = {(double)P[PR_VX * S + cc], (double)P[PR_VY * S + cc],
                               (double)P[PR_VZ * S + cc]}, vl[3];
                lower<double, FLAT>(mc, v, vl);
                double Dc = mc.sg * (double)P[PR_RHO * S + cc] / sqrt(1.0 - dot3(v, vl));
                sgm += 0.5 * sigma_cell(K, sig, cc, Dc);
            }
            sigma = (float)sgm;
        }
        float cFL, cFR, cUU;
        if (FLAT) {
            cFL = 0.5f; cFR = 0.5f; cUU = -0.5f;
        } else {
            const float sq = sqrt(m.gi[sym(D, D)]);
            const float bs = m.beta[D] / m.alpha;
            float ap = sq - bs, am = -sq - bs;
            ap = ap > 0.f ? ap : 0.f;
            am = am < 0.f ? am : 0.f;
            const float inv = 1.f / (ap - am);
            cFL = ap * inv; cFR = -am * inv; cUU = ap * am * inv;
        }
        float acc[NCO];
#pragma unroll
        for (int f = 0; f < NCO; f++) acc[f] = 0.f;
        ArrAcc<float> aa{acc};
        flux_accumulate<float, FLAT, D>(pL, m, sigma, gfac, useJ, JL, cFL, -cUU, aa);
        flux_accumulate<float, FLAT, D>(pR, m, sigma, gfac, useJ, JR, cFR, cUU, aa);
#pragma unroll
        for (int f = 0; f < NCO; f++) F[f * S + cR] = acc[f];
#pragma unroll
        for (int f = 0; f < NF; f++) up[f] = upn[f];
    }
}

// FP32 face fluxes along x for the TVD reconstructions, walking: each warp
// takes a segment of 128 faces of one x row (the row's last segment also
// its face n) in chunks of 32, lane L owning face and cell x0 + 32 ch + L.
// Each cell is reconstructed once (one slope for its states at the face
// below and above, the arithmetic of reconstruct()); a face takes the upper
// state of the cell below from the lane below (a warp shuffle; lane 0 from
// lane 31 of the chunk before, or, for the segment's first face, from the
// cell x0 - 1 reconstructed by every lane) and the lower state of its own
// cell, so that a warp stores 32 consecutive faces per field.  The block's
// four warps take four consecutive rows, staged by one tensor-map copy of
// 136 x 4 cells x 14 fields (cells x0-3 .. x0+132 of each row) and one of
// J^x, completion on an mbarrier (tma != 0), or with plain loads.
constexpr int XW_ROWS = 4;
constexpr int XW_LX = 136;

template <bool FLAT, int RC>
__global__ void __launch_bounds__(128, 6)
k_flux_xwalk(const StepConst K, const float *__restrict__ P, const float *__restrict__ Jc,
             const double *__restrict__ met, const double *__restrict__ sig, float *F,
             const __grid_constant__ CUtensorMap tmP, const __grid_constant__ CUtensorMap tmJ,
             int tma, unsigned long long *stats)
{
    static_assert(RC != RC_WENO5, "TVD reconstructions only (else k_flux_tile)");
    constexpr int D = 0;
    constexpr int NF = NPR + 1;
    constexpr int ROWSZ = XW_ROWS * XW_LX;   // floats per field
    constexpr int JOFF = NPR * ROWSZ;        // J^x rows (a multiple of 32 floats)
    static_assert(JOFF % 32 == 0, "128-byte aligned J rows");
    __shared__ __align__(128) float sm[JOFF + ROWSZ];
    __shared__ __align__(8) uint64_t bar;
    const Grid &G = K.G;
    const long long S = G.S;
    const bool useJ = K.qflux != 1;   // mode 2: Q row overwritten later
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int x0 = blockIdx.x * 128;
    const int j = blockIdx.y * XW_ROWS + w, k = blockIdx.z;
    const int x_end = blockIdx.x + 1 == gridDim.x ? G.n[0] + 1 : x0 + 128;   // faces x0 .. x_end-1
    if (tma) {
        if (threadIdx.x == 0) mbar_init(&bar, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            mbar_expect_tx(&bar, 4u * ROWSZ * (NPR + (useJ ? 1 : 0)));
            // padded coordinates: x of cell x0-3 is x0 (3 ghost cells)
            const int cy = blockIdx.y * XW_ROWS + G.g[1], cz = k + G.g[2];
            tma_load_4d(sm, &tmP, x0, cy, cz, 0, &bar);
            if (useJ) tma_load_3d(sm + JOFF, &tmJ, x0, cy, cz, &bar);
        }
        // the block gives up together if any thread's bounded wait ran out
        const bool arrived = mbar_wait(&bar, 0, TILE_WAIT_POLLS);
        if (__syncthreads_or(!arrived)) {
            if (threadIdx.x == 0) atomicOr(&stats[ST_TILE], 1ULL);
            if (!arrived) mbar_wait(&bar, 0, TILE_WAIT_POLLS);   // let copies in flight land
            return;
        }
    } else {
        // the same cells with plain loads (zeros past the row's ghost cells
        // and for rows past the grid: read by no face that is stored)
        const int nf_stage = useJ ? NF : NPR;
        for (int idx = threadIdx.x; idx < ROWSZ; idx += blockDim.x) {
            const int r = idx / XW_LX, xl = idx - r * XW_LX;
            const int ci = x0 - 3 + xl, cj = blockIdx.y * XW_ROWS + r;
            const bool ok = ci <= G.n[0] + 2 && cj < G.n[1];
            const long long c = ok ? cell_at(G, ci, cj, k) : 0;
            for (int f = 0; f < nf_stage; f++)
                sm[(f < NPR ? f * ROWSZ : JOFF) + idx] =
                    ok ? (f < NPR ? P[f * S + c] : Jc[D * S + c]) : 0.f;
        }
        __syncthreads();
    }
    if (j >= G.n[1]) return;   // the whole warp: rows past the grid
    // field f of this warp's row at column xl (cell x0 - 3 + xl)
    auto at = [&](int f, int xl) -> float {
        return f < NPR ? sm[f * ROWSZ + w * XW_LX + xl] : sm[JOFF + w * XW_LX + xl];
    };
    const float gfac = K.gfacf;
    const int nch = (x_end - x0 + 31) >> 5;   // 4, or 5 when the segment also takes face n
    // upper states of the cell x0 - 1 (column 2): the left state of face x0
    float carry[NF];
#pragma unroll
    for (int f = 0; f < NF; f++) {
        if (f == NPR && !useJ) { carry[f] = 0.f; continue; }
        const float st[3] = {at(f, 1), at(f, 2), at(f, 3)};
        float um;
        recon_cell<float, RC>(st, um, carry[f]);
    }
#pragma unroll 1
    for (int ch = 0; ch < nch; ch++) {
        const int fi = x0 + 32 * ch + lane;
        const bool live = fi < x_end;
        // column of cell fi; lanes past the segment's faces (which store
        // nothing and feed only lanes past it) read a clamped column
        const int xl = min(32 * ch + lane + 3, XW_LX - 2);
        float pL[NPR], pR[NPR];
        float JL = 0.f, JR = 0.f;
#pragma unroll
        for (int f = 0; f < NF; f++) {
            if (f == NPR && !useJ) continue;
            const float st[3] = {at(f, xl - 1), at(f, xl), at(f, xl + 1)};
            float um, up;
            recon_cell<float, RC>(st, um, up);
            const float below = __shfl_up_sync(0xffffffffu, up, 1);
            const float left = lane == 0 ? carry[f] : below;
            carry[f] = __shfl_sync(0xffffffffu, up, 31);   // for the next chunk's lane 0
            if (f < NPR) { pL[f] = left; pR[f] = um; }
            else { JL = left; JR = um; }
        }
        if (!live) continue;
        const long long cR = cell_at(G, fi, j, k), cL = cR - 1;
        Met<float> m;
        if (FLAT) {
            m.alpha = 1.f;
            m.beta[0] = m.beta[1] = m.beta[2] = 0.f;
            m.g[0] = m.g[3] = m.g[5] = 1.f;
            m.g[1] = m.g[2] = m.g[4] = 0.f;
            m.gi[0] = m.gi[3] = m.gi[5] = 1.f;
            m.gi[1] = m.gi[2] = m.gi[4] = 0.f;
            m.sg = m.isg = 1.f;
        } else {
            m.alpha = (float)(0.5 * (met[M_ALPHA * S + cL] + met[M_ALPHA * S + cR]));
            for (int a = 0; a < 3; a++)
                m.beta[a] = (float)(0.5 * (met[(M_BETA + a) * S + cL] + met[(M_BETA + a) * S + cR]));
            for (int a = 0; a < 6; a++)
                m.g[a] = (float)(0.5 * (met[(M_GAMMA + a) * S + cL] + met[(M_GAMMA + a) * S + cR]));
            met_complete(m);
        }
        // a face state with rho <= 0, p <= 0 or v^2 >= 1 falls back to its
        // cell's values (all fields)
#pragma unroll
        for (int sd = 0; sd < 2; sd++) {
            float *q = sd == 0 ? pL : pR;
            float v[3] = {q[PR_VX], q[PR_VY], q[PR_VZ]}, vl[3];
            lower<float, FLAT>(m, v, vl);
            if (!(q[PR_RHO] > 0.f) || !(q[PR_P] > 0.f) || !(dot3(v, vl) < 1.f)) {
                const int xc = sd == 0 ? xl - 1 : xl;
#pragma unroll
                for (int f = 0; f < NPR; f++) q[f] = at(f, xc);
                if (useJ) {
                    if (sd == 0) JL = at(NPR, xc);
                    else JR = at(NPR, xc);
                }
            }
        }
        float sigma = K.sigma0f;
        if (K.sigma_model == 1) {
            sigma = (float)(K.sigma0 * 0.5 * (sig[cL] + sig[cR]));
        } else if (K.sigma_model >= 2) {
            double sgm = 0.0;
            for (int sd = 0; sd < 2; sd++) {
                const long long cc = sd == 0 ? cL : cR;
                Met<double> mc;
                load_metric<FLAT>(met, S, cc, mc);
                double v[3] = {(double)P[PR_VX * S + cc], (double)P[PR_VY * S + cc],
                               (double)P[PR_VZ * S + cc]}, vl[3];
                lower<double, FLAT>(mc, v, vl);
                double Dc = mc.sg * (double)P[PR_RHO * S + cc] / sqrt(1.0 - dot3(v, vl));
                sgm += 0.5 * sigma_cell(K, sig, cc, Dc);
            }
            sigma = (float)sgm;
        }
        float cFL, cFR, cUU;
        if (FLAT) {
            cFL = 0.5f; cFR = 0.5f; cUU = -0.5f;
        } else {
            const float sq = sqrt(m.gi[sym(D, D)]);
            const float bs = m.beta[D] / m.alpha;
            float ap = sq - bs, am = -sq - bs;
            ap = ap > 0.f ? ap : 0.f;
            am = am < 0.f ? am : 0.f;
            const float inv = 1.f / (ap - am);
            cFL = ap * inv; cFR = -am * inv; cUU = ap * am * inv;
        }
        float acc[NCO];
#pragma unroll
        for (int f = 0; f < NCO; f++) acc[f] = 0.f;
        ArrAcc<float> aa{acc};
        flux_accumulate<float, FLAT, D>(pL, m, sigma, gfac, useJ, JL, cFL, -cUU, aa);
        flux_accumulate<float, FLAT, D>(pR, m, sigma, gfac, useJ, JR, cFR, cUU, aa);
#pragma unroll
        for (int f = 0; f < NCO; f++) F[f * S + cR] = acc[f];
    }
}

// Reconstruction of cell c along D: its state at the face below (m) and
// above (p) for the 14 primitives and, when J != nullptr, the current J^D.
template <class T, int RC>
__device__ __forceinline__ void cell_faces(const T *__restrict__ P, const T *__restrict__ Jc,
                                           long long S, long long c, long long s, int D,
                                           T m[NPR + 1], T p[NPR + 1])
{
#pragma unroll
    for (int f = 0; f <= NPR; f++) {
        if (f == NPR && !Jc) break;
        const T *q = f < NPR ? P + f * S + c : Jc + D * S + c;
        if (RC == RC_WENO5) {
            const T a = q[-2 * s], b = q[-s], cc = q[0], d = q[s], e = q[2 * s];
            p[f] = weno5(a, b, cc, d, e);
            m[f] = weno5(e, d, cc, b, a);
        } else {
            const T a = q[-s], b = q[0], d = q[s];
            const T h = T(0.5) * tvd_slope<T, RC>(a, b, d);
            p[f] = b + h;
            m[f] = b - h;
        }
    }
}

// Face fluxes in direction D for a run of M consecutive faces per thread:
// every cell is reconstructed once and its upper face state is carried to
// the next face in registers (the per-face kernel above reconstructs each
// cell twice).  Face f lies between cells f-1 and f along D and is stored at
// cell f.  Same arithmetic per face as k_flux.
template <class T, bool FLAT, int RC, int D, int M>
__global__ void __launch_bounds__(128) k_flux_run(const StepConst K, const T *__restrict__ P,
                                                  const T *__restrict__ Jc,
                                                  const double *__restrict__ met,
                                                  const double *__restrict__ sig, T *F)
{
    const Grid &G = K.G;
    const unsigned nrun = (unsigned)((G.n[D] + 1 + M - 1) / M);
    // thread -> (run along D, the two other coordinates), x fastest
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned e0, e1, run;
    const unsigned n0 = D == 0 ? nrun : (unsigned)G.n[0];
    const unsigned n1 = D == 1 ? nrun : (unsigned)G.n[1];
    const unsigned n2 = D == 2 ? nrun : (unsigned)G.n[2];
    if (t >= n0 * n1 * n2) return;
    const unsigned q0 = t / n0;
    const unsigned i0 = t - q0 * n0;
    const unsigned i2 = q0 / n1;
    const unsigned i1 = q0 - i2 * n1;
    int ijk[3] = {(int)i0, (int)i1, (int)i2};
    run = (unsigned)ijk[D];
    (void)e0; (void)e1;
    const int f0 = (int)run * M;
    const int fend = min(f0 + M, G.n[D] + 1);
    ijk[D] = f0 - 1;
    const long long s = dstride(G, D);
    const long long S = G.S;
    long long c = cell_at(G, ijk[0], ijk[1], ijk[2]);   // cell f0 - 1
    const bool useJ = K.qflux != 1;   // mode 2: Q row overwritten later
    const T *Jp = useJ ? Jc : nullptr;
    T mL[NPR + 1], pL[NPR + 1];                          // of the cell below the face
    cell_faces<T, RC>(P, Jp, S, c, s, D, mL, pL);
    const T gfac = kc<T>(K.gfac, K.gfacf);
    for (int f = f0; f < fend; f++) {
        const long long cL = c, cR = c + s;
        T mR[NPR + 1], pR[NPR + 1];
        cell_faces<T, RC>(P, Jp, S, cR, s, D, mR, pR);
        // face state arrays: left = upper state of cL, right = lower state of cR
        T sL[NPR], sR[NPR];
#pragma unroll
        for (int k = 0; k < NPR; k++) {
            sL[k] = pL[k];
            sR[k] = mR[k];
        }
        T JL = useJ ? pL[NPR] : T(0), JR = useJ ? mR[NPR] : T(0);
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
#pragma unroll
        for (int sd = 0; sd < 2; sd++) {
            T *q = sd == 0 ? sL : sR;
            T v[3] = {q[PR_VX], q[PR_VY], q[PR_VZ]}, vl[3];
            lower<T, FLAT>(m, v, vl);
            if (!(q[PR_RHO] > T(0)) || !(q[PR_P] > T(0)) || !(dot3(v, vl) < T(1))) {
                const long long cc = sd == 0 ? cL : cR;
#pragma unroll
                for (int k = 0; k < NPR; k++) q[k] = P[k * S + cc];
                if (useJ) {
                    if (sd == 0) JL = Jc[D * S + cc];
                    else JR = Jc[D * S + cc];
                }
            }
        }
        T sigma = kc<T>(K.sigma0, K.sigma0f);
        if (K.sigma_model == 1) {
            sigma = (T)(K.sigma0 * 0.5 * (sig[cL] + sig[cR]));
        } else if (K.sigma_model >= 2) {
            double sgm = 0.0;
            for (int sd = 0; sd < 2; sd++) {
                const long long cc = sd == 0 ? cL : cR;
                Met<double> mc;
                load_metric<FLAT>(met, S, cc, mc);
                double v[3] = {(double)P[PR_VX * S + cc], (double)P[PR_VY * S + cc],
                               (double)P[PR_VZ * S + cc]}, vl[3];
                lower<double, FLAT>(mc, v, vl);
                double Dc = mc.sg * (double)P[PR_RHO * S + cc] / sqrt(1.0 - dot3(v, vl));
                sgm += 0.5 * sigma_cell(K, sig, cc, Dc);
            }
            sigma = (T)sgm;
        }
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
        T acc[NCO];
#pragma unroll
        for (int k = 0; k < NCO; k++) acc[k] = T(0);
        ArrAcc<T> aa{acc};
        flux_accumulate<T, FLAT, D>(sL, m, sigma, gfac, useJ, JL, cFL, -cUU, aa);
        flux_accumulate<T, FLAT, D>(sR, m, sigma, gfac, useJ, JR, cFR, cUU, aa);
#pragma unroll
        for (int k = 0; k < NCO; k++) F[k * S + cR] = acc[k];
        // slide: the cell above becomes the cell below
#pragma unroll
        for (int k = 0; k <= NPR; k++) pL[k] = pR[k];
        c = cR;
    }
}

// Source vector of Eq. GRRMHD_flux_form without the stiff part of -alpha J
// (Sec. III.A split), at a cell with primitives pr.  Metric derivatives:
// second-order central differences of the cell-centred metric.
// Sources of a cell on a curved static metric, with the primitive-dependent
// quantities in R (double, or a dual number in the adjoint) and the metric,
// its derivatives and K_ij in FP64.
template <class R>
__device__ __forceinline__ void sources_curved(const StepConst &K, const R pr[NPR],
                                               const double *__restrict__ met, long long c,
                                               R Sv[NCO])
{
    const double kap = K.kappa;
    const Grid &G = K.G;
    const long long S = G.S;
    Met<double> m;
    load_metric<false>(met, S, c, m);
    const Met<R> mr = met_cast<R>(m);
    R U[NCO];
    prim_to_cons<R, false>(pr, mr, R(K.gfac), U);
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
    R v[3] = {pr[PR_VX], pr[PR_VY], pr[PR_VZ]};
    R E[3] = {pr[PR_EX], pr[PR_EY], pr[PR_EZ]};
    R B[3] = {pr[PR_BX], pr[PR_BY], pr[PR_BZ]};
    R vl[3], El[3], Bl[3];
    lower<R, false>(mr, v, vl);
    lower<R, false>(mr, E, El);
    lower<R, false>(mr, B, Bl);
    const R W2 = 1.0 / (1.0 - dot3(v, vl));
    const R hW2 = (pr[PR_RHO] + K.gfac * pr[PR_P]) * W2;
    const R pem = pr[PR_P] + 0.5 * (dot3(E, El) + dot3(B, Bl));
    R Sup[6];   // undensitised stress, indices up
    for (int a = 0; a < 3; a++)
        for (int b = a; b < 3; b++)
            Sup[sym(a, b)] = hW2 * v[a] * v[b] + gi[sym(a, b)] * pem - E[a] * E[b] - B[a] * B[b];
    const double al = m.alpha, sg = m.sg;
    R Su[3];
    R Sl[3] = {U[CO_SX], U[CO_SY], U[CO_SZ]};
    raise<R, false>(mr, Sl, Su);
    for (int a = 0; a < 3; a++) {
        R s = 0.0;
        for (int b = 0; b < 3; b++)
            for (int cc = 0; cc < 3; cc++) s += Sup[sym(b, cc)] * dg[a][sym(b, cc)];
        s *= 0.5 * al * sg;
        for (int b = 0; b < 3; b++) s += Sl[b] * db[a][b];
        s -= (U[CO_TAU] + U[CO_D]) * da[a];
        Sv[CO_SX + a] = s;
    }
    {
        R s = Sup[0] * Kij[0] + Sup[3] * Kij[3] + Sup[5] * Kij[5] +
                   2.0 * (Sup[1] * Kij[1] + Sup[2] * Kij[2] + Sup[4] * Kij[4]);
        s *= al * sg;
        for (int a = 0; a < 3; a++) s -= Su[a] * da[a];
        Sv[CO_TAU] = s;
    }
    for (int a = 0; a < 3; a++) {
        double G1 = gi[sym(a, 0)] * da[0] + gi[sym(a, 1)] * da[1] + gi[sym(a, 2)] * da[2];
        double G2 = gi[sym(a, 0)] * w[0] + gi[sym(a, 1)] * w[1] + gi[sym(a, 2)] * w[2];
        double geo = G1 - al * G2;
        R sB = 0.0, sE = 0.0;
        for (int b = 0; b < 3; b++) {
            sB -= U[CO_BX + b] * db[b][a];
            sE -= U[CO_EX + b] * db[b][a];
        }
        Sv[CO_BX + a] = sB + U[CO_PHI] * geo;
        Sv[CO_EX + a] = sE + U[CO_PSI] * geo - al * U[CO_Q] * v[a];
    }
    R Bda = 0.0, Eda = 0.0;
    for (int b = 0; b < 3; b++) {
        Bda += U[CO_BX + b] * da[b];
        Eda += U[CO_EX + b] * da[b];
    }
    Sv[CO_PHI] = -al * U[CO_PHI] * Ktr + Bda - al * kap * U[CO_PHI];
    Sv[CO_PSI] = -al * U[CO_PSI] * Ktr + Eda + al * U[CO_Q] - al * kap * U[CO_PSI];
    Sv[CO_D] = 0.0;
    Sv[CO_Q] = 0.0;
}

template <bool FLAT, class T>
__device__ __forceinline__ void sources(const StepConst &K, const T pr_in[NPR],
                                        const double *__restrict__ met, long long c,
                                        T Sv_out[NCO])
{
    const T kapT = kc<T>(K.kappa, K.kappaf);
    if (FLAT) {
        // only -Q v^i (E), -kappa Phi, Q - kappa Psi survive in flat space
        const T *pr = pr_in;
        T *Sv = Sv_out;
        for (int f = 0; f < NCO; f++) Sv[f] = T(0);
        const T Q = pr[PR_Q];
        const T kap = kapT;
        for (int a = 0; a < 3; a++) Sv[CO_EX + a] = -Q * pr[PR_VX + a];
        Sv[CO_PHI] = -kap * pr[PR_PHI];
        Sv[CO_PSI] = Q - kap * pr[PR_PSI];
    } else {
        // curved metric: evaluated in FP64 from the stage primitives
        double pr[NPR], Sv[NCO];
        for (int f = 0; f < NPR; f++) pr[f] = to_double<T>(pr_in[f]);
        sources_curved<double>(K, pr, met, c, Sv);
        for (int f = 0; f < NCO; f++) Sv_out[f] = from_double<T>(Sv[f]);
    }
}

// explicit right-hand side F(U) at an interior cell from the face fluxes (T)
template <bool FLAT, class T>
__device__ __forceinline__ void rhs_cell(const StepConst &K, const T pr[NPR],
                                         const double *__restrict__ met,
                                         const T *__restrict__ Fx, const T *__restrict__ Fy,
                                         const T *__restrict__ Fz, long long c, T r[NCO])
{
    sources<FLAT, T>(K, pr, met, c, r);
    const Grid &G = K.G;
    const T *Fd[3] = {Fx, Fy, Fz};
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if (G.g[d] == 0) continue;
        const long long s = dstride(G, d);
        const T ih = kc<T>(G.idx[d], K.idxf[d]);
        const T *F = Fd[d];
#pragma unroll
        for (int f = 0; f < NCO; f++) r[f] -= (F[f * G.S + c + s] - F[f * G.S + c]) * ih;
    }
}

// ---------------------------------------------------------------- stages

// Deferred recoveries: cells whose paper iteration is still undecided after
// the first pass's iterations are appended, with their iterate, to a work
// list (scratch memory of the handle); a second pass with full warps resumes
// them where they stopped (and runs the fallbacks), instead of letting one
// slow cell hold its warp.  A record holds the stage's conserved input (14) and the guess
// (p, v^i); when the list is full the cell falls back inline.
enum { DREC = NCO + 4 + PSTATE };
struct Defer {
    int *count;          // records written (may exceed cap; cap is the limit)
    int cap;             // 0: no deferral
    int *idx;            // interior linear index of the cell
    double *rec;         // DREC x cap, field-major
    int *hcount;         // records handed on to the warp-per-record pass
    int *hidx;           // their record slots
};

// warp-aggregated slot allocation; every lane of the warp must call it
__device__ __forceinline__ int defer_slot(const Defer &df, bool want)
{
    const unsigned full = 0xffffffffu;
    const unsigned mask = __ballot_sync(full, want);
    if (!mask) return -1;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(df.count, __popc(mask));
    base = __shfl_sync(full, base, leader);
    if (!want) return -1;
    const int slot = base + __popc(mask & ((1u << lane) - 1u));
    return slot < df.cap ? slot : -1;
}

__device__ __forceinline__ void defer_store(const Defer &df, int slot, long long t,
                                            const double u[NCO], double gp, const double gv[3],
                                            const PaperState &ps)
{
    df.idx[slot] = (int)t;
    const long long cap = df.cap;
    for (int f = 0; f < NCO; f++) df.rec[f * cap + slot] = u[f];
    df.rec[(NCO + 0) * cap + slot] = gp;
    for (int a = 0; a < 3; a++) df.rec[(NCO + 1 + a) * cap + slot] = gv[a];
    pstate_save(ps, df.rec + (NCO + 4) * cap + slot, cap);
}

__device__ __forceinline__ void load_rec_in(const double u[NCO], RecIn &in)
{
    in.D = u[CO_D];
    in.tau = u[CO_TAU];
    for (int a = 0; a < 3; a++) {
        in.S[a] = u[CO_SX + a];
        in.cB[a] = u[CO_BX + a];
        in.cE0[a] = u[CO_EX + a];
    }
}

// primitives of a cell: all 14 in T, the recovery guess (p, v^i) in FP64
template <class T>
__device__ __forceinline__ void prim_write(const StepConst &K, long long c, const double pr[NPR],
                                          T *P, double *Gs)
{
    const long long S = K.G.S;
    for (int f = 0; f < NPR; f++) P[f * S + c] = from_double<T>(pr[f]);
    for (int f = 0; f < 4; f++) Gs[f * S + c] = pr[PR_P + f];
}

// stage current J = Q v - Dt R/(alpha Dt) stored as T; the mixed path stores
// it in FP32 and forms it in FP32 from the FP64 operands
template <class T>
__device__ __forceinline__ T stage_current(double Q, double v, double dR, double iad)
{
    if constexpr (std::is_same<T, float>::value)
        return d2f_ftz(Q) * d2f_ftz(v) - d2f_ftz(dR) * d2f_ftz(iad);
    else
        return Q * v - dR * iad;
}

// outputs of stage 1 at a cell (primitives, Dt R1, stage current)
template <class T>
__device__ __forceinline__ void stage1_write(const StepConst &K, long long c, const double pr[NPR],
                                             const double E[3], const double u[NCO], double alpha,
                                             T *P, double *Gs, double *dR1, T *J1)
{
    const long long S = K.G.S;
    prim_write(K, c, pr, P, Gs);
    const double ig = K.igimex, iad = alpha == 1.0 ? K.idt : K.idt / alpha;
    for (int a = 0; a < 3; a++) {
        const double r = (E[a] - u[CO_EX + a]) * ig;
        dR1[a * S + c] = r;
        J1[a * S + c] = stage_current<T>(u[CO_Q], pr[PR_VX + a], r, iad);
    }
}

// outputs of stage 2 after its recovery (V already holds U^n + dt/2 F[U1])
template <class T>
__device__ __forceinline__ void stage2_write(const StepConst &K, long long c, const double p2[NPR],
                                             const double E[3], const double us[NCO], double alpha,
                                             const double *dR1, T *P2, double *G2, double *V,
                                             T *J2)
{
    const long long S = K.G.S;
    prim_write(K, c, p2, P2, G2);
    const double ig = K.igimex, iad = alpha == 1.0 ? K.idt : K.idt / alpha;
    for (int a = 0; a < 3; a++) {
        const double r2 = (E[a] - us[CO_EX + a]) * ig;
        V[(CO_EX + a) * S + c] += 0.5 * (dR1[a * S + c] + r2);
        J2[a * S + c] = stage_current<T>(us[CO_Q], p2[PR_VX + a], r2, iad);
    }
}

// outputs of the final recovery (U already holds U^{n+1})
template <bool FLAT, class T>
__device__ __forceinline__ void final_write(const StepConst &K, long long c, const double pn[NPR],
                                            int status, const Met<double> &m, double *U, T *P,
                                            double *Gs)
{
    const long long S = K.G.S;
    if (status == 2 || status == 3) {
        double u2[NCO];
        prim_to_cons<double, FLAT>(pn, m, K.gfac, u2);
        U[CO_D * S + c] = u2[CO_D];
        U[CO_TAU * S + c] = u2[CO_TAU];
        for (int a = 0; a < 3; a++) U[(CO_SX + a) * S + c] = u2[CO_SX + a];
    }
    prim_write(K, c, pn, P, Gs);
}

// The three stage kernels are FP64-pipe-bound; they are compiled for four
// blocks of 128 threads per SM (128 registers, a few spilled), which hides
// the latency of the FP64 reciprocals better than three blocks without
// spills (measured: stage 2 and the final kernel 3-12% faster; five blocks
// spill too much).
// Stage 1 (purely implicit): recovery of U^n with calE solved, guess P^n
// (Gin; may be Gs, read and written at the same cell).  Also the first
// stage of the general IMEX form, with K.gimex = A_11.
template <bool FLAT, class T>
__global__ void __launch_bounds__(128, 4)
k_stage1(const StepConst K, const double *__restrict__ U, T *P, const double *Gin, double *Gs,
         double *dR1, T *J1, const double *__restrict__ met, const double *__restrict__ sig,
         const Defer df, unsigned long long *stats)
{
    const Grid &G = K.G;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const Bricks bk = make_bricks(G.n);
    int i, j, k;
    const bool active = brick_coords(G, bk, t, i, j, k);
    int status = 0, iters = 0;
    long long c = 0;
    double u[NCO], pr[NPR], E[3], gp = 0.0, gv[3] = {0, 0, 0}, cc = 0.0;
    Met<double> m;
    PaperState ps;
    if (active) {
        c = cell_at(G, i, j, k);
        const long long S = G.S;
        load_metric<FLAT>(met, S, c, m);
        for (int f = 0; f < NCO; f++) u[f] = U[f * S + c];
        RecIn in;
        load_rec_in(u, in);
        cc = K.gimex * K.dt * m.alpha * sigma_cell(K, sig, c, in.D);
        gp = Gin[c];
        for (int a = 0; a < 3; a++) gv[a] = Gin[(1 + a) * S + c];
        status = recover<FLAT>(in, m, K.ro, true, cc, gp, gv, u[CO_PHI], u[CO_PSI], u[CO_Q], pr,
                               E, iters, df.cap ? REC_FIRST : REC_ALL, &ps);
    }
    const bool want = active && status == REC_DEFER;
    const int slot = defer_slot(df, want);
    if (want) {
        if (slot >= 0) {
            defer_store(df, slot, interior_index(G, i, j, k), u, gp, gv, ps);
        } else {
            RecIn in;
            load_rec_in(u, in);
            int it2 = 0;
            status = recover<FLAT>(in, m, K.ro, true, cc, gp, gv, u[CO_PHI], u[CO_PSI], u[CO_Q],
                                   pr, E, it2, REC_ALL);
            iters = it2;
        }
    }
    const bool deferred = want && slot >= 0;
    if (active && !deferred) stage1_write(K, c, pr, E, u, m.alpha, P, Gs, dR1, J1);
    record_stats(stats, active, status, deferred ? 0 : iters, !deferred);
}

// Stage 2: U* = U^n + dt F[U1] + (1-2gamma) Dt R1 on calE; implicit recovery
// (guess P1); V = U^n + dt/2 F[U1] + dt/2 (R1 + R2) (Eq. IMEX3 minus F[U2]).
// Us (optional): U* is also written there.
template <bool FLAT, class T>
__global__ void __launch_bounds__(128, 4)
k_stage2(const StepConst K, const double *__restrict__ U, const T *__restrict__ P1,
         const double *__restrict__ G1, const T *__restrict__ Fx, const T *__restrict__ Fy,
         const T *__restrict__ Fz, const double *__restrict__ dR1,
         const double *__restrict__ met, const double *__restrict__ sig, T *P2, double *G2,
         double *V, T *J2, const Defer df, unsigned long long *stats, double *Us)
{
    const Grid &G = K.G;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const Bricks bk = make_bricks(G.n);
    int i, j, k;
    const bool active = brick_coords(G, bk, t, i, j, k);
    int status = 0, iters = 0;
    long long c = 0;
    double us[NCO], p2[NPR], E[3], gp = 0.0, gv[3] = {0, 0, 0}, cc = 0.0;
    Met<double> m;
    PaperState ps;
    if (active) {
        c = cell_at(G, i, j, k);
        const long long S = G.S;
        T pr[NPR];
        for (int f = 0; f < NPR; f++) pr[f] = P1[f * S + c];
        T r[NCO];
        rhs_cell<FLAT, T>(K, pr, met, Fx, Fy, Fz, c, r);
        const double dt = K.dt, hdt = 0.5 * dt;
        for (int f = 0; f < NCO; f++) {
            const double uu = U[f * S + c], rf = to_double<T>(r[f]);
            us[f] = uu + dt * rf;
            V[f * S + c] = uu + hdt * rf;
        }
        for (int a = 0; a < 3; a++) us[CO_EX + a] += (1.0 - 2.0 * K.gimex) * dR1[a * S + c];
        if (Us)   // the adjoint keeps the recovery input U*
            for (int f = 0; f < NCO; f++) Us[f * S + c] = us[f];
        load_metric<FLAT>(met, S, c, m);
        RecIn in;
        load_rec_in(us, in);
        cc = K.gimex * dt * m.alpha * sigma_cell(K, sig, c, in.D);
        gp = G1[c];
        for (int a = 0; a < 3; a++) gv[a] = G1[(1 + a) * S + c];
        status = recover<FLAT>(in, m, K.ro, true, cc, gp, gv, us[CO_PHI], us[CO_PSI], us[CO_Q],
                               p2, E, iters, df.cap ? REC_FIRST : REC_ALL, &ps);
    }
    const bool want = active && status == REC_DEFER;
    const int slot = defer_slot(df, want);
    if (want) {
        if (slot >= 0) {
            defer_store(df, slot, interior_index(G, i, j, k), us, gp, gv, ps);
        } else {
            RecIn in;
            load_rec_in(us, in);
            int it2 = 0;
            status = recover<FLAT>(in, m, K.ro, true, cc, gp, gv, us[CO_PHI], us[CO_PSI],
                                   us[CO_Q], p2, E, it2, REC_ALL);
            iters = it2;
        }
    }
    const bool deferred = want && slot >= 0;
    if (active && !deferred) stage2_write(K, c, p2, E, us, m.alpha, dR1, P2, G2, V, J2);
    record_stats(stats, active, status, deferred ? 0 : iters, !deferred);
}

// Final: U^{n+1} = V + dt/2 F[U2]; recovery with calE fixed (guess P2).
template <bool FLAT, class T>
__global__ void __launch_bounds__(128, 4)
k_final(const StepConst K, const double *__restrict__ Vb, const T *__restrict__ P2,
        const double *__restrict__ G2, const T *__restrict__ Fx, const T *__restrict__ Fy,
        const T *__restrict__ Fz, const double *__restrict__ met, double *U, T *P, double *Gs,
        const Defer df, unsigned long long *stats)
{
    const Grid &G = K.G;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const Bricks bk = make_bricks(G.n);
    int i, j, k;
    const bool active = brick_coords(G, bk, t, i, j, k);
    int status = 0, iters = 0;
    long long c = 0;
    double un[NCO], pn[NPR], E[3], gp = 0.0, gv[3] = {0, 0, 0};
    Met<double> m;
    PaperState ps;
    if (active) {
        c = cell_at(G, i, j, k);
        const long long S = G.S;
        T pr[NPR];
        for (int f = 0; f < NPR; f++) pr[f] = P2[f * S + c];
        T r[NCO];
        rhs_cell<FLAT, T>(K, pr, met, Fx, Fy, Fz, c, r);
        const double hdt = 0.5 * K.dt;
        bool finite = true;
        for (int f = 0; f < NCO; f++) {
            un[f] = Vb[f * S + c] + hdt * to_double<T>(r[f]);
            finite = finite && isfinite(un[f]);
            U[f * S + c] = un[f];
        }
        if (!finite) atomicOr((unsigned long long *)&stats[ST_NAN], 1ULL);
        load_metric<FLAT>(met, S, c, m);
        RecIn in;
        load_rec_in(un, in);
        gp = G2[c];
        for (int a = 0; a < 3; a++) gv[a] = G2[(1 + a) * S + c];
        status = recover<FLAT>(in, m, K.ro, false, 0.0, gp, gv, un[CO_PHI], un[CO_PSI],
                               un[CO_Q], pn, E, iters, df.cap ? REC_FIRST : REC_ALL, &ps);
    }
    const bool want = active && status == REC_DEFER;
    const int slot = defer_slot(df, want);
    if (want) {
        if (slot >= 0) {
            defer_store(df, slot, interior_index(G, i, j, k), un, gp, gv, ps);
        } else {
            RecIn in;
            load_rec_in(un, in);
            int it2 = 0;
            status = recover<FLAT>(in, m, K.ro, false, 0.0, gp, gv, un[CO_PHI], un[CO_PSI],
                                   un[CO_Q], pn, E, it2, REC_ALL);
            iters = it2;
        }
    }
    const bool deferred = want && slot >= 0;
    if (active && !deferred) final_write<FLAT>(K, c, pn, status, m, U, P, Gs);
    record_stats(stats, active, status, deferred ? 0 : iters, !deferred);
}

// Primitives of a conserved state given alone (checkpoint restore): the
// recovery with calE fixed (Sec. III.B) at every interior cell, the guess
// (p, v^i) from Gin when given (the handle's current primitives), else
// v = 0 and the pressure of the state's energy density at rest,
// p = (Gamma-1) max(tau / sqrt(gamma) - (E^2 + B^2)/2, 0) (the atmosphere
// pressure if that is zero).  A cell whose recovery fails is reset to the
// atmosphere as in a step (its D, S_i, tau replaced).  One thread per cell,
// the whole recovery inline.
template <bool FLAT, class T>
__global__ void __launch_bounds__(128)
k_recover_cons(const StepConst K, double *U, const double *__restrict__ met,
               const double *Gin, T *P, double *Gs, unsigned long long *stats)
{
    const Grid &G = K.G;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const bool active = t < G.N;
    int status = 0, iters = 0;
    if (active) {
        int i, j, k;
        interior_coords(G, t, i, j, k);
        const long long c = cell_at(G, i, j, k);
        const long long S = G.S;
        Met<double> m;
        load_metric<FLAT>(met, S, c, m);
        double u[NCO];
        for (int f = 0; f < NCO; f++) u[f] = U[f * S + c];
        RecIn in;
        load_rec_in(u, in);
        double gp, gv[3] = {0.0, 0.0, 0.0};
        if (Gin) {
            gp = Gin[c];
            for (int a = 0; a < 3; a++) gv[a] = Gin[(1 + a) * S + c];
        } else {
            double El[3], Bl[3];
            lower<double, FLAT>(m, in.cE0, El);
            lower<double, FLAT>(m, in.cB, Bl);
            const double isg = FLAT ? 1.0 : m.isg;
            const double em = 0.5 * (dot3(in.cE0, El) + dot3(in.cB, Bl)) * isg * isg;
            const double e = in.tau * isg - em;
            gp = e > 0.0 ? (K.ro.Gam - 1.0) * e : K.ro.p_atmo;
            if (!(gp > 0.0)) gp = K.ro.p_atmo > 0.0 ? K.ro.p_atmo : 1e-300;
        }
        double pn[NPR], E[3];
        status = recover<FLAT>(in, m, K.ro, false, 0.0, gp, gv, u[CO_PHI], u[CO_PSI], u[CO_Q],
                               pn, E, iters, REC_ALL);
        final_write<FLAT>(K, c, pn, status, m, U, P, Gs);
    }
    record_stats(stats, active, status, iters);
}

// One row of the general IMEX-RK form (Sec. III.A) for the tableaux other
// than Table imex, at one cell: u = U^n + dt sum_q aF_q F_q, and on calE
// also + sum_q aR_q Dt R_q.  F_jnew (jnew >= 0, coefficient anew) is formed
// here from the face fluxes of its stage (primitives Pp) and, if a later row
// needs it (store), kept in Fst; the other F_q, those whose bit is set in
// fmask, come from Fst, and the Dt R_q of the bits of rmask (the nonzero
// coefficients: the FP64 pipe does no compares).
struct ImexRow {
    double aF[4], aR[4], anew;
    int fmask, rmask, jnew, store;
};

template <bool FLAT, class T>
__device__ __forceinline__ void row_combine(const StepConst &K, const ImexRow &row,
                                            const double *U, const T *__restrict__ Pp,
                                            const T *__restrict__ Fx, const T *__restrict__ Fy,
                                            const T *__restrict__ Fz,
                                            const double *__restrict__ met, double *Fst,
                                            const double *__restrict__ dRs, long long c,
                                            double u[NCO])
{
    const long long S = K.G.S;
    double acc[NCO];
#pragma unroll
    for (int f = 0; f < NCO; f++) acc[f] = 0.0;
    if (row.jnew >= 0) {
        T pr[NPR], r[NCO];
        for (int f = 0; f < NPR; f++) pr[f] = Pp[f * S + c];
        rhs_cell<FLAT, T>(K, pr, met, Fx, Fy, Fz, c, r);
        double *Fn = Fst + (long long)row.jnew * NCO * S + c;
#pragma unroll
        for (int f = 0; f < NCO; f++) {
            const double rf = to_double<T>(r[f]);
            if (row.store) Fn[f * S] = rf;
            acc[f] = row.anew * rf;
        }
    }
#pragma unroll
    for (int q = 0; q < 4; q++) {
        if (!((row.fmask >> q) & 1)) continue;
        const double a = row.aF[q];
#pragma unroll
        for (int f = 0; f < NCO; f++) acc[f] += a * Fst[((long long)q * NCO + f) * S + c];
    }
#pragma unroll
    for (int f = 0; f < NCO; f++) u[f] = U[f * S + c] + K.dt * acc[f];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        if (!((row.rmask >> q) & 1)) continue;
#pragma unroll
        for (int a = 0; a < 3; a++) u[CO_EX + a] += row.aR[q] * dRs[((long long)q * 3 + a) * S + c];
    }
}

// Stage i >= 2 of the general form: its explicit part (row i of the
// tableaux, F of stage i-1 formed here), then the implicit part solved with
// the recovery (K.gimex = A_ii, guess: stage i-1's primitives Gp) -> the
// stage's primitives P, guess Gs, Dt R_i and current J.
template <bool FLAT, class T>
__global__ void __launch_bounds__(128, 4)
k_stage_row(const StepConst K, const ImexRow row, const double *__restrict__ U,
            const T *__restrict__ Pp, const double *__restrict__ Gp, const T *__restrict__ Fx,
            const T *__restrict__ Fy, const T *__restrict__ Fz, double *Fst,
            const double *__restrict__ dRs, const double *__restrict__ met,
            const double *__restrict__ sig, T *P, double *Gs, double *dRi, T *J, const Defer df,
            unsigned long long *stats)
{
    const Grid &G = K.G;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const Bricks bk = make_bricks(G.n);
    int i, j, k;
    const bool active = brick_coords(G, bk, t, i, j, k);
    int status = 0, iters = 0;
    long long c = 0;
    double us[NCO], pr[NPR], E[3], gp = 0.0, gv[3] = {0, 0, 0}, cc = 0.0;
    Met<double> m;
    PaperState ps;
    if (active) {
        c = cell_at(G, i, j, k);
        const long long S = G.S;
        row_combine<FLAT, T>(K, row, U, Pp, Fx, Fy, Fz, met, Fst, dRs, c, us);
        load_metric<FLAT>(met, S, c, m);
        RecIn in;
        load_rec_in(us, in);
        cc = K.gimex * K.dt * m.alpha * sigma_cell(K, sig, c, in.D);
        gp = Gp[c];
        for (int a = 0; a < 3; a++) gv[a] = Gp[(1 + a) * S + c];
        status = recover<FLAT>(in, m, K.ro, true, cc, gp, gv, us[CO_PHI], us[CO_PSI], us[CO_Q],
                               pr, E, iters, df.cap ? REC_FIRST : REC_ALL, &ps);
    }
    const bool want = active && status == REC_DEFER;
    const int slot = defer_slot(df, want);
    if (want) {
        if (slot >= 0) {
            defer_store(df, slot, interior_index(G, i, j, k), us, gp, gv, ps);
        } else {
            RecIn in;
            load_rec_in(us, in);
            int it2 = 0;
            status = recover<FLAT>(in, m, K.ro, true, cc, gp, gv, us[CO_PHI], us[CO_PSI],
                                   us[CO_Q], pr, E, it2, REC_ALL);
            iters = it2;
        }
    }
    const bool deferred = want && slot >= 0;
    if (active && !deferred) stage1_write(K, c, pr, E, us, m.alpha, P, Gs, dRi, J);
    record_stats(stats, active, status, deferred ? 0 : iters, !deferred);
}

// Final of the general form: U^{n+1} from the weights row (F of the last
// stage formed here), written over U^n in place (each cell reads its own
// U^n first); recovery with calE fixed (guess: the last stage's primitives).
template <bool FLAT, class T>
__global__ void __launch_bounds__(128, 4)
k_final_row(const StepConst K, const ImexRow row, const T *__restrict__ Pp,
            const double *__restrict__ Gp, const T *__restrict__ Fx, const T *__restrict__ Fy,
            const T *__restrict__ Fz, double *Fst, const double *__restrict__ dRs,
            const double *__restrict__ met, double *U, T *P, double *Gs, const Defer df,
            unsigned long long *stats)
{
    const Grid &G = K.G;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const Bricks bk = make_bricks(G.n);
    int i, j, k;
    const bool active = brick_coords(G, bk, t, i, j, k);
    int status = 0, iters = 0;
    long long c = 0;
    double un[NCO], pn[NPR], E[3], gp = 0.0, gv[3] = {0, 0, 0};
    Met<double> m;
    PaperState ps;
    if (active) {
        c = cell_at(G, i, j, k);
        const long long S = G.S;
        row_combine<FLAT, T>(K, row, U, Pp, Fx, Fy, Fz, met, Fst, dRs, c, un);
        bool finite = true;
        for (int f = 0; f < NCO; f++) {
            finite = finite && isfinite(un[f]);
            U[f * S + c] = un[f];
        }
        if (!finite) atomicOr((unsigned long long *)&stats[ST_NAN], 1ULL);
        load_metric<FLAT>(met, S, c, m);
        RecIn in;
        load_rec_in(un, in);
        gp = Gp[c];
        for (int a = 0; a < 3; a++) gv[a] = Gp[(1 + a) * S + c];
        status = recover<FLAT>(in, m, K.ro, false, 0.0, gp, gv, un[CO_PHI], un[CO_PSI],
                               un[CO_Q], pn, E, iters, df.cap ? REC_FIRST : REC_ALL, &ps);
    }
    const bool want = active && status == REC_DEFER;
    const int slot = defer_slot(df, want);
    if (want) {
        if (slot >= 0) {
            defer_store(df, slot, interior_index(G, i, j, k), un, gp, gv, ps);
        } else {
            RecIn in;
            load_rec_in(un, in);
            int it2 = 0;
            status = recover<FLAT>(in, m, K.ro, false, 0.0, gp, gv, un[CO_PHI], un[CO_PSI],
                                   un[CO_Q], pn, E, it2, REC_ALL);
            iters = it2;
        }
    }
    const bool deferred = want && slot >= 0;
    if (active && !deferred) final_write<FLAT>(K, c, pn, status, m, U, P, Gs);
    record_stats(stats, active, status, deferred ? 0 : iters, !deferred);
}

// Deferred pass of stage 1 (STAGE 1), stage 2 (STAGE 2) or the final
// recovery (STAGE 3): one thread per record, fallbacks only.  The loop bound
// is uniform across a warp so that record_stats sees every lane.
template <bool FLAT, int STAGE, class T>
__global__ void __launch_bounds__(128)
k_deferred(const StepConst K, const Defer df, const double *__restrict__ met,
           const double *__restrict__ sig, const double *__restrict__ dR1, T *P, double *Gs,
           double *dRo, T *J, double *V, double *U, unsigned long long *stats)
{
    const Grid &G = K.G;
    const int n = min(*df.count, df.cap);
    const long long cap = df.cap;
    for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const int s = base + threadIdx.x;
        const bool active = s < n;
        int status = 0, iters = 0;
        if (active) {
            const long long t = df.idx[s];
            int i, j, k;
            interior_coords(G, t, i, j, k);
            const long long c = cell_at(G, i, j, k);
            double u[NCO], gv[3], pr[NPR], E[3];
            for (int f = 0; f < NCO; f++) u[f] = df.rec[f * cap + s];
            const double gp = df.rec[NCO * cap + s];
            for (int a = 0; a < 3; a++) gv[a] = df.rec[(NCO + 1 + a) * cap + s];
            PaperState ps;
            pstate_load(ps, df.rec + (NCO + 4) * cap + s, cap);
            Met<double> m;
            load_metric<FLAT>(met, G.S, c, m);
            RecIn in;
            load_rec_in(u, in);
            const bool implicit = STAGE != 3;
            const double cc =
                implicit ? K.gimex * K.dt * m.alpha * sigma_cell(K, sig, c, in.D) : 0.0;
            status = recover<FLAT>(in, m, K.ro, implicit, cc, gp, gv, u[CO_PHI], u[CO_PSI],
                                   u[CO_Q], pr, E, iters, REC_RESUME_NEWTON, &ps);
            if (status == REC_HARD) {
                // the pressure bracket on a whole warp (next pass)
                pstate_save(ps, df.rec + (NCO + 4) * cap + s, cap);
            } else {
                if (STAGE == 1) stage1_write(K, c, pr, E, u, m.alpha, P, Gs, dRo, J);
                if (STAGE == 2) stage2_write(K, c, pr, E, u, m.alpha, dR1, P, Gs, V, J);
                if (STAGE == 3) final_write<FLAT>(K, c, pr, status, m, U, P, Gs);
            }
        }
        const bool hard = active && status == REC_HARD;
        const unsigned mask = __ballot_sync(0xffffffffu, hard);
        if (mask) {
            const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
            int hb = 0;
            if (lane == leader) hb = atomicAdd(df.hcount, __popc(mask));
            hb = __shfl_sync(0xffffffffu, hb, leader);
            if (hard) df.hidx[hb + __popc(mask & ((1u << lane) - 1u))] = s;
        }
        record_stats(stats, active && !hard, status, iters);
    }
}

// The records whose paper iteration and both Newton methods failed: one warp
// per record runs the pressure bracket (recover's warp-cooperative form,
// every lane on the same record; lane 0 writes).  These are few (states
// without a root, hard fronts) and each is long, so the warp's lanes
// shorten the latency of the one record instead of running 32 records side
// by side.
template <bool FLAT, int STAGE, class T>
__global__ void __launch_bounds__(128)
k_deferred_hard(const StepConst K, const Defer df, const double *__restrict__ met,
                const double *__restrict__ sig, const double *__restrict__ dR1, T *P,
                double *Gs, double *dRo, T *J, double *V, double *U,
                unsigned long long *stats)
{
    const Grid &G = K.G;
    const int n = *df.hcount;
    const long long cap = df.cap;
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < n; w += warps) {
        const int s = df.hidx[w];
        const long long t = df.idx[s];
        int i, j, k;
        interior_coords(G, t, i, j, k);
        const long long c = cell_at(G, i, j, k);
        double u[NCO], gv[3], pr[NPR], E[3];
        for (int f = 0; f < NCO; f++) u[f] = df.rec[f * cap + s];
        const double gp = df.rec[NCO * cap + s];
        for (int a = 0; a < 3; a++) gv[a] = df.rec[(NCO + 1 + a) * cap + s];
        PaperState ps;
        pstate_load(ps, df.rec + (NCO + 4) * cap + s, cap);
        Met<double> m;
        load_metric<FLAT>(met, G.S, c, m);
        RecIn in;
        load_rec_in(u, in);
        const bool implicit = STAGE != 3;
        const double cc = implicit ? K.gimex * K.dt * m.alpha * sigma_cell(K, sig, c, in.D) : 0.0;
        int iters = 0;
        const int status = recover<FLAT, true>(in, m, K.ro, implicit, cc, gp, gv, u[CO_PHI],
                                               u[CO_PSI], u[CO_Q], pr, E, iters,
                                               REC_CHAIN_REST, &ps);
        if (lane == 0) {
            if (STAGE == 1) stage1_write(K, c, pr, E, u, m.alpha, P, Gs, dRo, J);
            if (STAGE == 2) stage2_write(K, c, pr, E, u, m.alpha, dR1, P, Gs, V, J);
            if (STAGE == 3) final_write<FLAT>(K, c, pr, status, m, U, P, Gs);
        }
        record_stats(stats, lane == 0, status, iters);
    }
}

// explicit right-hand side only (testing entry point)
template <bool FLAT, class T>
__global__ void k_rhs(const StepConst K, const T *__restrict__ P, const T *__restrict__ Fx,
                      const T *__restrict__ Fy, const T *__restrict__ Fz,
                      const double *__restrict__ met, double *out)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= K.G.N) return;
    int i, j, k;
    interior_coords(K.G, t, i, j, k);
    const long long c = cell_at(K.G, i, j, k), S = K.G.S;
    T pr[NPR], r[NCO];
    for (int f = 0; f < NPR; f++) pr[f] = P[f * S + c];
    rhs_cell<FLAT, T>(K, pr, met, Fx, Fy, Fz, c, r);
    for (int f = 0; f < NCO; f++) out[f * K.G.N + t] = (double)r[f];
}


} // namespace rmhd
