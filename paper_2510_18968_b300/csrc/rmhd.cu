// rmhd.cu -- host side of the C ABI declared in include/rmhd.h: parameter
// checks, device memory, stage sequencing of the IMEX-SSP2(2,2,2) step
// (arXiv:2510.18968 Sec. III.A, Eq. IMEX3) and of the general IMEX-RK form
// for the other SSP tableaux, and the testing entry points.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "../../include/rmhd.h"
#include "adjoint.cuh"
#include "kernels.cuh"

using namespace rmhd;

namespace {

const int TPB = 128;
const int NDEFER = 8;   // deferred-recovery counters: one per recovery of a step

char g_noh_err[512] = "";

struct Buffers {
    double *U = nullptr, *V = nullptr, *dR1 = nullptr;
    // explicit-path buffers in the path's storage type (8 or 4 bytes)
    void *PA = nullptr, *PB = nullptr, *J1 = nullptr, *J2 = nullptr;
    void *F[3] = {nullptr, nullptr, nullptr};
    // FP64 recovery guess (p, v^i); aliases fields 1..4 of PA / PB on FP64
    double *GA = nullptr, *GB = nullptr;
    bool own_guess = false;
    double *met = nullptr, *sig = nullptr, *stage = nullptr;
    unsigned long long *stats = nullptr;
    int *flag = nullptr;
    // deferred-recovery work lists (scratch): counters for the three
    // recoveries of a step, cell indices and records
    int *dcount = nullptr, *didx = nullptr;
    double *drec = nullptr;
    int dcap = 0;
    // general IMEX form (schemes other than Table imex): the F of earlier
    // stages that later rows use (NCO x S each, slot j = stage j) and every
    // stage's Dt R (3 x S each)
    double *Fst = nullptr, *dRs = nullptr;
};

// Double Butcher tableaux of the IMEX-RK schemes (Sec. III.A).  Table imex
// (scheme 0) is printed in the paper; schemes 1-3 are the SSP schemes it
// lists in Sec. I, with the coefficients published by Pareschi and Russo
// (J. Sci. Comput. 25, 2005).
struct Tableau {
    int s = 0;
    double At[4][4] = {}, wt[4] = {}, A[4][4] = {}, w[4] = {};
};

Tableau tableau(int scheme)
{
    Tableau T;
    const double g = 1.0 - 1.0 / sqrt(2.0);
    if (scheme == RMHD_IMEX_SSP222) {
        T.s = 2;
        T.At[1][0] = 1.0;
        T.A[0][0] = g;
        T.A[1][0] = 1.0 - 2.0 * g;
        T.A[1][1] = g;
        T.wt[0] = T.wt[1] = 0.5;
    } else if (scheme == RMHD_IMEX_SSP2332) {
        T.s = 3;
        T.At[1][0] = T.At[2][0] = T.At[2][1] = 0.5;
        T.A[0][0] = T.A[1][1] = 0.25;
        T.A[2][0] = T.A[2][1] = T.A[2][2] = 1.0 / 3.0;
        T.wt[0] = T.wt[1] = T.wt[2] = 1.0 / 3.0;
    } else if (scheme == RMHD_IMEX_SSP3332) {
        T.s = 3;
        T.At[1][0] = 1.0;
        T.At[2][0] = T.At[2][1] = 0.25;
        T.A[0][0] = T.A[1][1] = T.A[2][2] = g;
        T.A[1][0] = 1.0 - 2.0 * g;
        T.A[2][0] = 0.5 - g;
        T.wt[0] = T.wt[1] = 1.0 / 6.0;
        T.wt[2] = 2.0 / 3.0;
    } else if (scheme == RMHD_IMEX_SSP3433) {
        const double a = 0.24169426078821, be = 0.06042356519705, et = 0.12915286960590;
        T.s = 4;
        T.At[2][1] = 1.0;
        T.At[3][1] = T.At[3][2] = 0.25;
        for (int i = 0; i < 4; i++) T.A[i][i] = a;
        T.A[1][0] = -a;
        T.A[2][1] = 1.0 - a;
        T.A[3][0] = be;
        T.A[3][1] = et;
        T.A[3][2] = 0.5 - be - et - a;
        T.wt[1] = T.wt[2] = 1.0 / 6.0;
        T.wt[3] = 2.0 / 3.0;
    }
    for (int i = 0; i < T.s; i++) T.w[i] = T.wt[i];   // every scheme here has w = wt
    return T;
}

// F of stage j is formed (its face fluxes computed) when a later row or
// the weights use it; kept in Fst when a row after the next one, or the
// weights (j < s-1), use it
bool f_needed(const Tableau &T, int j)
{
    bool need = T.wt[j] != 0.0;
    for (int k = j + 1; k < T.s; k++) need = need || T.At[k][j] != 0.0;
    return need;
}

bool f_stored(const Tableau &T, int j)
{
    bool keep = j < T.s - 1 && T.wt[j] != 0.0;
    for (int k = j + 2; k < T.s; k++) keep = keep || T.At[k][j] != 0.0;
    return keep;
}

} // namespace

namespace {

// recorded trajectory and scratch of the adjoint (FP64 path)
struct AdjBuf {
    bool recorded = false;
    bool full = false;   // every step's state and stage states kept (no re-runs)
    double dt = 0.0;
    int nsteps = 0, every = 0, nck = 0;
    double *ckU = nullptr, *ckP = nullptr;     // checkpoints: nck x (14 x S)
    double *segU = nullptr, *segP = nullptr;   // one segment: (every + 1) x (14 x S)
    // stage states of the segment's steps (every x: P1, P2, U* 14 x S; J1, J2 3 x S)
    double *segP1 = nullptr, *segJ1 = nullptr, *segUs = nullptr, *segP2 = nullptr,
           *segJ2 = nullptr;
    double *endU = nullptr, *endP = nullptr;   // state after the recorded steps
    double *lamU = nullptr, *lamUn = nullptr, *lamR1 = nullptr, *lamP = nullptr;
    double *lamJ = nullptr, *lamdR1 = nullptr;
    double *C = nullptr;   // per-face stencil contributions: 6 x 15 x S
    double *lsigc = nullptr;   // per-cell dL/dlog sigma0, summed at the end
    double *lsig = nullptr;
    int *bad = nullptr;
};

void free_adj(AdjBuf &a)
{
    double **ptrs[] = {&a.ckU,  &a.ckP,   &a.segU,  &a.segP,   &a.segP1, &a.segJ1,
                       &a.segUs, &a.segP2, &a.segJ2, &a.endU,   &a.endP,  &a.lamU,
                       &a.lamUn, &a.lamR1, &a.lamP,  &a.lamJ,   &a.lamdR1, &a.lsig,
                       &a.C,     &a.lsigc};
    for (double **q : ptrs)
        if (*q) {
            cudaFree(*q);
            *q = nullptr;
        }
    if (a.bad) cudaFree(a.bad);
    a.bad = nullptr;
    a.recorded = false;
}

} // namespace

// one step captured as a CUDA graph, replayed by rmhd_step (valid for the
// step constants and metric flag it was captured with)
struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    StepConst K;
    bool flat = true;
    int precision = -1;
};

struct rmhd_s {
    rmhd_params p;
    cudaStream_t st;
    StepConst K;
    Buffers b;
    AdjBuf adj;
    StepGraph graph;
    bool flat = true;
    bool have_state = false;
    long long steps = 0;
    char err[512];
};

static int set_err(rmhd_t h, int code, const char *fmt, ...)
{
    char *dst = h ? h->err : g_noh_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return code;
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return set_err(h, RMHD_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

static inline unsigned nblk(long long n) { return (unsigned)((n + TPB - 1) / TPB); }

extern "C" void rmhd_default_params(rmhd_params *p)
{
    memset(p, 0, sizeof(*p));
    for (int d = 0; d < 3; d++) {
        p->n[d] = 1;
        p->dx[d] = 1.0;
        p->bc[d] = RMHD_BC_PERIODIC;
    }
    p->recon = RMHD_RECON_MINMOD;
    p->precision = RMHD_PREC_FP64;
    p->gamma_eos = 2.0;
    p->kappa = 1.0;
    p->sigma_model = RMHD_SIGMA_UNIFORM;
    p->rho_atmo = 1e-10;
    p->K_atmo = 100.0;
    p->atmo_tol = 1e-2;
    p->c2p_tol = 1e-14;
    p->c2p_maxit = 100;
    p->c2p_wmax = 100.0;
    p->qflux_mode = RMHD_QFLUX_STAGE;
    p->imex = RMHD_IMEX_SSP222;
}

static int check_params(rmhd_t h, const rmhd_params *p)
{
    if (!p) return set_err(h, RMHD_EINVAL, "params is NULL");
    for (int d = 0; d < 3; d++) {
        if (p->n[d] < 1) return set_err(h, RMHD_EINVAL, "n[%d] = %d < 1", d, p->n[d]);
        if (!(p->dx[d] > 0.0)) return set_err(h, RMHD_EINVAL, "dx[%d] must be > 0", d);
        if (p->bc[d] != RMHD_BC_PERIODIC && p->bc[d] != RMHD_BC_OUTFLOW)
            return set_err(h, RMHD_EINVAL, "bc[%d] = %d unknown", d, p->bc[d]);
        if (p->n[d] > 1 && p->n[d] < 3 && p->bc[d] == RMHD_BC_PERIODIC)
            return set_err(h, RMHD_EINVAL, "periodic direction %d needs n >= 3", d);
    }
    {
        // every padded field, and 14 of them together, must be indexable in
        // 32 bits (kernel index arithmetic)
        double cells = 1.0;
        for (int d = 0; d < 3; d++) cells *= (double)(p->n[d] + (p->n[d] > 1 ? 7 : 1));
        if (cells * 2.0 >= 2147483648.0)
            return set_err(h, RMHD_EINVAL, "grid too large: %.0f padded cells", cells);
    }
    if (p->recon < 0 || p->recon > 2) return set_err(h, RMHD_EINVAL, "recon %d unknown", p->recon);
    if (p->precision != RMHD_PREC_FP64 && p->precision != RMHD_PREC_MIXED)
        return set_err(h, RMHD_EINVAL, "precision %d unknown", p->precision);
    if (!(p->gamma_eos > 1.0)) return set_err(h, RMHD_EINVAL, "gamma_eos must be > 1");
    if (p->sigma_model < 0 || p->sigma_model > 3)
        return set_err(h, RMHD_EINVAL, "sigma_model %d unknown", p->sigma_model);
    if (!(p->sigma0 >= 0.0)) return set_err(h, RMHD_EINVAL, "sigma0 must be >= 0");
    if (!(p->rho_atmo > 0.0) || !(p->K_atmo >= 0.0) || !(p->atmo_tol >= 0.0))
        return set_err(h, RMHD_EINVAL, "atmosphere parameters out of range");
    if (!(p->c2p_tol > 0.0) || p->c2p_maxit < 1 || !(p->c2p_wmax > 1.0))
        return set_err(h, RMHD_EINVAL, "recovery parameters out of range");
    if (p->c2p_first_pass < 0) return set_err(h, RMHD_EINVAL, "c2p_first_pass must be >= 0");
    if (p->qflux_mode != RMHD_QFLUX_STAGE && p->qflux_mode != RMHD_QFLUX_FACE_OHM &&
        p->qflux_mode != RMHD_QFLUX_GAUSS)
        return set_err(h, RMHD_EINVAL, "qflux_mode %d unknown", p->qflux_mode);
    if (p->imex < RMHD_IMEX_SSP222 || p->imex > RMHD_IMEX_SSP3433)
        return set_err(h, RMHD_EINVAL, "imex scheme %d unknown", p->imex);
    return RMHD_OK;
}

static RecOpts rec_opts(const rmhd_params *p)
{
    RecOpts o;
    o.Gam = p->gamma_eos;
    o.tol = p->c2p_tol;
    o.v2max = 1.0 - 1.0 / (p->c2p_wmax * p->c2p_wmax);
    o.rho_atmo = p->rho_atmo;
    o.p_atmo = p->K_atmo * pow(p->rho_atmo, p->gamma_eos);
    o.atmo_floor = p->rho_atmo * (1.0 + p->atmo_tol);
    o.maxit = p->c2p_maxit;
    o.first_cap = p->c2p_first_pass > 0 ? p->c2p_first_pass : p->c2p_maxit;
    return o;
}

static void free_all(Buffers &b)
{
    void **ptrs[] = {(void **)&b.U, &b.PA, &b.PB, (void **)&b.V, (void **)&b.dR1, &b.J1, &b.J2,
                     &b.F[0], &b.F[1], &b.F[2], (void **)&b.met, (void **)&b.sig,
                     (void **)&b.stage, (void **)&b.Fst, (void **)&b.dRs};
    for (void **q : ptrs)
        if (*q) {
            cudaFree(*q);
            *q = nullptr;
        }
    if (b.own_guess) {
        if (b.GA) cudaFree(b.GA);
        if (b.GB) cudaFree(b.GB);
    }
    b.GA = b.GB = nullptr;
    if (b.stats) cudaFree(b.stats);
    if (b.flag) cudaFree(b.flag);
    if (b.dcount) cudaFree(b.dcount);
    if (b.didx) cudaFree(b.didx);
    if (b.drec) cudaFree(b.drec);
    b.stats = nullptr;
    b.flag = nullptr;
    b.dcount = b.didx = nullptr;
    b.drec = nullptr;
}

// ------------------------------------------------------------------ launches

template <class T> static void launch_ghosts(rmhd_t h, T *buf, int nf)
{
    const Grid &G = h->K.G;
    long long mx = 0;
    for (int d = 0; d < 3; d++) {
        if (!G.g[d]) continue;
        long long c = 2LL * G.g[d] * G.n[(d + 1) % 3] * G.n[(d + 2) % 3];
        if (c > mx) mx = c;
    }
    if (!mx) return;
    dim3 grid(nblk(mx), 3);
    k_ghosts<T><<<grid, TPB, 0, h->st>>>(h->K, buf, nf, 0);
}

// FP32 face fluxes through shared-memory tiles: x faces by rows of 128
// (k_flux_tile); y and z faces by walking runs (k_flux_walk, blocks of 32
// x-lines x FB faces) for the TVD reconstructions, whose cell slopes the
// two faces of a cell share, by 32 x 16 tiles (k_flux_tile) for WENO5
template <bool FLAT, int RC>
static void launch_flux_tile(rmhd_t h, const float *P, const float *J, float **Fd)
{
    const Grid &G = h->K.G;
    const Buffers &b = h->b;
    const unsigned n0 = G.n[0], n1 = G.n[1], n2 = G.n[2];
    if (G.g[0])
        k_flux_tile<FLAT, RC, 0><<<dim3((n0 + 127) / 128, n1, n2), TPB, 0, h->st>>>(
            h->K, P, J, b.met, b.sig, Fd[0]);
    if constexpr (RC == RC_WENO5) {
        if (G.g[1])
            k_flux_tile<FLAT, RC, 1><<<dim3((n0 + 31) / 32, (n1 + 15) / 16, n2), TPB, 0, h->st>>>(
                h->K, P, J, b.met, b.sig, Fd[1]);
        if (G.g[2])
            k_flux_tile<FLAT, RC, 2><<<dim3((n0 + 31) / 32, n1, (n2 + 15) / 16), TPB, 0, h->st>>>(
                h->K, P, J, b.met, b.sig, Fd[2]);
    } else {
        if (G.g[1])
            k_flux_walk<FLAT, RC, 1><<<dim3((n0 + 31) / 32, (n1 + FB - 1) / FB, n2), TPB, 0,
                                       h->st>>>(h->K, P, J, b.met, b.sig, Fd[1]);
        if (G.g[2])
            k_flux_walk<FLAT, RC, 2><<<dim3((n0 + 31) / 32, n1, (n2 + FB - 1) / FB), TPB, 0,
                                       h->st>>>(h->K, P, J, b.met, b.sig, Fd[2]);
    }
}

// faces per thread of the run flux kernel (FP64 path)
const int FLUX_RUN = 8;

// FP64: the run kernel reconstructs each cell once (ALU-bound path); FP32:
// shared-memory tiles (k_flux_tile, k_flux_walk; one thread per face,
// k_flux, beyond the tiles' grid-dimension limits)
template <class T, bool FLAT, int RC>
static void launch_flux_rc(rmhd_t h, const T *P, const T *J)
{
    const Grid &G = h->K.G;
    const Buffers &b = h->b;
    T *Fd[3] = {(T *)b.F[0], (T *)b.F[1], (T *)b.F[2]};
    const int M = FLUX_RUN;
    const bool run = sizeof(T) == sizeof(double);
    auto nthreads = [&](int d) {
        long long n = 1;
        for (int a = 0; a < 3; a++) n *= a == d ? (run ? (G.n[a] + 1 + M - 1) / M : G.n[a] + 1) : G.n[a];
        return n;
    };
    if (run) {
        if (G.g[0]) k_flux_run<T, FLAT, RC, 0, M><<<nblk(nthreads(0)), TPB, 0, h->st>>>(h->K, P, J, b.met, b.sig, Fd[0]);
        if (G.g[1]) k_flux_run<T, FLAT, RC, 1, M><<<nblk(nthreads(1)), TPB, 0, h->st>>>(h->K, P, J, b.met, b.sig, Fd[1]);
        if (G.g[2]) k_flux_run<T, FLAT, RC, 2, M><<<nblk(nthreads(2)), TPB, 0, h->st>>>(h->K, P, J, b.met, b.sig, Fd[2]);
        return;
    }
    if (G.n[1] <= 65535 && G.n[2] <= 65535) {   // grid-dimension limits of the tiles
        launch_flux_tile<FLAT, RC>(h, (const float *)P, (const float *)J, (float **)Fd);
        return;
    }
    if (G.g[0]) k_flux<T, FLAT, RC, 0><<<nblk(nthreads(0)), TPB, 0, h->st>>>(h->K, P, J, b.met, b.sig, Fd[0]);
    if (G.g[1]) k_flux<T, FLAT, RC, 1><<<nblk(nthreads(1)), TPB, 0, h->st>>>(h->K, P, J, b.met, b.sig, Fd[1]);
    if (G.g[2]) k_flux<T, FLAT, RC, 2><<<nblk(nthreads(2)), TPB, 0, h->st>>>(h->K, P, J, b.met, b.sig, Fd[2]);
}

template <class T, bool FLAT> static void launch_flux(rmhd_t h, const T *P, const T *J)
{
    switch (h->p.recon) {
    case RMHD_RECON_MINMOD: launch_flux_rc<T, FLAT, RC_MINMOD>(h, P, J); break;
    case RMHD_RECON_MC2: launch_flux_rc<T, FLAT, RC_MC2>(h, P, J); break;
    default: launch_flux_rc<T, FLAT, RC_WENO5>(h, P, J); break;
    }
}

static Defer defer_of(rmhd_t h, int which)
{
    Defer d;
    d.count = h->b.dcount + which;
    d.cap = h->b.dcap;
    d.idx = h->b.didx;
    d.rec = h->b.drec;
    return d;
}

// Deferred passes: 64-thread blocks, enough of them for every record of a
// list of up to 148 * 96 * 64 (909 K) records to get its own thread, so that
// no thread takes a second record after its first (a fallback record can
// run for thousands of FP64 instructions); blocks past the list's count
// return at once.  Small blocks free their slot as soon as their two warps
// are done, which evens out the tail of the few long records.
const int TPB_DEFER = 64;
static unsigned deferred_blocks(rmhd_t h)
{
    long long want = (h->b.dcap + TPB_DEFER - 1) / TPB_DEFER;
    const long long most = 148LL * 96;
    return (unsigned)(want < most ? (want > 0 ? want : 1) : most);
}

// Gauss's-law charge of a stage (interior), then the ghosts of q
template <bool FLAT, class T> static void gauss_charge(rmhd_t h, T *P, double *U)
{
    k_gauss<FLAT, T><<<nblk(h->K.G.N), TPB, 0, h->st>>>(h->K, P, h->b.met, U);
    launch_ghosts(h, P + (size_t)PR_Q * h->K.G.S, 1);
}

// The step in two parts: stages 1 and 2 (up to P2, J2 with their ghosts),
// then the final assembly and recovery.  ev (optional): 9 events recorded
// between the kernel groups; Us (optional): U* of stage 2 is written there.
template <bool FLAT, class T>
static void enqueue_stages12_t(rmhd_t h, cudaEvent_t *ev, double *Us)
{
    Buffers &b = h->b;
    const StepConst &K = h->K;
    const unsigned nb = nblk(make_bricks(K.G.n).threads);   // stage kernels: bricks
    auto mark = [&](int i) { if (ev) cudaEventRecord(ev[i], h->st); };
    const bool dfr = b.dcap > 0;
    const unsigned nbd = deferred_blocks(h);
    T *PA = (T *)b.PA, *PB = (T *)b.PB, *J1 = (T *)b.J1, *J2 = (T *)b.J2;
    T *F0 = (T *)b.F[0], *F1 = (T *)b.F[1], *F2 = (T *)b.F[2];
    if (dfr) cudaMemsetAsync(b.dcount, 0, NDEFER * sizeof(int), h->st);
    mark(0);
    k_stage1<FLAT, T><<<nb, TPB, 0, h->st>>>(K, b.U, PA, b.GA, b.GA, b.dR1, J1, b.met, b.sig,
                                             defer_of(h, 0), b.stats);
    if (dfr)
        k_deferred<FLAT, 1, T><<<nbd, TPB_DEFER, 0, h->st>>>(K, defer_of(h, 0), b.met, b.sig, nullptr,
                                                       PA, b.GA, b.dR1, J1, nullptr, nullptr,
                                                       b.stats);
    mark(1);
    launch_ghosts(h, PA, NPR);
    if (K.qflux == RMHD_QFLUX_GAUSS) gauss_charge<FLAT, T>(h, PA, nullptr);
    if (K.qflux != 1) launch_ghosts(h, J1, 3);
    mark(2);
    launch_flux<T, FLAT>(h, PA, J1);
    mark(3);
    k_stage2<FLAT, T><<<nb, TPB, 0, h->st>>>(K, b.U, PA, b.GA, F0, F1, F2, b.dR1, b.met, b.sig,
                                             PB, b.GB, b.V, J2, defer_of(h, 1), b.stats, Us);
    if (dfr)
        k_deferred<FLAT, 2, T><<<nbd, TPB_DEFER, 0, h->st>>>(K, defer_of(h, 1), b.met, b.sig, b.dR1,
                                                       PB, b.GB, nullptr, J2, b.V, nullptr,
                                                       b.stats);
    mark(4);
    launch_ghosts(h, PB, NPR);
    if (K.qflux == RMHD_QFLUX_GAUSS) gauss_charge<FLAT, T>(h, PB, nullptr);
    if (K.qflux != 1) launch_ghosts(h, J2, 3);
    mark(5);
}

template <bool FLAT, class T> static void enqueue_final_t(rmhd_t h, cudaEvent_t *ev)
{
    Buffers &b = h->b;
    const StepConst &K = h->K;
    const unsigned nb = nblk(make_bricks(K.G.n).threads);
    auto mark = [&](int i) { if (ev) cudaEventRecord(ev[i], h->st); };
    const bool dfr = b.dcap > 0;
    const unsigned nbd = deferred_blocks(h);
    T *PA = (T *)b.PA, *PB = (T *)b.PB, *J2 = (T *)b.J2;
    T *F0 = (T *)b.F[0], *F1 = (T *)b.F[1], *F2 = (T *)b.F[2];
    launch_flux<T, FLAT>(h, PB, J2);
    mark(6);
    k_final<FLAT, T><<<nb, TPB, 0, h->st>>>(K, b.V, PB, b.GB, F0, F1, F2, b.met, b.U, PA, b.GA,
                                            defer_of(h, 2), b.stats);
    if (dfr)
        k_deferred<FLAT, 3, T><<<nbd, TPB_DEFER, 0, h->st>>>(K, defer_of(h, 2), b.met, b.sig, nullptr,
                                                       PA, b.GA, nullptr, nullptr, nullptr, b.U,
                                                       b.stats);
    mark(7);
    launch_ghosts(h, PA, NPR);
    if (K.qflux == RMHD_QFLUX_GAUSS) gauss_charge<FLAT, T>(h, PA, b.U);
    mark(8);
}

template <bool FLAT, class T> static void enqueue_step_t(rmhd_t h, cudaEvent_t *ev)
{
    enqueue_stages12_t<FLAT, T>(h, ev, nullptr);
    enqueue_final_t<FLAT, T>(h, ev);
}

// events of a profiled step of the general form: the time between two
// consecutive marks is added to the group (RMHD_NPROF index) of the later
struct ProfMarks {
    static const int MAX = 48;
    cudaEvent_t ev[MAX];
    int grp[MAX];
    int n = 0;
};

// One step of the general IMEX form (schemes other than Table imex).  Stage
// 1: k_stage1 with gimex = A_11 on U^n.  Stage i >= 2: k_stage_row forms
// the row's explicit part (F of stage i-1 from the face fluxes of its
// primitives) and solves the implicit part with the recovery (gimex = A_ii),
// writing the stage's primitives, Dt R_i and current.  The stages alternate
// between the two primitive buffers so that the last one lands in PB;
// k_final_row forms U^{n+1} from the weights in place and recovers it into
// PA.  The face fluxes of a stage are computed only when a later row or the
// weights use its F.
template <bool FLAT, class T> static void enqueue_general_t(rmhd_t h, ProfMarks *pm)
{
    Buffers &b = h->b;
    const StepConst &K = h->K;
    const Tableau tab = tableau(h->p.imex);
    const int s = tab.s;
    const long long S = K.G.S;
    const unsigned nb = nblk(make_bricks(K.G.n).threads);
    const bool dfr = b.dcap > 0;
    const unsigned nbd = deferred_blocks(h);
    auto mark = [&](int g) {
        if (pm && pm->n < ProfMarks::MAX) {
            pm->grp[pm->n] = g;
            cudaEventRecord(pm->ev[pm->n++], h->st);
        }
    };
    T *Pb[2] = {(T *)b.PA, (T *)b.PB};
    double *Gb[2] = {b.GA, b.GB};
    T *J = (T *)b.J1;
    T *F0 = (T *)b.F[0], *F1 = (T *)b.F[1], *F2 = (T *)b.F[2];
    if (dfr) cudaMemsetAsync(b.dcount, 0, NDEFER * sizeof(int), h->st);
    mark(-1);
    int prev = 0;   // buffer of the previous stage's primitives (P^n: PA)
    for (int i = 0; i < s; i++) {
        const int cur = (s - 1 - i) % 2 == 0 ? 1 : 0;
        StepConst Ki = K;
        Ki.gimex = tab.A[i][i];
        Ki.igimex = 1.0 / tab.A[i][i];
        double *dRi = b.dRs + (size_t)i * 3 * S;
        if (i == 0) {
            k_stage1<FLAT, T><<<nb, TPB, 0, h->st>>>(Ki, b.U, Pb[cur], Gb[prev], Gb[cur], dRi, J,
                                                     b.met, b.sig, defer_of(h, i), b.stats);
        } else {
            // F of stage i-1 is formed here when any row or the weights use
            // it (its own coefficient in this row may be zero); the earlier
            // F come from Fst
            ImexRow row = {};
            row.jnew = f_needed(tab, i - 1) ? i - 1 : -1;
            row.store = f_stored(tab, i - 1) ? 1 : 0;
            row.anew = tab.At[i][i - 1];
            for (int j = 0; j < i; j++) {
                row.aF[j] = tab.At[i][j];
                row.aR[j] = tab.A[i][j];
                row.fmask |= j != row.jnew && tab.At[i][j] != 0.0 ? 1 << j : 0;
                row.rmask |= tab.A[i][j] != 0.0 ? 1 << j : 0;
            }
            k_stage_row<FLAT, T><<<nb, TPB, 0, h->st>>>(Ki, row, b.U, Pb[prev], Gb[prev], F0, F1,
                                                        F2, b.Fst, b.dRs, b.met, b.sig, Pb[cur],
                                                        Gb[cur], dRi, J, defer_of(h, i), b.stats);
        }
        if (dfr)
            k_deferred<FLAT, 1, T><<<nbd, TPB_DEFER, 0, h->st>>>(Ki, defer_of(h, i), b.met, b.sig,
                                                           nullptr, Pb[cur], Gb[cur], dRi, J,
                                                           nullptr, nullptr, b.stats);
        mark(i == 0 ? 0 : 3);
        if (f_needed(tab, i)) {
            launch_ghosts(h, Pb[cur], NPR);
            if (K.qflux == RMHD_QFLUX_GAUSS) gauss_charge<FLAT, T>(h, Pb[cur], nullptr);
            if (K.qflux != RMHD_QFLUX_FACE_OHM) launch_ghosts(h, J, 3);
            mark(1);
            launch_flux<T, FLAT>(h, Pb[cur], J);
            mark(i < s - 1 ? 2 : 4);
        }
        prev = cur;
    }
    // U^{n+1} = U^n + dt sum_j wt_j F_j + sum_j w_j Dt R_j, F_{s-1} formed here
    ImexRow row = {};
    row.jnew = s - 1;
    row.store = 0;
    row.anew = tab.wt[s - 1];
    for (int j = 0; j < s; j++) {
        row.aF[j] = tab.wt[j];
        row.aR[j] = tab.w[j];
        row.fmask |= j != row.jnew && tab.wt[j] != 0.0 ? 1 << j : 0;
        row.rmask |= tab.w[j] != 0.0 ? 1 << j : 0;
    }
    k_final_row<FLAT, T><<<nb, TPB, 0, h->st>>>(K, row, Pb[prev], Gb[prev], F0, F1, F2, b.Fst,
                                                b.dRs, b.met, b.U, Pb[0], Gb[0], defer_of(h, s),
                                                b.stats);
    if (dfr)
        k_deferred<FLAT, 3, T><<<nbd, TPB_DEFER, 0, h->st>>>(K, defer_of(h, s), b.met, b.sig, nullptr,
                                                       Pb[0], Gb[0], nullptr, nullptr, nullptr,
                                                       b.U, b.stats);
    mark(5);
    launch_ghosts(h, Pb[0], NPR);
    if (K.qflux == RMHD_QFLUX_GAUSS) gauss_charge<FLAT, T>(h, Pb[0], b.U);
    mark(1);
}

static void enqueue_step(rmhd_t h, cudaEvent_t *ev = nullptr, ProfMarks *pm = nullptr)
{
    const bool mixed = h->p.precision == RMHD_PREC_MIXED;
    if (h->p.imex != RMHD_IMEX_SSP222) {
        if (h->flat) {
            if (mixed) enqueue_general_t<true, float>(h, pm);
            else enqueue_general_t<true, double>(h, pm);
        } else {
            if (mixed) enqueue_general_t<false, float>(h, pm);
            else enqueue_general_t<false, double>(h, pm);
        }
        return;
    }
    if (h->flat) {
        if (mixed) enqueue_step_t<true, float>(h, ev);
        else enqueue_step_t<true, double>(h, ev);
    } else {
        if (mixed) enqueue_step_t<false, float>(h, ev);
        else enqueue_step_t<false, double>(h, ev);
    }
}

// copy a caller array (interior SoA, nf fields) into the staging buffer
static int stage_in(rmhd_t h, const double *src, int nf, int on_device)
{
    size_t bytes = sizeof(double) * nf * (size_t)h->K.G.N;
    CK(cudaMemcpyAsync(h->b.stage, src, bytes,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
    return RMHD_OK;
}

static int stage_out(rmhd_t h, double *dst, int nf, int on_device)
{
    size_t bytes = sizeof(double) * nf * (size_t)h->K.G.N;
    CK(cudaMemcpyAsync(dst, h->b.stage, bytes,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
    if (!on_device) CK(cudaStreamSynchronize(h->st));
    return RMHD_OK;
}

static int read_flag(rmhd_t h, int *v)
{
    CK(cudaMemcpyAsync(v, h->b.flag, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    return RMHD_OK;
}

// staged interior FP64 primitives -> padded primitives of the path's type
// (+ FP64 guess), ghosts filled
static void scatter_prims(rmhd_t h, void *P, double *Gs)
{
    const unsigned nb = nblk(h->K.G.N);
    if (h->p.precision == RMHD_PREC_MIXED) {
        k_scatter_prims<float><<<nb, TPB, 0, h->st>>>(h->K, h->b.stage, (float *)P, Gs);
        launch_ghosts(h, (float *)P, NPR);
    } else {
        k_scatter_prims<double><<<nb, TPB, 0, h->st>>>(h->K, h->b.stage, (double *)P, Gs);
        launch_ghosts(h, (double *)P, NPR);
    }
}

static void gather_prims(rmhd_t h, const void *P, const double *Gs)
{
    const unsigned nb = nblk(h->K.G.N);
    if (h->p.precision == RMHD_PREC_MIXED)
        k_gather_prims<float><<<nb, TPB, 0, h->st>>>(h->K, (const float *)P, Gs, h->b.stage);
    else
        k_gather_prims<double><<<nb, TPB, 0, h->st>>>(h->K, (const double *)P, Gs, h->b.stage);
}

// ------------------------------------------------------------------ API

extern "C" int rmhd_create(const rmhd_params *p, void *cuda_stream, rmhd_t *out)
{
    rmhd_t h = nullptr;
    if (!out) return set_err(nullptr, RMHD_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = check_params(nullptr, p);
    if (rc) return rc;
    h = new rmhd_s();
    h->p = *p;
    h->err[0] = 0;
    h->st = (cudaStream_t)cuda_stream;
    StepConst &K = h->K;
    memset(&K, 0, sizeof(K));
    Grid &G = K.G;
    for (int d = 0; d < 3; d++) {
        G.n[d] = p->n[d];
        G.g[d] = p->n[d] > 1 ? 3 : 0;
        G.idx[d] = 1.0 / p->dx[d];
        G.bc[d] = p->bc[d];
    }
    G.px = G.n[0] + 2 * G.g[0];
    G.pxy = G.px * (G.n[1] + 2 * G.g[1]);
    G.S = (long long)G.pxy * (G.n[2] + 2 * G.g[2]);
    G.N = (long long)G.n[0] * G.n[1] * G.n[2];
    K.gimex = 1.0 - 1.0 / sqrt(2.0);
    K.igimex = 1.0 / K.gimex;
    const Tableau tab = tableau(p->imex);
    K.gfac = p->gamma_eos / (p->gamma_eos - 1.0);
    K.gfacf = (float)K.gfac;
    K.kappaf = (float)p->kappa;
    for (int d = 0; d < 3; d++) K.idxf[d] = (float)G.idx[d];
    K.kappa = p->kappa;
    K.sigma_model = p->sigma_model;
    K.sigma0 = p->sigma0;
    K.sigma0f = (float)p->sigma0;
    K.sigma_exp = p->sigma_exp;
    K.D_atmo = p->D_atmo;
    K.qflux = p->qflux_mode;
    K.ro = rec_opts(p);

    Buffers &b = h->b;
    const bool mixed = p->precision == RMHD_PREC_MIXED;
    const size_t fb = sizeof(double) * (size_t)G.S;
    const size_t fe = (mixed ? sizeof(float) : sizeof(double)) * (size_t)G.S;
    const bool general = p->imex != RMHD_IMEX_SSP222;
    const size_t nstore = tab.s - 1;   // Fst slot j holds F of stage j (j < s-1)
    struct { void **ptr; size_t bytes; } allocs[] = {
        {(void **)&b.U, fb * NCO}, {&b.PA, fe * NPR}, {&b.PB, fe * NPR},
        {(void **)&b.V, fb * NCO}, {(void **)&b.dR1, fb * 3}, {&b.J1, fe * 3},
        {&b.J2, fe * 3}, {&b.F[0], fe * NCO}, {&b.F[1], fe * NCO}, {&b.F[2], fe * NCO},
        {(void **)&b.met, fb * NMET}, {(void **)&b.sig, fb},
        {(void **)&b.GA, mixed ? fb * 4 : 0}, {(void **)&b.GB, mixed ? fb * 4 : 0},
        {(void **)&b.Fst, general ? fb * NCO * nstore : 0},
        {(void **)&b.dRs, general ? fb * 3 * tab.s : 0}};
    b.own_guess = mixed;
    for (auto &a : allocs) {
        if (a.bytes == 0) continue;
        cudaError_t e = cudaMalloc(a.ptr, a.bytes);
        if (e != cudaSuccess) {
            free_all(b);
            set_err(nullptr, RMHD_ENOMEM, "cudaMalloc of %zu bytes failed: %s", a.bytes,
                    cudaGetErrorString(e));
            delete h;
            return RMHD_ENOMEM;
        }
        cudaMemsetAsync(*a.ptr, 0, a.bytes, h->st);
    }
    if (!mixed) {
        // FP64: the guess is fields 1..4 (p, v^i) of the primitive buffers
        b.GA = (double *)b.PA + G.S;
        b.GB = (double *)b.PB + G.S;
    }
    if (cudaMalloc((void **)&b.stage, sizeof(double) * NPR * (size_t)G.N) != cudaSuccess ||
        cudaMalloc((void **)&b.stats, sizeof(unsigned long long) * NSTAT) != cudaSuccess ||
        cudaMalloc((void **)&b.flag, sizeof(int)) != cudaSuccess) {
        free_all(b);
        set_err(nullptr, RMHD_ENOMEM, "cudaMalloc of staging buffers failed");
        delete h;
        return RMHD_ENOMEM;
    }
    cudaMemsetAsync(b.stats, 0, sizeof(unsigned long long) * NSTAT, h->st);
    // deferred-recovery work list: room for half of the cells (a fuller list
    // falls back to inline recovery)
    {
        long long cap = G.N / 2;
        if (cap < 1024) cap = 1024;
        if (cap > (1LL << 30) / DREC) cap = (1LL << 30) / DREC;
        b.dcap = (int)cap;
        if (cudaMalloc((void **)&b.dcount, NDEFER * sizeof(int)) != cudaSuccess ||
            cudaMalloc((void **)&b.didx, sizeof(int) * (size_t)cap) != cudaSuccess ||
            cudaMalloc((void **)&b.drec, sizeof(double) * DREC * (size_t)cap) != cudaSuccess) {
            free_all(b);
            set_err(nullptr, RMHD_ENOMEM, "cudaMalloc of the recovery work list failed");
            delete h;
            return RMHD_ENOMEM;
        }
    }
    // flat metric, unit conductivity profile; the state comes from
    // rmhd_set_prims or rmhd_set_state
    rc = rmhd_set_metric(h, nullptr, nullptr, nullptr, nullptr, 0);
    if (!rc) rc = rmhd_set_sigma(h, nullptr, 0);
    if (rc) {
        free_all(b);
        delete h;
        return rc;
    }
    *out = h;
    return RMHD_OK;
}

// fill field f of a padded buffer with a constant (interior and ghosts)
__global__ void k_fill(double *a, long long n, double v)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < n) a[t] = v;
}

// flags any interior cell whose metric differs from flat space
__global__ void k_not_flat(const StepConst K, const double *__restrict__ met, int *flag)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= K.G.N) return;
    int i, j, k;
    interior_coords(K.G, t, i, j, k);
    const long long c = cell_at(K.G, i, j, k);
    const double flat[NMET] = {1, 0, 0, 0, 1, 0, 0, 1, 0, 1, 0, 0, 0, 0, 0, 0};
    for (int f = 0; f < NMET; f++)
        if (met[f * K.G.S + c] != flat[f]) {
            atomicOr(flag, 1);
            return;
        }
}

extern "C" int rmhd_set_metric(rmhd_t h, const double *alpha, const double *beta,
                               const double *gamma, const double *K4, int on_device)
{
    if (!h) return set_err(nullptr, RMHD_EINVAL, "handle is NULL");
    const Grid &G = h->K.G;
    const long long S = G.S;
    double *met = h->b.met;
    if (!alpha) {
        // flat space
        const double vals[NMET] = {1, 0, 0, 0, 1, 0, 0, 1, 0, 1, 0, 0, 0, 0, 0, 0};
        for (int f = 0; f < NMET; f++)
            k_fill<<<nblk(S), TPB, 0, h->st>>>(met + f * S, S, vals[f]);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(h->st));
        h->flat = true;
        return RMHD_OK;
    }
    if (!beta || !gamma || !K4) return set_err(h, RMHD_EINVAL, "beta, gamma and K are required");
    // stage the 16 fields through a temporary padded copy so that a rejected
    // metric leaves the current one in place
    double *tmp = nullptr;
    CK(cudaMalloc((void **)&tmp, sizeof(double) * NMET * (size_t)S));
    const double *src[4] = {alpha, beta, gamma, K4};
    const int nf[4] = {1, 3, 6, 6};
    int off = 0;
    int rc = RMHD_OK;
    for (int a = 0; a < 4 && !rc; a++) {
        rc = stage_in(h, src[a], nf[a], on_device);
        if (!rc) k_scatter<double><<<nblk(G.N), TPB, 0, h->st>>>(h->K, h->b.stage, tmp + off * S, nf[a]);
        off += nf[a];
    }
    if (!rc) {
        launch_ghosts(h, tmp, NMET);
        cudaMemsetAsync(h->b.flag, 0, sizeof(int), h->st);
        k_check_metric<<<nblk(G.N), TPB, 0, h->st>>>(h->K, tmp, h->b.flag);
        int bad = 0;
        rc = read_flag(h, &bad);
        if (!rc && bad) rc = set_err(h, RMHD_EINVAL, "metric rejected: alpha <= 0, gamma_ij not "
                                                     "positive definite, or non-finite values");
    }
    if (!rc) {
        cudaMemcpyAsync(met, tmp, sizeof(double) * NMET * (size_t)S, cudaMemcpyDeviceToDevice,
                        h->st);
        // a metric equal to flat space everywhere selects the flat kernels
        cudaMemsetAsync(h->b.flag, 0, sizeof(int), h->st);
        k_not_flat<<<nblk(G.N), TPB, 0, h->st>>>(h->K, tmp, h->b.flag);
        int curved = 1;
        rc = read_flag(h, &curved);
        h->flat = !rc && !curved;
    }
    cudaFree(tmp);
    return rc;
}

extern "C" int rmhd_set_sigma(rmhd_t h, const double *profile, int on_device)
{
    if (!h) return set_err(nullptr, RMHD_EINVAL, "handle is NULL");
    const Grid &G = h->K.G;
    if (!profile) {
        k_fill<<<nblk(G.S), TPB, 0, h->st>>>(h->b.sig, G.S, 1.0);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(h->st));
        return RMHD_OK;
    }
    int rc = stage_in(h, profile, 1, on_device);
    if (rc) return rc;
    cudaMemsetAsync(h->b.flag, 0, sizeof(int), h->st);
    k_check_finite<<<nblk(G.N), TPB, 0, h->st>>>(G.N, h->b.stage, h->b.flag);
    int bad = 0;
    // negative values: reuse the finiteness kernel on -x via a host check below
    rc = read_flag(h, &bad);
    if (rc) return rc;
    if (bad) return set_err(h, RMHD_EINVAL, "sigma profile has non-finite values");
    // negativity check on the staged copy (host side, small cost at set-up)
    {
        size_t n = (size_t)G.N;
        double *hb = (double *)malloc(sizeof(double) * n);
        if (!hb) return set_err(h, RMHD_ENOMEM, "host buffer");
        CK(cudaMemcpy(hb, h->b.stage, sizeof(double) * n, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < n; i++)
            if (hb[i] < 0.0) {
                free(hb);
                return set_err(h, RMHD_EINVAL, "sigma profile has negative values");
            }
        free(hb);
    }
    k_scatter<double><<<nblk(G.N), TPB, 0, h->st>>>(h->K, h->b.stage, h->b.sig, 1);
    launch_ghosts(h, h->b.sig, 1);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->st));
    return RMHD_OK;
}

extern "C" int rmhd_set_prims(rmhd_t h, const double *prims, int on_device)
{
    if (!h) return set_err(nullptr, RMHD_EINVAL, "handle is NULL");
    if (!prims) return set_err(h, RMHD_EINVAL, "prims is NULL");
    const Grid &G = h->K.G;
    int rc = stage_in(h, prims, NPR, on_device);
    if (rc) return rc;
    // conserved values into V first: validate before touching the state
    cudaMemsetAsync(h->b.flag, 0, sizeof(int), h->st);
    if (h->flat)
        k_prim2con<true><<<nblk(G.N), TPB, 0, h->st>>>(h->K, h->b.stage, h->b.met, h->b.V,
                                                       h->b.flag);
    else
        k_prim2con<false><<<nblk(G.N), TPB, 0, h->st>>>(h->K, h->b.stage, h->b.met, h->b.V,
                                                        h->b.flag);
    int bad = 0;
    rc = read_flag(h, &bad);
    if (rc) return rc;
    if (bad) return set_err(h, RMHD_EINVAL, "prims rejected: rho <= 0, p < 0, v^2 >= 1 or "
                                            "non-finite values");
    CK(cudaMemcpyAsync(h->b.U, h->b.V, sizeof(double) * NCO * (size_t)G.S,
                       cudaMemcpyDeviceToDevice, h->st));
    scatter_prims(h, h->b.PA, h->b.GA);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->st));
    h->have_state = true;
    return RMHD_OK;
}

extern "C" int rmhd_set_state(rmhd_t h, const double *cons, const double *prims, int on_device)
{
    if (!h) return set_err(nullptr, RMHD_EINVAL, "handle is NULL");
    if (!cons || !prims) return set_err(h, RMHD_EINVAL, "cons and prims are required");
    const Grid &G = h->K.G;
    int bad = 0, rc;
    // each array crosses the bus once; both are validated before anything
    // is committed: the conserved values wait in V (step scratch)
    rc = stage_in(h, cons, NCO, on_device);
    if (rc) return rc;
    cudaMemsetAsync(h->b.flag, 0, sizeof(int), h->st);
    k_check_finite<<<nblk(NCO * G.N), TPB, 0, h->st>>>(NCO * G.N, h->b.stage, h->b.flag);
    k_scatter<double><<<nblk(G.N), TPB, 0, h->st>>>(h->K, h->b.stage, h->b.V, NCO);
    rc = stage_in(h, prims, NPR, on_device);
    if (rc) return rc;
    k_check_finite<<<nblk(NPR * G.N), TPB, 0, h->st>>>(NPR * G.N, h->b.stage, h->b.flag);
    rc = read_flag(h, &bad);
    if (rc) return rc;
    if (bad) return set_err(h, RMHD_EINVAL, "state has non-finite values");
    CK(cudaMemcpyAsync(h->b.U, h->b.V, sizeof(double) * NCO * (size_t)G.S,
                       cudaMemcpyDeviceToDevice, h->st));
    scatter_prims(h, h->b.PA, h->b.GA);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->st));
    h->have_state = true;
    return RMHD_OK;
}

// The step as a CUDA graph: captured once on a private stream (a legacy
// default stream cannot be captured), then launched on the handle's stream.
// Re-captured when the step constants, the metric flag or the precision
// change.  Replaying it removes the per-kernel launch cost, which is what a
// step of a small grid (the 1D shocktube) is made of.
static int step_graph(rmhd_t h, cudaGraphExec_t *out)
{
    StepGraph &g = h->graph;
    if (g.exec && g.flat == h->flat && g.precision == h->p.precision &&
        memcmp(&g.K, &h->K, sizeof(StepConst)) == 0) {
        *out = g.exec;
        return RMHD_OK;
    }
    if (g.exec) {
        cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
    }
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaStream_t user = h->st;
    h->st = cs;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        enqueue_step(h);
        e = cudaStreamEndCapture(cs, &graph);
    }
    h->st = user;
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return set_err(h, RMHD_ECUDA, "step graph capture failed: %s", cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        g.exec = nullptr;
        return set_err(h, RMHD_ECUDA, "step graph instantiation failed: %s",
                       cudaGetErrorString(e));
    }
    g.K = h->K;
    g.flat = h->flat;
    g.precision = h->p.precision;
    *out = g.exec;
    return RMHD_OK;
}

extern "C" int rmhd_step(rmhd_t h, double dt, int nsteps, long long *fail_count)
{
    if (!h) return set_err(nullptr, RMHD_EINVAL, "handle is NULL");
    if (!(dt > 0.0) || !isfinite(dt)) return set_err(h, RMHD_EINVAL, "dt must be > 0");
    if (nsteps < 0) return set_err(h, RMHD_EINVAL, "nsteps must be >= 0");
    if (!h->have_state) return set_err(h, RMHD_EINVAL, "no state: call rmhd_set_prims first");
    h->K.dt = dt;
    h->K.idt = 1.0 / dt;
    unsigned long long before[NSTAT];
    if (fail_count) {
        CK(cudaMemcpyAsync(before, h->b.stats, sizeof(before), cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
    }
    if (nsteps >= 2) {
        cudaGraphExec_t exec = nullptr;
        int rc = step_graph(h, &exec);
        if (rc) return rc;
        for (int s = 0; s < nsteps; s++) CK(cudaGraphLaunch(exec, h->st));
    } else {
        for (int s = 0; s < nsteps; s++) enqueue_step(h);
    }
    CK(cudaGetLastError());
    h->steps += nsteps;
    if (!fail_count) return RMHD_OK;
    unsigned long long after[NSTAT];
    CK(cudaMemcpyAsync(after, h->b.stats, sizeof(after), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    *fail_count = (long long)(after[ST_FAIL] - before[ST_FAIL]);
    if (after[ST_NAN]) return set_err(h, RMHD_ENAN, "non-finite conserved values");
    if (*fail_count > 0)
        return set_err(h, RMHD_EC2P, "%lld recoveries reset to the atmosphere", *fail_count);
    return RMHD_OK;
}

extern "C" int rmhd_step_profiled(rmhd_t h, double dt, int nsteps, double ms[RMHD_NPROF])
{
    if (!h || !ms) return set_err(h, RMHD_EINVAL, "NULL argument");
    if (!(dt > 0.0) || !isfinite(dt) || nsteps < 0)
        return set_err(h, RMHD_EINVAL, "dt must be > 0 and nsteps >= 0");
    if (!h->have_state) return set_err(h, RMHD_EINVAL, "no state: call rmhd_set_prims first");
    h->K.dt = dt;
    h->K.idt = 1.0 / dt;
    for (int g = 0; g < RMHD_NPROF; g++) ms[g] = 0.0;
    if (h->p.imex != RMHD_IMEX_SSP222) {
        ProfMarks pm;
        for (int i = 0; i < ProfMarks::MAX; i++) CK(cudaEventCreate(&pm.ev[i]));
        int rc = RMHD_OK;
        for (int st = 0; st < nsteps && !rc; st++) {
            pm.n = 0;
            enqueue_step(h, nullptr, &pm);
            cudaError_t e = cudaEventSynchronize(pm.ev[pm.n - 1]);
            if (e != cudaSuccess) {
                rc = set_err(h, RMHD_ECUDA, "step failed: %s", cudaGetErrorString(e));
                break;
            }
            for (int k = 1; k < pm.n; k++) {
                float t = 0.f;
                cudaEventElapsedTime(&t, pm.ev[k - 1], pm.ev[k]);
                ms[pm.grp[k]] += t;
            }
        }
        for (int i = 0; i < ProfMarks::MAX; i++) cudaEventDestroy(pm.ev[i]);
        if (!rc) h->steps += nsteps;
        return rc;
    }
    cudaEvent_t ev[9];
    for (int i = 0; i < 9; i++) CK(cudaEventCreate(&ev[i]));
    int rc = RMHD_OK;
    for (int s = 0; s < nsteps && !rc; s++) {
        enqueue_step(h, ev);
        cudaError_t e = cudaEventSynchronize(ev[8]);
        if (e != cudaSuccess) {
            rc = set_err(h, RMHD_ECUDA, "step failed: %s", cudaGetErrorString(e));
            break;
        }
        // groups: stage1, ghosts, fluxes of stage 2, stage2, fluxes of the
        // final assembly, final
        const int from[RMHD_NPROF] = {0, 1, 2, 3, 5, 6};
        const int to[RMHD_NPROF] = {1, 2, 3, 4, 6, 7};
        for (int g = 0; g < RMHD_NPROF; g++) {
            float t = 0.f;
            cudaEventElapsedTime(&t, ev[from[g]], ev[to[g]]);
            ms[g] += t;
        }
        float t1 = 0.f, t2 = 0.f;
        cudaEventElapsedTime(&t1, ev[4], ev[5]);
        cudaEventElapsedTime(&t2, ev[7], ev[8]);
        ms[1] += t1 + t2;
    }
    for (int i = 0; i < 9; i++) cudaEventDestroy(ev[i]);
    if (!rc) h->steps += nsteps;
    return rc;
}

extern "C" int rmhd_get_prims(rmhd_t h, double *prims, int on_device)
{
    if (!h || !prims) return set_err(h, RMHD_EINVAL, "NULL argument");
    gather_prims(h, h->b.PA, h->b.GA);
    CK(cudaGetLastError());
    return stage_out(h, prims, NPR, on_device);
}

extern "C" int rmhd_get_cons(rmhd_t h, double *cons, int on_device)
{
    if (!h || !cons) return set_err(h, RMHD_EINVAL, "NULL argument");
    k_gather<<<nblk(h->K.G.N), TPB, 0, h->st>>>(h->K, h->b.U, h->b.stage, NCO);
    CK(cudaGetLastError());
    return stage_out(h, cons, NCO, on_device);
}

extern "C" int rmhd_get_stats(rmhd_t h, long long stats[8])
{
    if (!h || !stats) return set_err(h, RMHD_EINVAL, "NULL argument");
    unsigned long long s[NSTAT];
    CK(cudaMemcpyAsync(s, h->b.stats, sizeof(s), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    stats[0] = (long long)s[ST_CALLS];
    stats[1] = (long long)s[ST_ITERS];
    stats[2] = (long long)s[ST_FALLBACK];
    stats[3] = (long long)s[ST_FAIL];
    stats[4] = (long long)s[ST_FLOOR];
    stats[5] = (long long)s[ST_MAXIT];
    stats[6] = (long long)s[ST_NAN];
    stats[7] = h->steps;
    return RMHD_OK;
}

template <class T> static int rhs_t(rmhd_t h, const double *J, int on_device)
{
    const Grid &G = h->K.G;
    T *J2 = (T *)h->b.J2, *PB = (T *)h->b.PB;
    T *F0 = (T *)h->b.F[0], *F1 = (T *)h->b.F[1], *F2 = (T *)h->b.F[2];
    if (J) {
        int rc = stage_in(h, J, 3, on_device);
        if (rc) return rc;
        k_scatter<T><<<nblk(G.N), TPB, 0, h->st>>>(h->K, h->b.stage, J2, 3);
    } else {
        CK(cudaMemsetAsync(J2, 0, sizeof(T) * 3 * (size_t)G.S, h->st));
    }
    launch_ghosts(h, J2, 3);
    if (h->flat) {
        launch_flux<T, true>(h, PB, J2);
        k_rhs<true, T><<<nblk(G.N), TPB, 0, h->st>>>(h->K, PB, F0, F1, F2, h->b.met, h->b.stage);
    } else {
        launch_flux<T, false>(h, PB, J2);
        k_rhs<false, T><<<nblk(G.N), TPB, 0, h->st>>>(h->K, PB, F0, F1, F2, h->b.met, h->b.stage);
    }
    return RMHD_OK;
}

extern "C" int rmhd_rhs(rmhd_t h, const double *prims, const double *J, double *rhs,
                        int on_device)
{
    if (!h || !prims || !rhs) return set_err(h, RMHD_EINVAL, "NULL argument");
    int rc = stage_in(h, prims, NPR, on_device);
    if (rc) return rc;
    scatter_prims(h, h->b.PB, h->b.GB);
    if (h->p.precision == RMHD_PREC_MIXED) rc = rhs_t<float>(h, J, on_device);
    else rc = rhs_t<double>(h, J, on_device);
    if (rc) return rc;
    CK(cudaGetLastError());
    return stage_out(h, rhs, NCO, on_device);
}

extern "C" int rmhd_con2prim_points(const rmhd_params *p, int npts, const double *cons,
                                    const double *guess, const double *alpha,
                                    const double *gamma, const double *sigma, int implicit,
                                    double c, double *prim, double *cons_out, int *iters,
                                    int *status, void *cuda_stream)
{
    rmhd_t h = nullptr;
    if (!p) return set_err(h, RMHD_EINVAL, "params is NULL");
    if (npts < 0) return set_err(h, RMHD_EINVAL, "npts < 0");
    if (npts == 0) return RMHD_OK;
    if (!cons || !guess || !alpha || !gamma || !prim || !cons_out || !iters || !status ||
        (implicit && !sigma))
        return set_err(h, RMHD_EINVAL, "NULL array");
    if (!(p->gamma_eos > 1.0) || !(p->c2p_tol > 0.0) || p->c2p_maxit < 1 || !(p->c2p_wmax > 1.0))
        return set_err(h, RMHD_EINVAL, "recovery parameters out of range");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    k_recover_points<<<nblk(npts), TPB, 0, st>>>(rec_opts(p), npts, cons, guess, alpha, gamma,
                                                 sigma, implicit, c,
                                                 p->gamma_eos / (p->gamma_eos - 1.0), prim,
                                                 cons_out, iters, status);
    CK(cudaGetLastError());
    return RMHD_OK;
}

// ------------------------------------------------------------------ adjoint

extern "C" int rmhd_set_sigma0(rmhd_t h, double sigma0)
{
    if (!h) return set_err(nullptr, RMHD_EINVAL, "handle is NULL");
    if (!(sigma0 >= 0.0) || !isfinite(sigma0)) return set_err(h, RMHD_EINVAL, "sigma0 must be >= 0");
    h->p.sigma0 = sigma0;
    h->K.sigma0 = sigma0;
    h->K.sigma0f = (float)sigma0;
    return RMHD_OK;
}

static size_t fbytes(rmhd_t h, int nf) { return sizeof(double) * nf * (size_t)h->K.G.S; }

// copy the FP64 state (U, P with the guess fields) to / from a slot
static int save_state(rmhd_t h, double *U, double *P)
{
    CK(cudaMemcpyAsync(U, h->b.U, fbytes(h, NCO), cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(P, h->b.PA, fbytes(h, NPR), cudaMemcpyDeviceToDevice, h->st));
    return RMHD_OK;
}
static int load_state(rmhd_t h, const double *U, const double *P)
{
    CK(cudaMemcpyAsync(h->b.U, U, fbytes(h, NCO), cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(h->b.PA, P, fbytes(h, NPR), cudaMemcpyDeviceToDevice, h->st));
    return RMHD_OK;
}

template <bool FLAT> static void launch_adj_flux(rmhd_t h, const double *P, const double *J,
                                                 const double *lamR, double scale)
{
    const Grid &G = h->K.G;
    AdjBuf &a = h->adj;
    auto nfaces = [&](int d) {
        long long n = 1;
        for (int q = 0; q < 3; q++) n *= q == d ? G.n[q] + 1 : G.n[q];
        return n;
    };
#define RMHD_ADJ_FLUX(RC)                                                                   \
    do {                                                                                    \
        if (G.g[0]) {                                                                       \
            k_adj_flux<FLAT, RC, 0><<<nblk(nfaces(0)), TPB, 0, h->st>>>(                    \
                h->K, P, J, h->b.met, lamR, scale, a.C);                                    \
            k_adj_gather<0><<<nblk(G.N), TPB, 0, h->st>>>(h->K, a.C, a.lamP, a.lamJ);       \
        }                                                                                   \
        if (G.g[1]) {                                                                       \
            k_adj_flux<FLAT, RC, 1><<<nblk(nfaces(1)), TPB, 0, h->st>>>(                    \
                h->K, P, J, h->b.met, lamR, scale, a.C);                                    \
            k_adj_gather<1><<<nblk(G.N), TPB, 0, h->st>>>(h->K, a.C, a.lamP, a.lamJ);       \
        }                                                                                   \
        if (G.g[2]) {                                                                       \
            k_adj_flux<FLAT, RC, 2><<<nblk(nfaces(2)), TPB, 0, h->st>>>(                    \
                h->K, P, J, h->b.met, lamR, scale, a.C);                                    \
            k_adj_gather<2><<<nblk(G.N), TPB, 0, h->st>>>(h->K, a.C, a.lamP, a.lamJ);       \
        }                                                                                   \
    } while (0)
    switch (h->p.recon) {
    case RMHD_RECON_MINMOD: RMHD_ADJ_FLUX(RC_MINMOD); break;
    case RMHD_RECON_MC2: RMHD_ADJ_FLUX(RC_MC2); break;
    default: RMHD_ADJ_FLUX(RC_WENO5); break;
    }
#undef RMHD_ADJ_FLUX
}

// events bracketing the kernel groups of the backward sweep (profiling)
struct AdjTimer {
    bool on = false;
    cudaStream_t st = nullptr;
    struct Mark {
        cudaEvent_t a, b;
        int g;
    };
    Mark m[4096];
    int n = 0;
    int open = -1;
    void begin(int g)
    {
        if (!on || n >= 4096) return;
        cudaEventCreate(&m[n].a);
        cudaEventCreate(&m[n].b);
        m[n].g = g;
        cudaEventRecord(m[n].a, st);
        open = n++;
    }
    void end()
    {
        if (!on || open < 0) return;
        cudaEventRecord(m[open].b, st);
        open = -1;
    }
    void collect(double *ms)
    {
        for (int g = 0; g < RMHD_NADJPROF; g++) ms[g] = 0.0;
        for (int i = 0; i < n; i++) {
            float t = 0.f;
            cudaEventElapsedTime(&t, m[i].a, m[i].b);
            ms[m[i].g] += t;
            cudaEventDestroy(m[i].a);
            cudaEventDestroy(m[i].b);
        }
        n = 0;
    }
};

// stage states of one recorded step (slot q of the segment)
struct StageSlot {
    const double *U, *P1, *J1, *Us, *P2, *J2;
};

static StageSlot stage_slot(rmhd_t h, int q)
{
    const AdjBuf &a = h->adj;
    const size_t S = (size_t)h->K.G.S;
    return {a.segU + (size_t)q * NCO * S, a.segP1 + (size_t)q * NPR * S,
            a.segJ1 + (size_t)q * 3 * S,  a.segUs + (size_t)q * NCO * S,
            a.segP2 + (size_t)q * NPR * S, a.segJ2 + (size_t)q * 3 * S};
}

// lamU <- dL/dU^n from lamU = dL/dU^{n+1}, from the stage states of step n
template <bool FLAT>
static int adjoint_step_t(rmhd_t h, const StageSlot &q, const double *Pnext, AdjTimer &tm)
{
    AdjBuf &a = h->adj;
    Buffers &b = h->b;
    const StepConst &K = h->K;
    const unsigned nb = nblk(K.G.N);
    // cells the final recovery reset keep no derivative in D, S_i, tau
    k_adj_reset_mask<<<nb, TPB, 0, h->st>>>(K, Pnext, a.lamU);
    const double *P1 = q.P1, *P2 = q.P2, *J1 = q.J1, *J2 = q.J2;
    // F(P2, J2) entered U^{n+1} with weight dt/2
    tm.begin(RMHD_ADJ_SOURCES);
    k_adj_sources<FLAT><<<nb, TPB, 0, h->st>>>(K, P2, b.met, a.lamU, 0.5 * K.dt, a.lamP);
    CK(cudaMemsetAsync(a.lamJ, 0, fbytes(h, 3), h->st));
    tm.end();
    tm.begin(RMHD_ADJ_FLUX);
    launch_adj_flux<FLAT>(h, P2, J2, a.lamU, 0.5 * K.dt);
    tm.end();
    tm.begin(RMHD_ADJ_STAGES);
    k_adj_stage2<FLAT><<<nb, TPB, 0, h->st>>>(K, q.Us, P2, b.met, b.sig, a.lamU, a.lamP, a.lamJ,
                                              a.lamR1, a.lamdR1, a.lamUn, a.lsigc, a.bad);
    tm.end();
    // F(P1, J1): its adjoint is lamR1
    tm.begin(RMHD_ADJ_SOURCES);
    k_adj_sources<FLAT><<<nb, TPB, 0, h->st>>>(K, P1, b.met, a.lamR1, 1.0, a.lamP);
    CK(cudaMemsetAsync(a.lamJ, 0, fbytes(h, 3), h->st));
    tm.end();
    tm.begin(RMHD_ADJ_FLUX);
    launch_adj_flux<FLAT>(h, P1, J1, a.lamR1, 1.0);
    tm.end();
    tm.begin(RMHD_ADJ_STAGES);
    k_adj_stage1<FLAT><<<nb, TPB, 0, h->st>>>(K, q.U, P1, b.met, b.sig, a.lamP, a.lamJ, a.lamdR1,
                                              a.lamUn, a.lsigc, a.bad);
    tm.end();
    double *t = a.lamU;
    a.lamU = a.lamUn;
    a.lamUn = t;
    CK(cudaGetLastError());
    return RMHD_OK;
}

// one FP64 step that keeps its state (U^n, P^n) and its stage states in
// segment slot q; with final = false the step stops after stage 2
static int record_step(rmhd_t h, int q, bool final = true)
{
    AdjBuf &a = h->adj;
    const size_t S = (size_t)h->K.G.S;
    int rc = save_state(h, a.segU + (size_t)q * NCO * S, a.segP + (size_t)q * NPR * S);
    if (rc) return rc;
    if (h->flat) enqueue_stages12_t<true, double>(h, nullptr, a.segUs + (size_t)q * NCO * S);
    else enqueue_stages12_t<false, double>(h, nullptr, a.segUs + (size_t)q * NCO * S);
    CK(cudaMemcpyAsync(a.segP1 + (size_t)q * NPR * S, h->b.PA, fbytes(h, NPR),
                       cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(a.segJ1 + (size_t)q * 3 * S, h->b.J1, fbytes(h, 3),
                       cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(a.segP2 + (size_t)q * NPR * S, h->b.PB, fbytes(h, NPR),
                       cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(a.segJ2 + (size_t)q * 3 * S, h->b.J2, fbytes(h, 3),
                       cudaMemcpyDeviceToDevice, h->st));
    if (final) {
        if (h->flat) enqueue_final_t<true, double>(h, nullptr);
        else enqueue_final_t<false, double>(h, nullptr);
    }
    return RMHD_OK;
}

extern "C" int rmhd_adjoint_forward(rmhd_t h, double dt, int nsteps, int checkpoint_every)
{
    if (!h) return set_err(nullptr, RMHD_EINVAL, "handle is NULL");
    if (!(dt > 0.0) || !isfinite(dt)) return set_err(h, RMHD_EINVAL, "dt must be > 0");
    if (nsteps < 1 || checkpoint_every < 0)
        return set_err(h, RMHD_EINVAL, "nsteps must be >= 1 and checkpoint_every >= 0");
    if (!h->have_state) return set_err(h, RMHD_EINVAL, "no state: call rmhd_set_prims first");
    if (h->p.precision != RMHD_PREC_FP64)
        return set_err(h, RMHD_EINVAL, "the adjoint needs precision RMHD_PREC_FP64");
    if (h->p.qflux_mode != RMHD_QFLUX_STAGE)
        return set_err(h, RMHD_EINVAL, "the adjoint needs qflux_mode RMHD_QFLUX_STAGE");
    if (h->p.imex != RMHD_IMEX_SSP222)
        return set_err(h, RMHD_EINVAL, "the adjoint needs imex RMHD_IMEX_SSP222");
    for (int d = 0; d < 3; d++)
        if (h->K.G.g[d] && h->K.G.n[d] < 3)
            return set_err(h, RMHD_EINVAL, "the adjoint needs n >= 3 in active directions");
    AdjBuf &a = h->adj;
    free_adj(a);
    a.dt = dt;
    a.nsteps = nsteps;
    a.full = checkpoint_every == 0;
    a.every = a.full || checkpoint_every > nsteps ? nsteps : checkpoint_every;
    a.nck = (nsteps + a.every - 1) / a.every;
    const size_t u = fbytes(h, NCO), pz = fbytes(h, NPR);
    struct {
        double **p;
        size_t n;
    } al[] = {{&a.ckU, a.nck * u},       {&a.ckP, a.nck * pz},   {&a.segU, (a.every + 1) * u},
              {&a.segP, (a.every + 1) * pz}, {&a.endU, u},       {&a.endP, pz},
              {&a.lamU, u},              {&a.lamUn, u},          {&a.lamR1, u},
              {&a.lamP, pz},             {&a.lamJ, fbytes(h, 3)}, {&a.lamdR1, fbytes(h, 3)},
              {&a.segP1, a.every * pz},  {&a.segJ1, a.every * fbytes(h, 3)},
              {&a.segUs, a.every * u},   {&a.segP2, a.every * pz},
              {&a.segJ2, a.every * fbytes(h, 3)}, {&a.lsig, sizeof(double)},
              {&a.C, fbytes(h, ADJ_SLOTS * ADJ_NF)}, {&a.lsigc, fbytes(h, 1)}};
    for (auto &e : al) {
        cudaError_t err = cudaMalloc((void **)e.p, e.n);
        if (err != cudaSuccess) {
            free_adj(a);
            return set_err(h, RMHD_ENOMEM, "adjoint buffers: %s", cudaGetErrorString(err));
        }
        CK(cudaMemsetAsync(*e.p, 0, e.n, h->st));
    }
    CK(cudaMalloc((void **)&a.bad, sizeof(int)));
    h->K.dt = dt;
    h->K.idt = 1.0 / dt;
    for (int n = 0; n < nsteps; n++) {
        if (n % a.every == 0) {
            int rc = save_state(h, a.ckU + (size_t)(n / a.every) * NCO * h->K.G.S,
                                a.ckP + (size_t)(n / a.every) * NPR * h->K.G.S);
            if (rc) return rc;
        }
        if (a.full) {
            // the whole tape: the state and the stage states of every step
            int rc = record_step(h, n);
            if (rc) return rc;
        } else {
            enqueue_step(h);
        }
    }
    int rc = save_state(h, a.endU, a.endP);
    if (rc) return rc;
    CK(cudaGetLastError());
    unsigned long long st[NSTAT];
    CK(cudaMemcpyAsync(st, h->b.stats, sizeof(st), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    h->steps += nsteps;
    if (st[ST_NAN]) return set_err(h, RMHD_ENAN, "non-finite conserved values");
    a.recorded = true;
    return RMHD_OK;
}

extern "C" int rmhd_adjoint_backward(rmhd_t h, const double *lam_prims, double *grad_prims0,
                                     double *grad_log_sigma0, int on_device,
                                     double ms[RMHD_NADJPROF])
{
    if (!h) return set_err(nullptr, RMHD_EINVAL, "handle is NULL");
    AdjBuf &a = h->adj;
    if (!a.recorded) return set_err(h, RMHD_EINVAL, "no recorded steps: call rmhd_adjoint_forward");
    if (!lam_prims || !grad_prims0) return set_err(h, RMHD_EINVAL, "NULL array");
    const StepConst &K = h->K;
    const Grid &G = K.G;
    const size_t S = (size_t)G.S;
    const unsigned nb = nblk(G.N);
    h->K.dt = a.dt;
    h->K.idt = 1.0 / a.dt;
    static thread_local AdjTimer tm;
    tm.on = ms != nullptr;
    tm.st = h->st;
    tm.n = 0;
    unsigned long long stats0[NSTAT];
    CK(cudaMemcpyAsync(stats0, h->b.stats, sizeof(stats0), cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemsetAsync(a.lsigc, 0, fbytes(h, 1), h->st));
    CK(cudaMemsetAsync(a.bad, 0, sizeof(int), h->st));
    CK(cudaMemsetAsync(a.lamU, 0, fbytes(h, NCO), h->st));
    CK(cudaMemsetAsync(a.lamUn, 0, fbytes(h, NCO), h->st));
    // dL/dP^N -> dL/dU^N through the last recovery
    int rc = stage_in(h, lam_prims, NPR, on_device);
    if (rc) return rc;
    CK(cudaMemsetAsync(a.lamP, 0, fbytes(h, NPR), h->st));
    k_scatter<double><<<nb, TPB, 0, h->st>>>(h->K, h->b.stage, a.lamP, NPR);
    if (h->flat)
        k_adj_final<true><<<nb, TPB, 0, h->st>>>(h->K, a.endU, a.endP, h->b.met, a.lamP, a.lamU,
                                                 a.bad);
    else
        k_adj_final<false><<<nb, TPB, 0, h->st>>>(h->K, a.endU, a.endP, h->b.met, a.lamP,
                                                  a.lamU, a.bad);
    for (int seg = a.nck - 1; seg >= 0; seg--) {
        const int s0 = seg * a.every;
        const int s1 = s0 + a.every < a.nsteps ? s0 + a.every : a.nsteps;
        // states s0 .. s1-1 of the segment, then P^{s1}
        // re-run the segment from its checkpoint, keeping every step's
        // state and stage states (already kept when the whole tape is)
        if (!a.full) {
            tm.begin(RMHD_ADJ_RECOMPUTE);
            rc = load_state(h, a.ckU + (size_t)seg * NCO * S, a.ckP + (size_t)seg * NPR * S);
            if (rc) return rc;
            for (int n = s0; n < s1; n++) {
                rc = record_step(h, n - s0, n + 1 < s1);
                if (rc) return rc;
            }
            tm.end();
        }
        const double *Pend = seg + 1 < a.nck ? a.ckP + (size_t)(seg + 1) * NPR * S : a.endP;
        for (int n = s1 - 1; n >= s0; n--) {
            const double *Pnext = n + 1 == s1 ? Pend : a.segP + (size_t)(n + 1 - s0) * NPR * S;
            const StageSlot q = stage_slot(h, n - s0);
            rc = h->flat ? adjoint_step_t<true>(h, q, Pnext, tm)
                         : adjoint_step_t<false>(h, q, Pnext, tm);
            if (rc) return rc;
        }
    }
    // U^0 = prim2con(P^0)
    if (h->flat)
        k_adj_prim2con<true><<<nb, TPB, 0, h->st>>>(h->K, a.ckP, h->b.met, a.lamU, h->b.stage);
    else
        k_adj_prim2con<false><<<nb, TPB, 0, h->st>>>(h->K, a.ckP, h->b.met, a.lamU,
                                                     h->b.stage);
    rc = stage_out(h, grad_prims0, NPR, on_device);
    if (rc) return rc;
    k_adj_sum<<<1, 1024, 0, h->st>>>(h->K, a.lsigc, a.lsig);
    double ls = 0.0;
    int bad = 0;
    CK(cudaMemcpyAsync(&ls, a.lsig, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(&bad, a.bad, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    // the recorded end state and the statistics are left as the forward left them
    rc = load_state(h, a.endU, a.endP);   // the FP64 guess lives in P
    if (rc) return rc;
    CK(cudaMemcpyAsync(h->b.stats, stats0, sizeof(stats0), cudaMemcpyHostToDevice, h->st));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    if (grad_log_sigma0) *grad_log_sigma0 = ls;
    if (ms) tm.collect(ms);
    if (bad) return set_err(h, RMHD_ENAN, "singular recovery Jacobian in the adjoint");
    return RMHD_OK;
}

// ------------------------------------------------------------------ testing

__global__ void k_test_rcp64(long long n, const double *__restrict__ x, double *out)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < n) out[t] = rcp64(x[t]);
}

extern "C" int rmhd_test_rcp64(const double *x, double *out, long long n, void *cuda_stream)
{
    if (n < 0 || (n > 0 && (!x || !out))) return set_err(nullptr, RMHD_EINVAL, "bad arguments");
    if (n == 0) return RMHD_OK;
    k_test_rcp64<<<nblk(n), TPB, 0, (cudaStream_t)cuda_stream>>>(n, x, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_err(nullptr, RMHD_ECUDA, "launch failed: %s", cudaGetErrorString(e));
    return RMHD_OK;
}

__global__ void k_test_mm3(long long n, const double *__restrict__ a,
                           const double *__restrict__ b, const double *__restrict__ c,
                           double *out)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < n) out[t] = mm3<double>(a[t], b[t], c[t]);
}

extern "C" int rmhd_test_mm3(const double *a, const double *b, const double *c, double *out,
                             long long n, void *cuda_stream)
{
    if (n < 0 || (n > 0 && (!a || !b || !c || !out)))
        return set_err(nullptr, RMHD_EINVAL, "bad arguments");
    if (n == 0) return RMHD_OK;
    k_test_mm3<<<nblk(n), TPB, 0, (cudaStream_t)cuda_stream>>>(n, a, b, c, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_err(nullptr, RMHD_ECUDA, "launch failed: %s", cudaGetErrorString(e));
    return RMHD_OK;
}

__global__ void k_test_mm3f(long long n, const float *__restrict__ a,
                            const float *__restrict__ b, const float *__restrict__ c,
                            float *out)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < n) out[t] = mm3<float>(a[t], b[t], c[t]);
}

extern "C" int rmhd_test_mm3f(const float *a, const float *b, const float *c, float *out,
                              long long n, void *cuda_stream)
{
    if (n < 0 || (n > 0 && (!a || !b || !c || !out)))
        return set_err(nullptr, RMHD_EINVAL, "bad arguments");
    if (n == 0) return RMHD_OK;
    k_test_mm3f<<<nblk(n), TPB, 0, (cudaStream_t)cuda_stream>>>(n, a, b, c, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_err(nullptr, RMHD_ECUDA, "launch failed: %s", cudaGetErrorString(e));
    return RMHD_OK;
}

extern "C" const char *rmhd_last_error(rmhd_t h) { return h ? h->err : g_noh_err; }

// error text of an entry point without a handle (used by the other source file)
__attribute__((visibility("hidden"))) void rmhd_internal_set_error(const char *msg)
{
    snprintf(g_noh_err, sizeof g_noh_err, "%s", msg);
}

extern "C" int rmhd_destroy(rmhd_t h)
{
    if (!h) return RMHD_OK;
    cudaStreamSynchronize(h->st);
    if (h->graph.exec) cudaGraphExecDestroy(h->graph.exec);
    free_adj(h->adj);
    free_all(h->b);
    delete h;
    return RMHD_OK;
}
