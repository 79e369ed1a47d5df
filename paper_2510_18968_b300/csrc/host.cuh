// host.cuh -- host-side state of a solver handle (device buffers, step
// constants, captured step graph, adjoint recording) and the small helpers
// every translation unit of the library shares: error text, argument
// staging, ghost fills.  The stage sequencing of a step lives in
// step_impl.cuh, compiled once per (metric, precision) combination.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "../../include/rmhd.h"
#include "kernels.cuh"

using namespace rmhd;

namespace rmhd_host {

const int TPB = 128;
const int NDEFER = 8;   // deferred-recovery counters: one per recovery of a step

// text of the calling thread's last error of a call without a handle
extern thread_local char g_noh_err[512];

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
    int *dcount = nullptr, *didx = nullptr;   // dcount: NDEFER list counters, then NDEFER
    int *hidx = nullptr;                      // counters of the warp-per-record lists
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

inline Tableau tableau(int scheme)
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
inline bool f_needed(const Tableau &T, int j)
{
    bool need = T.wt[j] != 0.0;
    for (int k = j + 1; k < T.s; k++) need = need || T.At[k][j] != 0.0;
    return need;
}

inline bool f_stored(const Tableau &T, int j)
{
    bool keep = j < T.s - 1 && T.wt[j] != 0.0;
    for (int k = j + 2; k < T.s; k++) keep = keep || T.At[k][j] != 0.0;
    return keep;
}

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

inline void free_adj(AdjBuf &a)
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

} // namespace rmhd_host

using namespace rmhd_host;

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

// events of a profiled step of the general form: the time between two
// consecutive marks is added to the group (RMHD_NPROF index) of the later
struct ProfMarks {
    static const int MAX = 48;
    cudaEvent_t ev[MAX];
    int grp[MAX];
    int n = 0;
};

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


// ------------------------------------------------------ step sequencing
// Defined in step_impl.cuh and instantiated for every (FLAT, T) in the
// step_*.cu files, so that the heavy kernel templates of one combination
// compile in a translation unit of their own.
template <bool FLAT, class T> void enqueue_stages12_t(rmhd_t h, cudaEvent_t *ev, double *Us);
template <bool FLAT, class T> void enqueue_final_t(rmhd_t h, cudaEvent_t *ev);
template <bool FLAT, class T> void enqueue_step_t(rmhd_t h, cudaEvent_t *ev);
template <bool FLAT, class T> void enqueue_general_t(rmhd_t h, ProfMarks *pm);
template <bool FLAT, class T> void launch_recover_cons(rmhd_t h, bool guess);
template <bool FLAT, class T> void launch_rhs(rmhd_t h, const T *P, const T *J);

// one step of the handle's scheme, metric and precision
static inline void enqueue_step(rmhd_t h, cudaEvent_t *ev = nullptr, ProfMarks *pm = nullptr)
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
