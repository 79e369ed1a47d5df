// step_impl.cuh -- stage sequencing of one step on the handle's stream
// (arXiv:2510.18968 Sec. III.A: Table imex / Eq. IMEX3, and the general
// IMEX-RK form for the other SSP tableaux), the face-flux launches, the
// whole-grid recovery of rmhd_set_cons and the right-hand side of
// rmhd_rhs.  Included by the step_*.cu files only, each of which
// instantiates these templates for one (metric, precision) combination.
#pragma once
#include "host.cuh"

// FP32 face fluxes through shared-memory tiles: for the TVD reconstructions,
// whose cell slopes the two faces of a cell share, x faces by walking warps
// (k_flux_xwalk, segments of 128 faces of four rows) and y and z faces by
// walking runs (k_flux_walk, blocks of 32 x-lines x FB faces); for WENO5 x
// faces by rows of 128 (k_flux_tile) and y, z faces by 32 x 16 tiles
// Tensor maps of the stage's primitives (14 fields) and of J^D for the tile
// copies of one flux kernel, boxes {bx, by, bz}; false (plain staging) when
// x is inactive or the driver refuses a map.
static bool flux_maps(rmhd_t h, const float *P, const float *J, int D, int bx, int by, int bz,
                      CUtensorMap *tmP, CUtensorMap *tmJ)
{
    const Grid &G = h->K.G;
    memset(tmP, 0, sizeof(*tmP));
    memset(tmJ, 0, sizeof(*tmJ));
    if (G.g[0] != 3 || G.px % 4 != 0 || !P) return false;
    const int py = G.n[1] + 2 * G.g[1], pz = G.n[2] + 2 * G.g[2];
    if (!make_tile_map(tmP, P, G.px, py, pz, G.S, NPR, bx, by, bz)) return false;
    if (h->K.qflux != 1 && J && !make_tile_map(tmJ, J + (size_t)D * G.S, G.px, py, pz, G.S, 0,
                                               bx, by, bz))
        return false;
    g_tile_copy_launches.fetch_add(1);
    return true;
}

template <bool FLAT, int RC>
static void launch_flux_tile(rmhd_t h, const float *P, const float *J, float **Fd)
{
    const Grid &G = h->K.G;
    const Buffers &b = h->b;
    const unsigned n0 = G.n[0], n1 = G.n[1], n2 = G.n[2];
    CUtensorMap tmP, tmJ;
    if (G.g[0]) {
        if constexpr (RC != RC_WENO5) {
            const int tma = flux_maps(h, P, J, 0, XW_LX, XW_ROWS, 1, &tmP, &tmJ);
            k_flux_xwalk<FLAT, RC><<<dim3((n0 + 127) / 128, (n1 + XW_ROWS - 1) / XW_ROWS, n2), TPB,
                                     0, h->st>>>(h->K, P, J, b.met, b.sig, Fd[0], tmP, tmJ, tma,
                                                 b.stats);
        } else {
            const int tma = flux_maps(h, P, J, 0, 136, 1, 1, &tmP, &tmJ);
            k_flux_tile<FLAT, RC, 0><<<dim3((n0 + 127) / 128, n1, n2), TPB, 0, h->st>>>(
                h->K, P, J, b.met, b.sig, Fd[0], tmP, tmJ, tma, b.stats);
        }
    }
    if constexpr (RC == RC_WENO5) {
        if (G.g[1]) {
            const int tma = flux_maps(h, P, J, 1, 36, 22, 1, &tmP, &tmJ);
            k_flux_tile<FLAT, RC, 1><<<dim3((n0 + 31) / 32, (n1 + 15) / 16, n2), TPB, 0, h->st>>>(
                h->K, P, J, b.met, b.sig, Fd[1], tmP, tmJ, tma, b.stats);
        }
        if (G.g[2]) {
            const int tma = flux_maps(h, P, J, 2, 36, 1, 22, &tmP, &tmJ);
            k_flux_tile<FLAT, RC, 2><<<dim3((n0 + 31) / 32, n1, (n2 + 15) / 16), TPB, 0, h->st>>>(
                h->K, P, J, b.met, b.sig, Fd[2], tmP, tmJ, tma, b.stats);
        }
    } else {
        if (G.g[1]) {
            const int tma = flux_maps(h, P, J, 1, WALK_PITCH, WALK_LD, 1, &tmP, &tmJ);
            k_flux_walk<FLAT, RC, 1><<<dim3((n0 + 31) / 32, (n1 + FB - 1) / FB, n2), TPB, 0,
                                       h->st>>>(h->K, P, J, b.met, b.sig, Fd[1], tmP, tmJ, tma,
                                                b.stats);
        }
        if (G.g[2]) {
            const int tma = flux_maps(h, P, J, 2, WALK_PITCH, 1, WALK_LD, &tmP, &tmJ);
            k_flux_walk<FLAT, RC, 2><<<dim3((n0 + 31) / 32, n1, (n2 + FB - 1) / FB), TPB, 0,
                                       h->st>>>(h->K, P, J, b.met, b.sig, Fd[2], tmP, tmJ, tma,
                                                b.stats);
        }
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
    constexpr bool run = sizeof(T) == sizeof(double);
    auto nthreads = [&](int d) {
        long long n = 1;
        for (int a = 0; a < 3; a++) n *= a == d ? (run ? (G.n[a] + 1 + M - 1) / M : G.n[a] + 1) : G.n[a];
        return n;
    };
    if constexpr (run) {
        if (G.g[0]) k_flux_run<T, FLAT, RC, 0, M><<<nblk(nthreads(0)), TPB, 0, h->st>>>(h->K, P, J, b.met, b.sig, Fd[0]);
        if (G.g[1]) k_flux_run<T, FLAT, RC, 1, M><<<nblk(nthreads(1)), TPB, 0, h->st>>>(h->K, P, J, b.met, b.sig, Fd[1]);
        if (G.g[2]) k_flux_run<T, FLAT, RC, 2, M><<<nblk(nthreads(2)), TPB, 0, h->st>>>(h->K, P, J, b.met, b.sig, Fd[2]);
    } else {
        if (G.n[1] <= 65535 && G.n[2] <= 65535) {   // grid-dimension limits of the tiles
            launch_flux_tile<FLAT, RC>(h, P, J, Fd);
            return;
        }
        if (G.g[0]) k_flux<T, FLAT, RC, 0><<<nblk(nthreads(0)), TPB, 0, h->st>>>(h->K, P, J, b.met, b.sig, Fd[0]);
        if (G.g[1]) k_flux<T, FLAT, RC, 1><<<nblk(nthreads(1)), TPB, 0, h->st>>>(h->K, P, J, b.met, b.sig, Fd[1]);
        if (G.g[2]) k_flux<T, FLAT, RC, 2><<<nblk(nthreads(2)), TPB, 0, h->st>>>(h->K, P, J, b.met, b.sig, Fd[2]);
    }
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
    d.hcount = h->b.dcount + NDEFER + which;
    d.hidx = h->b.hidx;
    return d;
}

// Deferred passes: 64-thread blocks, enough of them for every record of a
// list of up to 148 * 96 * 64 (909 K) records to get its own thread, so that
// no thread takes a second record after its first (a fallback record can
// run for thousands of FP64 instructions); blocks past the list's count
// return at once.  Small blocks free their slot as soon as their two warps
// are done, which evens out the tail of the few long records.
const int TPB_DEFER = 64;
// warp-per-record passes: four warps per block, four blocks per SM; blocks
// past the list's count return at once
const unsigned HARD_BLOCKS = 148 * 4;
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
void enqueue_stages12_t(rmhd_t h, cudaEvent_t *ev, double *Us)
{
    Buffers &b = h->b;
    const StepConst &K = h->K;
    const unsigned nb = nblk(make_bricks(K.G.n).threads);   // stage kernels: bricks
    auto mark = [&](int i) { if (ev) cudaEventRecord(ev[i], h->st); };
    const bool dfr = b.dcap > 0;
    const unsigned nbd = deferred_blocks(h);
    T *PA = (T *)b.PA, *PB = (T *)b.PB, *J1 = (T *)b.J1, *J2 = (T *)b.J2;
    T *F0 = (T *)b.F[0], *F1 = (T *)b.F[1], *F2 = (T *)b.F[2];
    if (dfr) cudaMemsetAsync(b.dcount, 0, 2 * NDEFER * sizeof(int), h->st);
    mark(0);
    k_stage1<FLAT, T><<<nb, TPB, 0, h->st>>>(K, b.U, PA, b.GA, b.GA, b.dR1, J1, b.met, b.sig,
                                             defer_of(h, 0), b.stats);
    if (dfr) {
        k_deferred<FLAT, 1, T><<<nbd, TPB_DEFER, 0, h->st>>>(K, defer_of(h, 0), b.met, b.sig, nullptr,
                                                       PA, b.GA, b.dR1, J1, nullptr, nullptr,
                                                       b.stats);
        k_deferred_hard<FLAT, 1, T><<<HARD_BLOCKS, 128, 0, h->st>>>(K, defer_of(h, 0), b.met, b.sig, nullptr,
                                                       PA, b.GA, b.dR1, J1, nullptr, nullptr,
                                                       b.stats);
    }
    mark(1);
    launch_ghosts(h, PA, NPR);
    if (K.qflux == RMHD_QFLUX_GAUSS) gauss_charge<FLAT, T>(h, PA, nullptr);
    if (K.qflux != 1) launch_ghosts(h, J1, 3);
    mark(2);
    launch_flux<T, FLAT>(h, PA, J1);
    mark(3);
    k_stage2<FLAT, T><<<nb, TPB, 0, h->st>>>(K, b.U, PA, b.GA, F0, F1, F2, b.dR1, b.met, b.sig,
                                             PB, b.GB, b.V, J2, defer_of(h, 1), b.stats, Us);
    if (dfr) {
        k_deferred<FLAT, 2, T><<<nbd, TPB_DEFER, 0, h->st>>>(K, defer_of(h, 1), b.met, b.sig, b.dR1,
                                                       PB, b.GB, nullptr, J2, b.V, nullptr,
                                                       b.stats);
        k_deferred_hard<FLAT, 2, T><<<HARD_BLOCKS, 128, 0, h->st>>>(K, defer_of(h, 1), b.met, b.sig, b.dR1,
                                                       PB, b.GB, nullptr, J2, b.V, nullptr,
                                                       b.stats);
    }
    mark(4);
    launch_ghosts(h, PB, NPR);
    if (K.qflux == RMHD_QFLUX_GAUSS) gauss_charge<FLAT, T>(h, PB, nullptr);
    if (K.qflux != 1) launch_ghosts(h, J2, 3);
    mark(5);
}

template <bool FLAT, class T> void enqueue_final_t(rmhd_t h, cudaEvent_t *ev)
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
    if (dfr) {
        k_deferred<FLAT, 3, T><<<nbd, TPB_DEFER, 0, h->st>>>(K, defer_of(h, 2), b.met, b.sig, nullptr,
                                                       PA, b.GA, nullptr, nullptr, nullptr, b.U,
                                                       b.stats);
        k_deferred_hard<FLAT, 3, T><<<HARD_BLOCKS, 128, 0, h->st>>>(K, defer_of(h, 2), b.met, b.sig, nullptr,
                                                       PA, b.GA, nullptr, nullptr, nullptr, b.U,
                                                       b.stats);
    }
    mark(7);
    launch_ghosts(h, PA, NPR);
    if (K.qflux == RMHD_QFLUX_GAUSS) gauss_charge<FLAT, T>(h, PA, b.U);
    mark(8);
}

template <bool FLAT, class T> void enqueue_step_t(rmhd_t h, cudaEvent_t *ev)
{
    enqueue_stages12_t<FLAT, T>(h, ev, nullptr);
    enqueue_final_t<FLAT, T>(h, ev);
}

// One step of the general IMEX form (schemes other than Table imex).  Stage
// 1: k_stage1 with gimex = A_11 on U^n.  Stage i >= 2: k_stage_row forms
// the row's explicit part (F of stage i-1 from the face fluxes of its
// primitives) and solves the implicit part with the recovery (gimex = A_ii),
// writing the stage's primitives, Dt R_i and current.  The stages alternate
// between the two primitive buffers so that the last one lands in PB;
// k_final_row forms U^{n+1} from the weights in place and recovers it into
// PA.  The face fluxes of a stage are computed only when a later row or the
// weights use its F.
template <bool FLAT, class T> void enqueue_general_t(rmhd_t h, ProfMarks *pm)
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
    if (dfr) cudaMemsetAsync(b.dcount, 0, 2 * NDEFER * sizeof(int), h->st);
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
        if (dfr) {
            k_deferred<FLAT, 1, T><<<nbd, TPB_DEFER, 0, h->st>>>(Ki, defer_of(h, i), b.met, b.sig,
                                                           nullptr, Pb[cur], Gb[cur], dRi, J,
                                                           nullptr, nullptr, b.stats);
            k_deferred_hard<FLAT, 1, T><<<HARD_BLOCKS, 128, 0, h->st>>>(Ki, defer_of(h, i), b.met, b.sig,
                                                           nullptr, Pb[cur], Gb[cur], dRi, J,
                                                           nullptr, nullptr, b.stats);
        }
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
    if (dfr) {
        k_deferred<FLAT, 3, T><<<nbd, TPB_DEFER, 0, h->st>>>(K, defer_of(h, s), b.met, b.sig, nullptr,
                                                       Pb[0], Gb[0], nullptr, nullptr, nullptr,
                                                       b.U, b.stats);
        k_deferred_hard<FLAT, 3, T><<<HARD_BLOCKS, 128, 0, h->st>>>(K, defer_of(h, s), b.met, b.sig, nullptr,
                                                       Pb[0], Gb[0], nullptr, nullptr, nullptr,
                                                       b.U, b.stats);
    }
    mark(5);
    launch_ghosts(h, Pb[0], NPR);
    if (K.qflux == RMHD_QFLUX_GAUSS) gauss_charge<FLAT, T>(h, Pb[0], b.U);
    mark(1);
}


template <bool FLAT, class T> void launch_recover_cons(rmhd_t h, bool guess)
{
    k_recover_cons<FLAT, T><<<nblk(h->K.G.N), TPB, 0, h->st>>>(
        h->K, h->b.U, h->b.met, guess ? h->b.GA : nullptr, (T *)h->b.PA, h->b.GA, h->b.stats);
    launch_ghosts(h, (T *)h->b.PA, NPR);
}

// face fluxes of the stage whose primitives (with ghosts) are P and whose
// charge-flux current is J, then F(U) at every interior cell into the
// staging buffer
template <bool FLAT, class T> void launch_rhs(rmhd_t h, const T *P, const T *J)
{
    T *F0 = (T *)h->b.F[0], *F1 = (T *)h->b.F[1], *F2 = (T *)h->b.F[2];
    launch_flux<T, FLAT>(h, P, J);
    k_rhs<FLAT, T><<<nblk(h->K.G.N), TPB, 0, h->st>>>(h->K, P, F0, F1, F2, h->b.met, h->b.stage);
}

#define RMHD_INSTANTIATE_STEP(FLAT, T)                                                  \
    template void enqueue_stages12_t<FLAT, T>(rmhd_t, cudaEvent_t *, double *);           \
    template void enqueue_final_t<FLAT, T>(rmhd_t, cudaEvent_t *);                        \
    template void enqueue_step_t<FLAT, T>(rmhd_t, cudaEvent_t *);                         \
    template void enqueue_general_t<FLAT, T>(rmhd_t, ProfMarks *);                        \
    template void launch_recover_cons<FLAT, T>(rmhd_t, bool);                             \
    template void launch_rhs<FLAT, T>(rmhd_t, const T *, const T *);
