// adjoint_host.cu -- host side of the discrete adjoint of the FP64 step
// (rmhd_set_sigma0, rmhd_adjoint_forward, rmhd_adjoint_backward): recording
// with checkpoints, segment re-runs and the reverse sweep of the kernels in
// adjoint.cuh.
#include "host.cuh"
#include "adjoint.cuh"

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

