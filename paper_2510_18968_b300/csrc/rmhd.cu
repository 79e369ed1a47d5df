// rmhd.cu -- host side of the C ABI declared in include/rmhd.h: parameter
// checks, device memory, the set-up and read-out entry points, the step
// entry points (launches or a captured graph of the stage sequencing in
// step_impl.cuh), and the testing entry points.  The adjoint entry points
// are in adjoint_host.cu.
#include <atomic>

#include "host.cuh"

namespace rmhd_host {
// text of the calling thread's last error of a call without a handle
thread_local char g_noh_err[512] = "";
} // namespace rmhd_host

namespace rmhd {
// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library), looked up once per process
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return (EncodeTiledFn)p;
    }();
    return fn;
}

// tile copies enabled (rmhd_test_tile_copies), launches that used them
static std::atomic<int> g_tile_copies{1};
std::atomic<long long> g_tile_copy_launches{0};

bool make_tile_map(CUtensorMap *map, const float *base, int px, int py, int pz,
                   long long field_stride, int nf, int bx, int by, int bz)
{
    const EncodeTiledFn fn = encode_tiled();
    if (!fn || !g_tile_copies.load()) return false;
    // every stride a multiple of 16 bytes, the box's x extent too, the base
    // 16-byte aligned: the conditions of a tile copy (the driver checks
    // them again)
    if ((px * 4) % 16 || (field_stride * 4) % 16 || (bx * 4) % 16 ||
        ((uintptr_t)base) % 16)
        return false;
    const cuuint32_t rank = nf > 0 ? 4 : 3;
    const cuuint64_t dims[4] = {(cuuint64_t)px, (cuuint64_t)py, (cuuint64_t)pz,
                                (cuuint64_t)(nf > 0 ? nf : 1)};
    const cuuint64_t strides[3] = {(cuuint64_t)px * 4, (cuuint64_t)px * py * 4,
                                   (cuuint64_t)field_stride * 4};
    const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz,
                               (cuuint32_t)(nf > 0 ? nf : 1)};
    const cuuint32_t elem[4] = {1, 1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, (void *)base, dims, strides, box, elem,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}
} // namespace rmhd

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
    // a cell whose first paper iteration did not converge goes to Newton at
    // once when the iteration would contract by less than 0.3 per step
    // (measured on the magnetised blast exterior: about 20 or more further
    // paper iterations, more than a Newton solve costs)
    o.kappa0 = 0.3;
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
    if (b.hidx) cudaFree(b.hidx);
    if (b.drec) cudaFree(b.drec);
    b.stats = nullptr;
    b.flag = nullptr;
    b.dcount = b.didx = b.hidx = nullptr;
    b.drec = nullptr;
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
    // x pitch rounded up to 4 cells when x is active: every row and every
    // field then starts on a 16-byte boundary in both precisions, which the
    // tensor-map (TMA) tile loads require; the pad cells are never read
    G.px = G.g[0] ? (G.n[0] + 2 * G.g[0] + 3) / 4 * 4 : G.n[0];
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
        if (cudaMalloc((void **)&b.dcount, 2 * NDEFER * sizeof(int)) != cudaSuccess ||
            cudaMalloc((void **)&b.didx, sizeof(int) * (size_t)cap) != cudaSuccess ||
            cudaMalloc((void **)&b.hidx, sizeof(int) * (size_t)cap) != cudaSuccess ||
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

// flags a conserved state that is not finite or has D <= 0
__global__ void k_check_cons(long long N, const double *__restrict__ a, int *bad)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= N) return;
    bool ok = a[t] > 0.0;   // D
    for (int f = 0; f < NCO; f++) ok = ok && isfinite(a[f * N + t]);
    if (!ok) atomicOr(bad, 1);
}

extern "C" int rmhd_set_cons(rmhd_t h, const double *cons, int on_device)
{
    if (!h) return set_err(nullptr, RMHD_EINVAL, "handle is NULL");
    if (!cons) return set_err(h, RMHD_EINVAL, "cons is NULL");
    const Grid &G = h->K.G;
    int bad = 0;
    int rc = stage_in(h, cons, NCO, on_device);
    if (rc) return rc;
    cudaMemsetAsync(h->b.flag, 0, sizeof(int), h->st);
    k_check_cons<<<nblk(G.N), TPB, 0, h->st>>>(G.N, h->b.stage, h->b.flag);
    rc = read_flag(h, &bad);
    if (rc) return rc;
    if (bad) return set_err(h, RMHD_EINVAL, "cons rejected: D <= 0 or non-finite values");
    unsigned long long before[NSTAT], after[NSTAT];
    CK(cudaMemcpyAsync(before, h->b.stats, sizeof(before), cudaMemcpyDeviceToHost, h->st));
    k_scatter<double><<<nblk(G.N), TPB, 0, h->st>>>(h->K, h->b.stage, h->b.U, NCO);
    const bool guess = h->have_state;
    const bool mixed = h->p.precision == RMHD_PREC_MIXED;
    if (h->flat) {
        if (mixed) launch_recover_cons<true, float>(h, guess);
        else launch_recover_cons<true, double>(h, guess);
    } else {
        if (mixed) launch_recover_cons<false, float>(h, guess);
        else launch_recover_cons<false, double>(h, guess);
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(after, h->b.stats, sizeof(after), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    h->have_state = true;
    const long long fails = (long long)(after[ST_FAIL] - before[ST_FAIL]);
    if (fails > 0)
        return set_err(h, RMHD_EC2P, "%lld recoveries reset to the atmosphere", fails);
    return RMHD_OK;
}

// ---------------------------------------------------- z-layers of the state
// The state a step starts from is U (FP64), the primitives P (the path's
// storage type) and, on the mixed path, the FP64 recovery guess G (p, v^i).
// A packed z-range holds, for its nk interior layers (nx*ny cells each), the
// 14 fields of U, then the 14 of P, then the 4 of G (mixed only), each field
// x fastest, copied bit for bit.

template <class T>
__global__ void k_zlayers(const StepConst K, int k0, int nk, T *padded, T *packed, int nf,
                          int unpack)
{
    const Grid &G = K.G;
    const long long plane = (long long)G.n[0] * G.n[1];
    const long long cells = plane * nk;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= cells) return;
    const int i = (int)(t % G.n[0]);
    const int j = (int)((t / G.n[0]) % G.n[1]);
    const int k = k0 + (int)(t / plane);
    const long long c = cell_at(G, i, j, k);
    for (int f = 0; f < nf; f++) {
        if (unpack) padded[f * G.S + c] = packed[f * cells + t];
        else packed[f * cells + t] = padded[f * G.S + c];
    }
}

static long long layer_bytes(rmhd_t h)
{
    const bool mixed = h->p.precision == RMHD_PREC_MIXED;
    const long long plane = (long long)h->K.G.n[0] * h->K.G.n[1];
    return plane * (long long)(NCO * 8 + NPR * (mixed ? 4 : 8) + (mixed ? 4 * 8 : 0));
}

extern "C" long long rmhd_state_layer_bytes(rmhd_t h) { return h ? layer_bytes(h) : -1; }

static int zlayers(rmhd_t h, int k0, int nk, void *buf, int on_device, int unpack)
{
    if (!h || !buf) return set_err(h, RMHD_EINVAL, "NULL argument");
    const Grid &G = h->K.G;
    if (k0 < 0 || nk < 1 || k0 + nk > G.n[2])
        return set_err(h, RMHD_EINVAL, "z-layers [%d, %d) outside [0, %d)", k0, k0 + nk, G.n[2]);
    if (!h->have_state) return set_err(h, RMHD_EINVAL, "no state: call rmhd_set_prims first");
    const size_t bytes = (size_t)layer_bytes(h) * nk;
    char *dev = (char *)buf;
    if (!on_device) {
        // through the staging buffer (14 N doubles)
        if (bytes > sizeof(double) * NCO * (size_t)G.N)
            return set_err(h, RMHD_EINVAL, "%d layers exceed the staging buffer; pass device "
                                           "memory", nk);
        dev = (char *)h->b.stage;
        if (unpack) CK(cudaMemcpyAsync(dev, buf, bytes, cudaMemcpyHostToDevice, h->st));
    }
    const long long cells = (long long)G.n[0] * G.n[1] * nk;
    const bool mixed = h->p.precision == RMHD_PREC_MIXED;
    k_zlayers<double><<<nblk(cells), TPB, 0, h->st>>>(h->K, k0, nk, h->b.U, (double *)dev, NCO,
                                                      unpack);
    dev += sizeof(double) * NCO * cells;
    if (mixed) {
        k_zlayers<float><<<nblk(cells), TPB, 0, h->st>>>(h->K, k0, nk, (float *)h->b.PA,
                                                         (float *)dev, NPR, unpack);
        dev += sizeof(float) * NPR * cells;
        k_zlayers<double><<<nblk(cells), TPB, 0, h->st>>>(h->K, k0, nk, h->b.GA, (double *)dev, 4,
                                                          unpack);
    } else {
        k_zlayers<double><<<nblk(cells), TPB, 0, h->st>>>(h->K, k0, nk, (double *)h->b.PA,
                                                          (double *)dev, NPR, unpack);
    }
    CK(cudaGetLastError());
    if (!on_device) {
        if (!unpack) CK(cudaMemcpyAsync(buf, h->b.stage, bytes, cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
    }
    return RMHD_OK;
}

extern "C" int rmhd_get_state_layers(rmhd_t h, int k0, int nk, void *buf, int on_device)
{
    return zlayers(h, k0, nk, buf, on_device, 0);
}

extern "C" int rmhd_set_state_layers(rmhd_t h, int k0, int nk, const void *buf, int on_device)
{
    return zlayers(h, k0, nk, (void *)buf, on_device, 1);
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
    if (after[ST_TILE]) return set_err(h, RMHD_ECUDA, "a stencil tile load did not complete");
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
    if (J) {
        int rc = stage_in(h, J, 3, on_device);
        if (rc) return rc;
        k_scatter<T><<<nblk(G.N), TPB, 0, h->st>>>(h->K, h->b.stage, J2, 3);
    } else {
        CK(cudaMemsetAsync(J2, 0, sizeof(T) * 3 * (size_t)G.S, h->st));
    }
    launch_ghosts(h, J2, 3);
    if (h->flat) launch_rhs<true, T>(h, PB, J2);
    else launch_rhs<false, T>(h, PB, J2);
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

// the pressure bracket and atmosphere of the fallback chain on independent
// flat points (testing entry point): one thread per point, or (WARP) one
// warp per point with lane 0 writing
template <bool WARP>
__global__ void __launch_bounds__(128)
k_test_bracket_points(const RecOpts ro, int npts, const double *__restrict__ cons,
                      const double *__restrict__ guess, const double *__restrict__ sigma,
                      int implicit, double c, double *prim, int *status)
{
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = WARP ? gt >> 5 : gt;
    if (t >= npts) return;   // the whole warp when WARP
    Met<double> m;
    m.alpha = 1.0;
    m.beta[0] = m.beta[1] = m.beta[2] = 0.0;
    m.g[0] = m.g[3] = m.g[5] = 1.0;
    m.g[1] = m.g[2] = m.g[4] = 0.0;
    met_complete(m);
    RecIn in;
    in.D = cons[CO_D * npts + t];
    in.tau = cons[CO_TAU * npts + t];
    for (int a = 0; a < 3; a++) {
        in.S[a] = cons[(CO_SX + a) * npts + t];
        in.cB[a] = cons[(CO_BX + a) * npts + t];
        in.cE0[a] = cons[(CO_EX + a) * npts + t];
    }
    const double gp = guess[PR_P * npts + t];
    const double gv[3] = {guess[PR_VX * npts + t], guess[PR_VY * npts + t],
                          guess[PR_VZ * npts + t]};
    // a record whose paper iteration and both Newton methods gave up
    PaperState ps = {};
    ps.p = gp;
    for (int a = 0; a < 3; a++) ps.v[a] = gv[a];
    ps.outcome = 0;
    double pr[NPR], E[3];
    int it = 0;
    const double cc = implicit ? c * sigma[t] : 0.0;
    const int st = recover<true, WARP>(in, m, ro, implicit != 0, cc, gp, gv,
                                       cons[CO_PHI * npts + t], cons[CO_PSI * npts + t],
                                       cons[CO_Q * npts + t], pr, E, it, REC_CHAIN_REST, &ps);
    if (WARP && (threadIdx.x & 31) != 0) return;
    for (int f = 0; f < NPR; f++) prim[f * npts + t] = pr[f];
    status[t] = st;
}

// parameters the pointwise recovery entry points use (rmhd_con2prim_points
// and rmhd_con2prim_points_noalloc check the same set)
__attribute__((visibility("hidden"))) bool rmhd_internal_recovery_params_ok(const rmhd_params *p)
{
    return p->gamma_eos > 1.0 && p->c2p_tol > 0.0 && p->c2p_maxit >= 1 && p->c2p_wmax > 1.0 &&
           p->rho_atmo > 0.0 && p->K_atmo >= 0.0 && p->atmo_tol >= 0.0;
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
    if (!rmhd_internal_recovery_params_ok(p))
        return set_err(h, RMHD_EINVAL, "recovery parameters out of range");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    k_recover_points<<<nblk(npts), TPB, 0, st>>>(rec_opts(p), npts, cons, guess, alpha, gamma,
                                                 sigma, implicit, c,
                                                 p->gamma_eos / (p->gamma_eos - 1.0), prim,
                                                 cons_out, iters, status);
    CK(cudaGetLastError());
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

extern "C" int rmhd_test_bracket_points(const rmhd_params *p, int npts, const double *cons,
                                        const double *guess, const double *sigma, int implicit,
                                        double c, int one_warp, double *prim, int *status,
                                        void *cuda_stream)
{
    rmhd_t h = nullptr;
    if (!p) return set_err(h, RMHD_EINVAL, "params is NULL");
    if (npts < 0) return set_err(h, RMHD_EINVAL, "npts < 0");
    if (npts == 0) return RMHD_OK;
    if (!cons || !guess || !prim || !status || (implicit && !sigma))
        return set_err(h, RMHD_EINVAL, "NULL array");
    if (!rmhd_internal_recovery_params_ok(p))
        return set_err(h, RMHD_EINVAL, "recovery parameters out of range");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (one_warp)
        k_test_bracket_points<true><<<nblk(32LL * npts), TPB, 0, st>>>(
            rec_opts(p), npts, cons, guess, sigma, implicit, c, prim, status);
    else
        k_test_bracket_points<false><<<nblk(npts), TPB, 0, st>>>(
            rec_opts(p), npts, cons, guess, sigma, implicit, c, prim, status);
    CK(cudaGetLastError());
    return RMHD_OK;
}

extern "C" int rmhd_test_tile_copies(int enable)
{
    return rmhd::g_tile_copies.exchange(enable != 0 ? 1 : 0);
}

extern "C" long long rmhd_test_tile_copy_launches(void)
{
    return rmhd::g_tile_copy_launches.load();
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
