// noalloc.cu -- pointwise implicit-E + recovery that allocates no memory.
//
// Some callers cannot allocate device memory at the time they need a
// recovery: simulation drivers that size one memory pool at start-up and
// treat any later device allocation as an error, time-critical loops that
// cannot afford the device-wide synchronisation and unpredictable latency of
// cudaMalloc / cudaFree, and host programs that embed this library and own
// all device memory themselves.  For them rmhd_con2prim_points_noalloc runs
// the same two-pass recovery as the stepping kernels (paper iteration first;
// points it does not converge are listed and finished by a second pass with
// the fallbacks), but its work list lives in a fixed array compiled into this
// library instead of memory obtained from cudaMalloc.
//
// The array is a file-scope __device__ object of RMHD_NOALLOC_MAX_POINTS
// entries plus a counter (about 256 KB); every GPU that loads the library
// holds one copy until the process exits.  Host code cannot use the array's
// name as a device address (in host code it names a host-side stand-in), so
// the address is obtained once per device with cudaGetSymbolAddress, with
// that device current, on the first call made on that device; make that
// first call before any stream capture.  All calls share the one list:
// calls that overlap on the GPU (other streams, other host threads) race
// and must be serialised by the caller.  A device reset (cudaDeviceReset)
// destroys the context that held the array; the next call notices that the
// address it kept no longer belongs to a live allocation and looks it up
// again in the new context.
#include <cuda_runtime.h>
#include <mutex>
#include <stdio.h>

#include "../../include/rmhd.h"
#include "physics.cuh"
#include "recovery.cuh"

using namespace rmhd;

namespace {

// counter in the first 256 bytes, then the point indices
struct NoAllocScratch {
    int count;
    int pad[63];
    int idx[RMHD_NOALLOC_MAX_POINTS];
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

const int MAX_DEVICES = 64;
std::mutex g_mutex;
NoAllocScratch *g_addr[MAX_DEVICES] = {nullptr};
// error text of the calling thread's last failed call
thread_local char g_err[256] = "";

} // namespace

// error text reported by rmhd_last_error(NULL) and the parameter check
// shared with rmhd_con2prim_points (both defined with the C ABI)
void rmhd_internal_set_error(const char *msg);
bool rmhd_internal_recovery_params_ok(const rmhd_params *p);

namespace {

int fail(int code)
{
    rmhd_internal_set_error(g_err);
    return code;
}

__device__ __forceinline__ void load_point(int npts, int t, const double *__restrict__ cons,
                                           const double *__restrict__ alpha,
                                           const double *__restrict__ gam, Met<double> &m,
                                           RecIn &in)
{
    m.alpha = alpha[t];
    m.beta[0] = m.beta[1] = m.beta[2] = 0.0;
    for (int a = 0; a < 6; a++) m.g[a] = gam[a * npts + t];
    met_complete(m);
    in.D = cons[CO_D * npts + t];
    in.tau = cons[CO_TAU * npts + t];
    for (int a = 0; a < 3; a++) {
        in.S[a] = cons[(CO_SX + a) * npts + t];
        in.cB[a] = cons[(CO_BX + a) * npts + t];
        in.cE0[a] = cons[(CO_EX + a) * npts + t];
    }
}

__device__ __forceinline__ void store_point(int npts, int t, int st, int it, const double pr[NPR],
                                            const double E[3], const Met<double> &m, double gfac,
                                            const double *__restrict__ cons, double *prim,
                                            double *cons_out, int *iters, int *status)
{
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

// pass 1: the paper iteration; a point it does not converge is listed
__global__ void __launch_bounds__(128)
k_points_first_pass(const RecOpts ro, int npts, const double *__restrict__ cons,
                    const double *__restrict__ guess, const double *__restrict__ alpha,
                    const double *__restrict__ gam, const double *__restrict__ sigma,
                    int implicit, double c, double gfac, NoAllocScratch *scr, double *prim,
                    double *cons_out, int *iters, int *status)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npts) return;
    Met<double> m;
    RecIn in;
    load_point(npts, t, cons, alpha, gam, m, in);
    const double gv[3] = {guess[PR_VX * npts + t], guess[PR_VY * npts + t],
                          guess[PR_VZ * npts + t]};
    const double cc = implicit ? c * m.alpha * sigma[t] : 0.0;
    double pr[NPR], E[3];
    int it = 0;
    const int st = recover<false>(in, m, ro, implicit != 0, cc, guess[PR_P * npts + t], gv,
                                  cons[CO_PHI * npts + t], cons[CO_PSI * npts + t],
                                  cons[CO_Q * npts + t], pr, E, it, REC_PRIMARY);
    if (st == REC_DEFER) {
        // npts <= capacity, so every listed point has a slot
        const int slot = atomicAdd(&scr->count, 1);
        scr->idx[slot] = t;
        iters[t] = it;
        return;
    }
    store_point(npts, t, st, it, pr, E, m, gfac, cons, prim, cons_out, iters, status);
}

// pass 2: fallbacks for the listed points, one thread each
__global__ void __launch_bounds__(128)
k_points_second_pass(const RecOpts ro, int npts, const double *__restrict__ cons,
                     const double *__restrict__ guess, const double *__restrict__ alpha,
                     const double *__restrict__ gam, const double *__restrict__ sigma,
                     int implicit, double c, double gfac, const NoAllocScratch *scr,
                     double *prim, double *cons_out, int *iters, int *status)
{
    const int n = scr->count;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const int t = scr->idx[s];
        Met<double> m;
        RecIn in;
        load_point(npts, t, cons, alpha, gam, m, in);
        const double gv[3] = {guess[PR_VX * npts + t], guess[PR_VY * npts + t],
                              guess[PR_VZ * npts + t]};
        const double cc = implicit ? c * m.alpha * sigma[t] : 0.0;
        double pr[NPR], E[3];
        int it = 0;
        const int st = recover<false>(in, m, ro, implicit != 0, cc, guess[PR_P * npts + t], gv,
                                      cons[CO_PHI * npts + t], cons[CO_PSI * npts + t],
                                      cons[CO_Q * npts + t], pr, E, it, REC_FALLBACK);
        store_point(npts, t, st, iters[t] + it, pr, E, m, gfac, cons, prim, cons_out, iters,
                    status);
    }
}

// device address of this device's copy of the array (set-up on first use)
int scratch_address(NoAllocScratch **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        snprintf(g_err, sizeof g_err, "cudaGetDevice failed: %s", cudaGetErrorString(e));
        return fail(RMHD_ECUDA);
    }
    if (dev < 0 || dev >= MAX_DEVICES) {
        snprintf(g_err, sizeof g_err, "device %d beyond the %d supported", dev, MAX_DEVICES);
        return fail(RMHD_EINVAL);
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (g_addr[dev]) {
        // still an address of device memory in the current context?  (not
        // after a device reset; the lookup below then runs again)
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, g_addr[dev]) != cudaSuccess ||
            at.type != cudaMemoryTypeDevice || at.device != dev) {
            cudaGetLastError();   // clear the error of the stale query
            g_addr[dev] = nullptr;
        }
    }
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            snprintf(g_err, sizeof g_err, "cudaGetSymbolAddress failed: %s",
                     cudaGetErrorString(e));
            return fail(RMHD_ECUDA);
        }
        g_addr[dev] = (NoAllocScratch *)p;
    }
    *out = g_addr[dev];
    return RMHD_OK;
}

} // namespace

extern "C" int rmhd_con2prim_points_noalloc(const rmhd_params *p, int npts, const double *cons,
                                            const double *guess, const double *alpha,
                                            const double *gamma, const double *sigma,
                                            int implicit, double c, double *prim,
                                            double *cons_out, int *iters, int *status,
                                            void *cuda_stream)
{
    if (!p) {
        snprintf(g_err, sizeof g_err, "params is NULL");
        return fail(RMHD_EINVAL);
    }
    if (npts < 0 || npts > RMHD_NOALLOC_MAX_POINTS) {
        snprintf(g_err, sizeof g_err,
                 "npts = %d outside [0, %d], the capacity of the built-in work list", npts,
                 RMHD_NOALLOC_MAX_POINTS);
        return fail(RMHD_EINVAL);
    }
    if (npts == 0) return RMHD_OK;
    if (!cons || !guess || !alpha || !gamma || !prim || !cons_out || !iters || !status ||
        (implicit && !sigma)) {
        snprintf(g_err, sizeof g_err, "NULL array");
        return fail(RMHD_EINVAL);
    }
    if (!rmhd_internal_recovery_params_ok(p)) {
        snprintf(g_err, sizeof g_err, "recovery parameters out of range");
        return fail(RMHD_EINVAL);
    }
    NoAllocScratch *scr = nullptr;
    int rc = scratch_address(&scr);
    if (rc) return rc;
    RecOpts ro;
    ro.Gam = p->gamma_eos;
    ro.tol = p->c2p_tol;
    ro.v2max = 1.0 - 1.0 / (p->c2p_wmax * p->c2p_wmax);
    ro.rho_atmo = p->rho_atmo;
    ro.p_atmo = p->K_atmo * pow(p->rho_atmo, p->gamma_eos);
    ro.atmo_floor = p->rho_atmo * (1.0 + p->atmo_tol);
    ro.maxit = p->c2p_maxit;
    ro.first_cap = p->c2p_maxit;
    ro.kappa0 = 0.3;   // as rmhd_con2prim_points
    const double gfac = p->gamma_eos / (p->gamma_eos - 1.0);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the list keeps the previous call's contents: clear the counter
    cudaError_t e = cudaMemsetAsync(&scr->count, 0, sizeof(int), st);
    if (e != cudaSuccess) {
        snprintf(g_err, sizeof g_err, "cudaMemsetAsync failed: %s", cudaGetErrorString(e));
        return fail(RMHD_ECUDA);
    }
    const int tpb = 128, nb = (npts + tpb - 1) / tpb;
    k_points_first_pass<<<nb, tpb, 0, st>>>(ro, npts, cons, guess, alpha, gamma, sigma, implicit,
                                            c, gfac, scr, prim, cons_out, iters, status);
    k_points_second_pass<<<nb < 148 * 8 ? nb : 148 * 8, tpb, 0, st>>>(
        ro, npts, cons, guess, alpha, gamma, sigma, implicit, c, gfac, scr, prim, cons_out, iters,
        status);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(g_err, sizeof g_err, "launch failed: %s", cudaGetErrorString(e));
        return fail(RMHD_ECUDA);
    }
    return RMHD_OK;
}
