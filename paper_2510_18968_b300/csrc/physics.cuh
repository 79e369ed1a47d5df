// physics.cuh -- pointwise device physics of the resistive GRMHD step
// (arXiv:2510.18968, Sec. II-III), templated on the floating type T and on a
// flat-metric switch.  With FLAT the lapse is 1, the shift 0 and gamma_ij the
// identity, and every metric factor is dropped at compile time (multiplying
// by 1 and adding 0 are exact, so FLAT and the general path agree bit for bit
// up to the order of fused multiply-adds).
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

namespace rmhd {

// primitive and conserved slots (Sec. III.B order and Eq. GRRMHD_flux_form)
enum { PR_RHO = 0, PR_P, PR_VX, PR_VY, PR_VZ, PR_EX, PR_EY, PR_EZ, PR_BX, PR_BY,
       PR_BZ, PR_PSI, PR_PHI, PR_Q, NPR };
enum { CO_D = 0, CO_SX, CO_SY, CO_SZ, CO_TAU, CO_BX, CO_BY, CO_BZ, CO_EX, CO_EY,
       CO_EZ, CO_PHI, CO_PSI, CO_Q, NCO };

// symmetric 3x3 packed as xx, xy, xz, yy, yz, zz
__host__ __device__ constexpr int sym(int i, int j)
{
    return i == j ? (i == 0 ? 0 : (i == 1 ? 3 : 5))
                  : ((i + j) == 1 ? 1 : ((i + j) == 2 ? 2 : 4));
}

template <class T> struct Met {
    T alpha, beta[3];
    T g[6], gi[6];
    T sg, isg;  // sqrt(det gamma), 1/sqrt(det gamma)
};

// gamma^{ij} (adjugate / det) and sqrt(gamma) (Sec. II.A)
template <class T> __device__ __forceinline__ void met_complete(Met<T> &m)
{
    const T *g = m.g;
    T c00 = g[3] * g[5] - g[4] * g[4];
    T c01 = g[4] * g[2] - g[1] * g[5];
    T c02 = g[1] * g[4] - g[3] * g[2];
    T det = g[0] * c00 + g[1] * c01 + g[2] * c02;
    T id = T(1) / det;
    m.gi[0] = c00 * id;
    m.gi[1] = c01 * id;
    m.gi[2] = c02 * id;
    m.gi[3] = (g[0] * g[5] - g[2] * g[2]) * id;
    m.gi[4] = (g[2] * g[1] - g[0] * g[4]) * id;
    m.gi[5] = (g[0] * g[3] - g[1] * g[1]) * id;
    m.sg = sqrt(det);
    m.isg = T(1) / m.sg;
}

// 1/x in FP64 by Newton-Raphson refinement of a single-precision seed:
// r <- r + r (1 - x r) doubles the number of correct bits per step, from
// the ~22 bits of the FP32 hardware reciprocal to well past the 53 of a
// double in two steps (the result is within an ulp or two of 1/x).  About
// four FP64 FMAs instead of the FP64 division sequence, which on B300 costs
// ~11 FMAs of the FP64 pipe.  The seed's float <-> double conversions are
// done by moving the exponent and mantissa fields on the integer pipe (on
// B300 the FP64 pipe runs conversions at the rate of an FMA): x is
// truncated to 23 mantissa bits, which a seed tolerates, and the float
// reciprocal widens exactly.  Arguments with |x| outside [2^-120, 2^120)
// (and 0, inf, NaN) take the plain division.
__device__ __forceinline__ double rcp64(double x)
{
    const unsigned long long bx = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(bx >> 32), ex = (hi >> 20) & 0x7ffu;
    if (ex < 903u || ex >= 1143u) return 1.0 / x;
    const unsigned fx = (hi & 0x80000000u) | ((ex - 896u) << 23) | ((unsigned)(bx >> 29) & 0x7fffffu);
    const unsigned rb = __float_as_uint(__fdividef(1.0f, __uint_as_float(fx)));
    double r = __hiloint2double((int)((rb & 0x80000000u) | ((((rb >> 23) & 0xffu) + 896u) << 20) |
                                      ((rb & 0x7fffffu) >> 3)),
                                (int)(rb << 29));
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}

// float <-> double for the mixed path's stored FP32 stencil values, by
// moving the sign, exponent and mantissa fields on the integer pipe without
// branches (on B300 the FP64 pipe runs conversions at the rate of an FMA,
// and the recovery kernels that convert the FP32 right-hand side in and the
// primitives out are FP64-pipe-bound).  Exact, with round to nearest even
// for double -> float, for every value whose result is a normal number,
// zero, infinity or NaN; magnitudes below the smallest normal float
// (~1.2e-38) are flushed to a signed zero.
__device__ __forceinline__ double f2d_ftz(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned sign = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    unsigned hi = sign | ((e + 896u) << 20) | (m >> 3);
    hi = e == 0xffu ? (sign | 0x7ff00000u | (m >> 3)) : hi;
    hi = e == 0u ? sign : hi;
    const unsigned lo = e == 0u ? 0u : m << 29;
    return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ float d2f_ftz(double d)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    const unsigned hi = (unsigned)(u >> 32), sign = hi & 0x80000000u;
    const unsigned e = (hi >> 20) & 0x7ffu;
    const unsigned mf = (unsigned)(u >> 29) & 0x7fffffu, rest = (unsigned)u & 0x1fffffffu;
    unsigned bits = sign | ((e - 896u) << 23) | mf;
    // nearest, ties to even; a carry out of the mantissa raises the exponent
    bits += (rest > 0x10000000u) | ((rest == 0x10000000u) & mf);
    const bool nan = e == 0x7ffu && (u << 12) != 0ULL;
    bits = e > 1150u ? (sign | 0x7f800000u | (nan ? 0x400000u : 0u)) : bits;
    bits = e < 897u ? sign : bits;
    return __uint_as_float(bits);
}

// a double stored as T, and a T read as double
template <class T> __device__ __forceinline__ T from_double(double x)
{
    if constexpr (std::is_same<T, float>::value) return d2f_ftz(x);
    else return (T)x;
}
template <class T> __device__ __forceinline__ double to_double(T x)
{
    if constexpr (std::is_same<T, float>::value) return f2d_ftz(x);
    else return (double)x;
}

// the same metric in another arithmetic type (constants for a dual number)
template <class R> __device__ __forceinline__ Met<R> met_cast(const Met<double> &m)
{
    Met<R> r;
    r.alpha = R(m.alpha);
    for (int a = 0; a < 3; a++) r.beta[a] = R(m.beta[a]);
    for (int a = 0; a < 6; a++) {
        r.g[a] = R(m.g[a]);
        r.gi[a] = R(m.gi[a]);
    }
    r.sg = R(m.sg);
    r.isg = R(m.isg);
    return r;
}

template <class T, bool FLAT>
__device__ __forceinline__ void lower(const Met<T> &m, const T u[3], T ul[3])
{
    if (FLAT) {
        ul[0] = u[0]; ul[1] = u[1]; ul[2] = u[2];
    } else {
        ul[0] = m.g[0] * u[0] + m.g[1] * u[1] + m.g[2] * u[2];
        ul[1] = m.g[1] * u[0] + m.g[3] * u[1] + m.g[4] * u[2];
        ul[2] = m.g[2] * u[0] + m.g[4] * u[1] + m.g[5] * u[2];
    }
}

template <class T, bool FLAT>
__device__ __forceinline__ void raise(const Met<T> &m, const T ul[3], T u[3])
{
    if (FLAT) {
        u[0] = ul[0]; u[1] = ul[1]; u[2] = ul[2];
    } else {
        u[0] = m.gi[0] * ul[0] + m.gi[1] * ul[1] + m.gi[2] * ul[2];
        u[1] = m.gi[1] * ul[0] + m.gi[3] * ul[1] + m.gi[4] * ul[2];
        u[2] = m.gi[2] * ul[0] + m.gi[4] * ul[1] + m.gi[5] * ul[2];
    }
}

template <class T> __device__ __forceinline__ T dot3(const T a[3], const T b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// (a x b)_i = eta_ijk a_j b_k
template <class T>
__device__ __forceinline__ void cross3(const T a[3], const T b[3], T c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

template <class T> __device__ __forceinline__ T sg_of(const Met<T> &m, bool flat)
{
    return flat ? T(1) : m.sg;
}

// ---------------------------------------------------------------------------
// Conserved vector and flux in direction D at one state.
// U: Eqs. conserved_dens, conserved_tau, conserved_S, densitised EM fields.
// F: flux column of Eq. GRRMHD_flux_form, with the undensitised stress inside
//    the S_i flux; the charge-flux current is Jd when useJ, else Ohm's law
//    (Eq. Ohm_law) at this state.  gfac = Gamma/(Gamma-1): h = rho + gfac p.
// Accumulates cF*F + cU*U into acc (the HLLE combination), so that neither U
// nor F has to stay live as an array.  acc.add(f, x) receives the term of
// field f: an array (ArrAcc, the flux kernels) or a weighted sum of the
// fields (WeightedAcc, the adjoint's lambda . (cF F + cU U)).
// ---------------------------------------------------------------------------
template <class T> struct ArrAcc {
    T *a;
    __device__ __forceinline__ void add(int f, const T &x) { a[f] += x; }
};
template <class T> struct WeightedAcc {
    const double *w;
    T sum;
    __device__ __forceinline__ void add(int f, const T &x) { sum += w[f] * x; }
};

template <class T, bool FLAT, int D, class Acc>
__device__ __forceinline__ void flux_accumulate(const T pr[NPR], const Met<T> &m,
                                                T sigma, T gfac, bool useJ, T Jd,
                                                T cF, T cU, Acc &acc)
{
    const T sg = FLAT ? T(1) : m.sg;
    const T a = FLAT ? T(1) : m.alpha;
    const T bD = FLAT ? T(0) : m.beta[D];
    T v[3] = {pr[PR_VX], pr[PR_VY], pr[PR_VZ]};
    T E[3] = {pr[PR_EX], pr[PR_EY], pr[PR_EZ]};
    T B[3] = {pr[PR_BX], pr[PR_BY], pr[PR_BZ]};
    T vl[3], El[3], Bl[3];
    lower<T, FLAT>(m, v, vl);
    lower<T, FLAT>(m, E, El);
    lower<T, FLAT>(m, B, Bl);
    const T rho = pr[PR_RHO], p = pr[PR_P];
    const T v2 = dot3(v, vl);
    // Lorentz factor: in FP64 one reciprocal square root instead of a
    // square root and a division (both FP64-pipe sequences on B300); in
    // FP32 the hardware reciprocal square root (rsqrtf, within 2 ulp), one
    // instruction instead of the IEEE square root and division sequences
    T W;
    if constexpr (std::is_same<T, double>::value) W = rsqrt(1.0 - v2);
    else W = rsqrtf(T(1) - v2);
    const T h = rho + gfac * p;
    const T hW2 = h * W * W;
    const T em = T(0.5) * (dot3(E, El) + dot3(B, Bl));

    // conserved vector
    const T Dc = sg * rho * W;
    const T tau = sg * (hW2 - p + em) - Dc;
    T ExB[3];
    cross3(E, B, ExB);
    T S[3];
#pragma unroll
    for (int i = 0; i < 3; i++) S[i] = sg * (hW2 * vl[i] + sg * ExB[i]);

    // D, S_i, tau
    acc.add(CO_D, cF * ((a * v[D] - bD) * Dc) + cU * Dc);
#pragma unroll
    for (int i = 0; i < 3; i++) {
        T st = hW2 * v[D] * vl[i] - E[D] * El[i] - B[D] * Bl[i];
        if (i == D) st += p + em;
        T f = a * sg * st;
        if (!FLAT) f -= bD * S[i];
        acc.add(CO_SX + i, cF * f + cU * S[i]);
    }
    T SD = S[D];
    if (!FLAT) SD = m.gi[sym(D, 0)] * S[0] + m.gi[sym(D, 1)] * S[1] + m.gi[sym(D, 2)] * S[2];
    {
        T f = a * (SD - v[D] * Dc);
        if (!FLAT) f -= bD * tau;
        acc.add(CO_TAU, cF * f + cU * tau);
    }
    // B^i: alpha (eps^{iDj} calE_j + gamma^{iD} Phi) - beta^D calB^i, with
    // eps^{iDj} calE_j = (e_D x E_lower)_i; E^i: -[alpha(...B...) + beta^D calE^i]
    const T Phi = sg * pr[PR_PHI], Psi = sg * pr[PR_PSI], Qc = sg * pr[PR_Q];
    T eE[3] = {T(0), T(0), T(0)}, eB[3] = {T(0), T(0), T(0)};
    if (D == 0) { eE[1] = -El[2]; eE[2] = El[1]; eB[1] = -Bl[2]; eB[2] = Bl[1]; }
    if (D == 1) { eE[0] = El[2]; eE[2] = -El[0]; eB[0] = Bl[2]; eB[2] = -Bl[0]; }
    if (D == 2) { eE[0] = -El[1]; eE[1] = El[0]; eB[0] = -Bl[1]; eB[1] = Bl[0]; }
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const T gid = FLAT ? (i == D ? T(1) : T(0)) : m.gi[sym(i, D)];
        const T cB = sg * B[i], cE = sg * E[i];
        T fB = a * (eE[i] + gid * Phi);
        T fE = -(a * (eB[i] - gid * Psi));
        if (!FLAT) {
            fB -= bD * cB;
            fE -= bD * cE;
        }
        acc.add(CO_BX + i, cF * fB + cU * cB);
        acc.add(CO_EX + i, cF * fE + cU * cE);
    }
    {
        T fPhi = a * sg * B[D], fPsi = a * sg * E[D];
        if (!FLAT) {
            fPhi -= bD * Phi;
            fPsi -= bD * Psi;
        }
        acc.add(CO_PHI, cF * fPhi + cU * Phi);
        acc.add(CO_PSI, cF * fPsi + cU * Psi);
    }
    T J = Jd;
    if (!useJ) {
        // Ohm's law: Q v^D + W sigma [calE^D + eps^{Djk} v_j calB_k - (v.calE) v^D]
        T vB[3];
        cross3(vl, Bl, vB);
        J = Qc * v[D] + W * sigma * (sg * E[D] + vB[D] - sg * dot3(vl, E) * v[D]);
    }
    {
        T f = a * J;
        if (!FLAT) f -= bD * Qc;
        acc.add(CO_Q, cF * f + cU * Qc);
    }
}

// prim -> con only (set-up, atmosphere resets)
template <class T, bool FLAT>
__device__ __forceinline__ void prim_to_cons(const T pr[NPR], const Met<T> &m, T gfac,
                                             T U[NCO])
{
    const T sg = FLAT ? T(1) : m.sg;
    T v[3] = {pr[PR_VX], pr[PR_VY], pr[PR_VZ]};
    T E[3] = {pr[PR_EX], pr[PR_EY], pr[PR_EZ]};
    T B[3] = {pr[PR_BX], pr[PR_BY], pr[PR_BZ]};
    T vl[3], El[3], Bl[3];
    lower<T, FLAT>(m, v, vl);
    lower<T, FLAT>(m, E, El);
    lower<T, FLAT>(m, B, Bl);
    const T rho = pr[PR_RHO], p = pr[PR_P];
    const T W = T(1) / sqrt(T(1) - dot3(v, vl));
    const T hW2 = (rho + gfac * p) * W * W;
    const T em = T(0.5) * (dot3(E, El) + dot3(B, Bl));
    U[CO_D] = sg * rho * W;
    U[CO_TAU] = sg * (hW2 - p + em) - U[CO_D];
    T ExB[3];
    cross3(E, B, ExB);
#pragma unroll
    for (int i = 0; i < 3; i++) {
        U[CO_SX + i] = sg * (hW2 * vl[i] + sg * ExB[i]);
        U[CO_BX + i] = sg * B[i];
        U[CO_EX + i] = sg * E[i];
    }
    U[CO_PHI] = sg * pr[PR_PHI];
    U[CO_PSI] = sg * pr[PR_PSI];
    U[CO_Q] = sg * pr[PR_Q];
}

// ---------------------------------------------------------------------------
// Reconstruction of a six-point stencil s[0..5] = u_{i-2..i+3} to the left
// (from u_i) and right (from u_{i+1}) states of the face between u_i, u_{i+1}.
// ---------------------------------------------------------------------------
enum { RC_MINMOD = 0, RC_MC2 = 1, RC_WENO5 = 2 };

// minmod limiters: 0 unless all arguments share a sign, else the one nearest
// zero.  In FP32 (issue-bound stencil) written with selects and no
// branches; in FP64 (FP64-pipe-bound) with branches, so that only the
// needed min or max is computed.  Same value either way.
template <class T> __device__ __forceinline__ T mm2(T a, T b)
{
    if (sizeof(T) == sizeof(float)) {
        const T r = fabs(a) <= fabs(b) ? a : b;
        return a * b <= T(0) ? T(0) : r;
    }
    if (a * b <= T(0)) return T(0);
    return fabs(a) <= fabs(b) ? a : b;
}

// mm3 on doubles with integer operations on the bit patterns, for the FP64
// pipe-bound flux kernels (on B300 the FP64 pipe runs compares and min/max
// at the rate of an FMA): x > 0 holds for the patterns 1 .. 0x7ff0...0
// (NaN and +-0 excluded), x < 0 for those with the sign bit and a magnitude
// in the same range, and same-signed doubles order like their magnitude
// patterns.  Same result as the floating-point form for every input.
__device__ __forceinline__ double mm3_bits(double a, double b, double c)
{
    const unsigned long long MAG = 0x7fffffffffffffffULL, INF = 0x7ff0000000000000ULL;
    const unsigned long long ua = (unsigned long long)__double_as_longlong(a),
                             ub = (unsigned long long)__double_as_longlong(b),
                             uc = (unsigned long long)__double_as_longlong(c);
    const unsigned long long ma = ua & MAG, mb = ub & MAG, mc = uc & MAG;
    // every magnitude a nonzero number (not NaN), and all signs equal
    const bool num = (ma - 1ULL < INF) & (mb - 1ULL < INF) & (mc - 1ULL < INF);
    const unsigned long long sgn = ua & ~MAG;
    if (!num || (ub & ~MAG) != sgn || (uc & ~MAG) != sgn) return 0.0;
    // the value nearest zero: the smallest magnitude, with the common sign
    unsigned long long m = ma < mb ? ma : mb;
    m = m < mc ? m : mc;
    return __longlong_as_double((long long)(sgn | m));
}

// mm3 on floats for the issue-bound FP32 stencil: the smallest magnitude
// by two min instructions on |a|, |b|, |c|, given a's sign; zero when the
// signs differ, which (a ^ b) | (a ^ c) shows in its sign bit.  A zero
// argument makes the magnitude zero.  Same value as the comparison form
// for every non-NaN input (a zero result may carry a's sign).  NaN
// arguments differ from the FP64 limiters: fminf ignores a NaN, so with
// one NaN argument and the other two of a's sign the result is the smaller
// of those two (the FP64 forms return 0); a NaN a gives a NaN slope.  The
// mixed path's primitives are finite wherever the stencil reads them (a
// non-finite conserved value stops the step with RMHD_ENAN first).
__device__ __forceinline__ float mm3_f32(float a, float b, float c)
{
    const float m = fminf(fabsf(a), fminf(fabsf(b), fabsf(c)));
    const unsigned ua = __float_as_uint(a), ub = __float_as_uint(b), uc = __float_as_uint(c);
    const unsigned differ = ((ua ^ ub) | (ua ^ uc)) & 0x80000000u;
    return differ ? 0.0f : __uint_as_float(__float_as_uint(m) | (ua & 0x80000000u));
}

template <class T> __device__ __forceinline__ T mm3(T a, T b, T c)
{
    if constexpr (std::is_same<T, float>::value) {
        return mm3_f32(a, b, c);
    }
    if constexpr (std::is_same<T, double>::value) {
        return mm3_bits(a, b, c);
    } else {
        if (a > T(0) && b > T(0) && c > T(0)) return fmin(a, fmin(b, c));
        if (a < T(0) && b < T(0) && c < T(0)) return fmax(a, fmax(b, c));
        return T(0);
    }
}

template <class T, int RC> __device__ __forceinline__ T tvd_slope(T um, T u0, T up)
{
    if (RC == RC_MINMOD) return mm2(u0 - um, up - u0);
    return mm3(T(2) * (u0 - um), T(0.5) * (up - um), T(2) * (up - u0));
}

// Jiang-Shu WENO5 face value between c and d from (a..e) = u_{i-2..i+2}
// FP64 WENO5 with every rounding written out (explicit FMAs, products and
// sums that the compiler may not contract): the run flux kernel inlines the
// reconstruction of a run's first cell apart from the others, and with
// contraction left to the compiler the two copies could round differently,
// making a face's value depend on where a run starts (a grid cut into
// z-slabs would then not reproduce the whole grid bit for bit).  Same
// weights and algebra as the generic form below.
__device__ __forceinline__ double weno5_f64(double a, double b, double c, double d, double e)
{
    const double eps = 1e-6, sixth = 1.0 / 6.0, k13 = 13.0 / 12.0;
    const double q0 = __dmul_rn(__fma_rn(11.0, c, __fma_rn(-7.0, b, __dmul_rn(2.0, a))), sixth);
    const double q1 = __dmul_rn(__fma_rn(2.0, d, __fma_rn(5.0, c, -b)), sixth);
    const double q2 = __dmul_rn(__dsub_rn(__fma_rn(5.0, d, __dmul_rn(2.0, c)), e), sixth);
    double t1 = __dadd_rn(__fma_rn(-2.0, b, a), c);
    double t2 = __fma_rn(3.0, c, __fma_rn(-4.0, b, a));
    const double b0 = __fma_rn(__dmul_rn(k13, t1), t1, __dmul_rn(__dmul_rn(0.25, t2), t2));
    t1 = __dadd_rn(__fma_rn(-2.0, c, b), d);
    t2 = __dsub_rn(b, d);
    const double b1 = __fma_rn(__dmul_rn(k13, t1), t1, __dmul_rn(__dmul_rn(0.25, t2), t2));
    t1 = __dadd_rn(__fma_rn(-2.0, d, c), e);
    t2 = __dadd_rn(__fma_rn(-4.0, d, __dmul_rn(3.0, c)), e);
    const double b2 = __fma_rn(__dmul_rn(k13, t1), t1, __dmul_rn(__dmul_rn(0.25, t2), t2));
    // the normalised weights d_k/s_k / sum_j d_j/s_j, s_k = (eps + b_k)^2,
    // over the common denominator s_0 s_1 s_2: one division instead of
    // four (FP64 divisions are a sequence of FP64-pipe instructions on
    // B300).  The products stay finite while every b_k < 1e77, i.e. for
    // jumps below ~1e38 in a primitive; FP32 keeps the four divisions,
    // whose products would overflow much sooner.
    const double e0 = __dadd_rn(eps, b0), e1 = __dadd_rn(eps, b1), e2 = __dadd_rn(eps, b2);
    const double s0 = __dmul_rn(e0, e0), s1 = __dmul_rn(e1, e1), s2 = __dmul_rn(e2, e2);
    const double n0 = __dmul_rn(0.1, __dmul_rn(s1, s2)), n1 = __dmul_rn(0.6, __dmul_rn(s0, s2)),
                 n2 = __dmul_rn(0.3, __dmul_rn(s0, s1));
    const double num = __fma_rn(n2, q2, __fma_rn(n1, q1, __dmul_rn(n0, q0)));
    return num / __dadd_rn(__dadd_rn(n0, n1), n2);
}

template <class T> __device__ __forceinline__ T weno5(T a, T b, T c, T d, T e)
{
    if constexpr (std::is_same<T, double>::value) return weno5_f64(a, b, c, d, e);
    const T eps = T(1e-6);
    const T sixth = T(1) / T(6);
    T q0 = (T(2) * a - T(7) * b + T(11) * c) * sixth;
    T q1 = (-b + T(5) * c + T(2) * d) * sixth;
    T q2 = (T(2) * c + T(5) * d - e) * sixth;
    const T k13 = T(13) / T(12);
    T t1 = a - T(2) * b + c, t2 = a - T(4) * b + T(3) * c;
    T b0 = k13 * t1 * t1 + T(0.25) * t2 * t2;
    t1 = b - T(2) * c + d;
    t2 = b - d;
    T b1 = k13 * t1 * t1 + T(0.25) * t2 * t2;
    t1 = c - T(2) * d + e;
    t2 = T(3) * c - T(4) * d + e;
    T b2 = k13 * t1 * t1 + T(0.25) * t2 * t2;
    if constexpr (std::is_same<T, float>::value) {
        // FP32: the approximate division (__fdividef, within 2 ulp for
        // divisors below 2^126) instead of the IEEE sequence, four per state
        const float w0 = __fdividef(0.1f, (eps + b0) * (eps + b0));
        const float w1 = __fdividef(0.6f, (eps + b1) * (eps + b1));
        const float w2 = __fdividef(0.3f, (eps + b2) * (eps + b2));
        return __fdividef(w0 * q0 + w1 * q1 + w2 * q2, w0 + w1 + w2);
    } else {
        T w0 = T(0.1) / ((eps + b0) * (eps + b0));
        T w1 = T(0.6) / ((eps + b1) * (eps + b1));
        T w2 = T(0.3) / ((eps + b2) * (eps + b2));
        return (w0 * q0 + w1 * q1 + w2 * q2) / (w0 + w1 + w2);
    }
}

template <class T, int RC>
__device__ __forceinline__ void reconstruct(const T s[6], T &uL, T &uR)
{
    if (RC == RC_WENO5) {
        uL = weno5(s[0], s[1], s[2], s[3], s[4]);
        uR = weno5(s[5], s[4], s[3], s[2], s[1]);
    } else {
        uL = s[2] + T(0.5) * tvd_slope<T, RC>(s[1], s[2], s[3]);
        uR = s[3] - T(0.5) * tvd_slope<T, RC>(s[2], s[3], s[4]);
    }
}

} // namespace rmhd
