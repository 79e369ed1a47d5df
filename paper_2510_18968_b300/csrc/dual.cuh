// dual.cuh -- forward-mode dual numbers for the adjoint kernels.
//
// Dual<N> carries a value and N directional derivatives.  Running the same
// templated device physics on Dual<N> with unit seeds gives N columns of its
// Jacobian at the evaluation point; the adjoint kernels transpose those
// columns against the incoming adjoint.  Comparisons and branches act on the
// value only, so a dual evaluation follows the branch the FP64 evaluation
// takes and differentiates that branch (limiter selections, first-order
// fallbacks, the atmosphere reset are frozen at the primal point).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace rmhd {

// keep the plain overloads visible next to the dual ones below
using ::fabs;
using ::fmax;
using ::fmin;
using ::rsqrt;
using ::sqrt;

template <int N> struct Dual {
    double v;
    double d[N];
    __host__ __device__ Dual() : v(0.0)
    {
#pragma unroll
        for (int k = 0; k < N; k++) d[k] = 0.0;
    }
    __host__ __device__ Dual(double x) : v(x)
    {
#pragma unroll
        for (int k = 0; k < N; k++) d[k] = 0.0;
    }
    __host__ __device__ explicit operator double() const { return v; }
    __host__ __device__ Dual &operator+=(const Dual &b)
    {
        v += b.v;
#pragma unroll
        for (int k = 0; k < N; k++) d[k] += b.d[k];
        return *this;
    }
    __host__ __device__ Dual &operator-=(const Dual &b)
    {
        v -= b.v;
#pragma unroll
        for (int k = 0; k < N; k++) d[k] -= b.d[k];
        return *this;
    }
    __host__ __device__ Dual &operator*=(const Dual &b)
    {
#pragma unroll
        for (int k = 0; k < N; k++) d[k] = d[k] * b.v + v * b.d[k];
        v *= b.v;
        return *this;
    }
};

// a dual with derivative 1 in direction k
template <int N> __host__ __device__ inline Dual<N> seed(double x, int k)
{
    Dual<N> r(x);
    r.d[k] = 1.0;
    return r;
}

template <int N> __host__ __device__ inline Dual<N> operator-(const Dual<N> &a)
{
    Dual<N> r;
    r.v = -a.v;
#pragma unroll
    for (int k = 0; k < N; k++) r.d[k] = -a.d[k];
    return r;
}
template <int N> __host__ __device__ inline Dual<N> operator+(const Dual<N> &a, const Dual<N> &b)
{
    Dual<N> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int k = 0; k < N; k++) r.d[k] = a.d[k] + b.d[k];
    return r;
}
template <int N> __host__ __device__ inline Dual<N> operator-(const Dual<N> &a, const Dual<N> &b)
{
    Dual<N> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int k = 0; k < N; k++) r.d[k] = a.d[k] - b.d[k];
    return r;
}
template <int N> __host__ __device__ inline Dual<N> operator*(const Dual<N> &a, const Dual<N> &b)
{
    Dual<N> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int k = 0; k < N; k++) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
template <int N> __host__ __device__ inline Dual<N> operator/(const Dual<N> &a, const Dual<N> &b)
{
    Dual<N> r;
    const double ib = 1.0 / b.v;
    r.v = a.v * ib;
#pragma unroll
    for (int k = 0; k < N; k++) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
    return r;
}
// mixed operands: a plain double is a constant
template <int N> __host__ __device__ inline Dual<N> operator+(const Dual<N> &a, double b)
{
    Dual<N> r = a;
    r.v += b;
    return r;
}
template <int N> __host__ __device__ inline Dual<N> operator+(double a, const Dual<N> &b)
{
    return b + a;
}
template <int N> __host__ __device__ inline Dual<N> operator-(const Dual<N> &a, double b)
{
    Dual<N> r = a;
    r.v -= b;
    return r;
}
template <int N> __host__ __device__ inline Dual<N> operator-(double a, const Dual<N> &b)
{
    Dual<N> r = -b;
    r.v += a;
    return r;
}
template <int N> __host__ __device__ inline Dual<N> operator*(const Dual<N> &a, double b)
{
    Dual<N> r;
    r.v = a.v * b;
#pragma unroll
    for (int k = 0; k < N; k++) r.d[k] = a.d[k] * b;
    return r;
}
template <int N> __host__ __device__ inline Dual<N> operator*(double a, const Dual<N> &b)
{
    return b * a;
}
template <int N> __host__ __device__ inline Dual<N> operator/(const Dual<N> &a, double b)
{
    return a * (1.0 / b);
}
template <int N> __host__ __device__ inline Dual<N> operator/(double a, const Dual<N> &b)
{
    return Dual<N>(a) / b;
}

#define RMHD_DUAL_CMP(op)                                                                   \
    template <int N> __host__ __device__ inline bool operator op(const Dual<N> &a,          \
                                                                 const Dual<N> &b)          \
    {                                                                                       \
        return a.v op b.v;                                                                  \
    }                                                                                       \
    template <int N> __host__ __device__ inline bool operator op(const Dual<N> &a, double b) \
    {                                                                                       \
        return a.v op b;                                                                    \
    }                                                                                       \
    template <int N> __host__ __device__ inline bool operator op(double a, const Dual<N> &b) \
    {                                                                                       \
        return a op b.v;                                                                    \
    }
RMHD_DUAL_CMP(<)
RMHD_DUAL_CMP(<=)
RMHD_DUAL_CMP(>)
RMHD_DUAL_CMP(>=)
RMHD_DUAL_CMP(==)
#undef RMHD_DUAL_CMP

// d sqrt(x) = dx / (2 sqrt(x))
template <int N> __device__ inline Dual<N> sqrt(const Dual<N> &a)
{
    Dual<N> r;
    r.v = ::sqrt(a.v);
    const double h = 0.5 / r.v;
#pragma unroll
    for (int k = 0; k < N; k++) r.d[k] = a.d[k] * h;
    return r;
}
// d x^{-1/2} = -x^{-3/2} dx / 2
template <int N> __device__ inline Dual<N> rsqrt(const Dual<N> &a)
{
    Dual<N> r;
    r.v = ::rsqrt(a.v);
    const double h = -0.5 * r.v / a.v;
#pragma unroll
    for (int k = 0; k < N; k++) r.d[k] = a.d[k] * h;
    return r;
}
template <int N> __device__ inline Dual<N> fabs(const Dual<N> &a) { return a.v < 0.0 ? -a : a; }
template <int N> __device__ inline Dual<N> fmin(const Dual<N> &a, const Dual<N> &b)
{
    return b.v < a.v ? b : a;
}
template <int N> __device__ inline Dual<N> fmax(const Dual<N> &a, const Dual<N> &b)
{
    return b.v > a.v ? b : a;
}

// value of a plain or dual number
__device__ __forceinline__ double val(double x) { return x; }
template <int N> __device__ __forceinline__ double val(const Dual<N> &x) { return x.v; }

} // namespace rmhd
