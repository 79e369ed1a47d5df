/*
 * tangent.h -- TEST INFRASTRUCTURE ONLY: forward-mode tangent numbers for the
 * tangent-linear build of the oracle (rmhd_oracle.c compiled as C++ with
 * ORC_TANGENT defined).
 *
 * A tangent number carries a value v and its directional derivative d; every
 * operation applies the chain rule to d alongside the FP64 operation on v, so
 * that the oracle's step, run on tangent numbers seeded with a direction u of
 * its inputs, returns the step's results and their derivatives along u (the
 * tangent-linear model).  Comparisons look at v only: branches (limiters,
 * recovery decisions, atmosphere resets) are taken as the value path takes
 * them and their derivative follows the branch taken.  v is computed by the
 * same FP64 operations as in the plain C build.
 */
#ifndef ORC_TANGENT_H
#define ORC_TANGENT_H

#include <cmath>
#include <math.h>

struct tl {
    double v, d;
    tl() : v(0.0), d(0.0) {}
    tl(double x) : v(x), d(0.0) {}
    tl(double x, double dx) : v(x), d(dx) {}
    tl &operator+=(const tl &b) { d += b.d; v += b.v; return *this; }
    tl &operator-=(const tl &b) { d -= b.d; v -= b.v; return *this; }
    tl &operator*=(const tl &b) { *this = tl(v * b.v, d * b.v + v * b.d); return *this; }
    tl &operator/=(const tl &b) { *this = tl(v / b.v, (d * b.v - v * b.d) / (b.v * b.v)); return *this; }
};

static inline tl operator+(const tl &a, const tl &b) { return tl(a.v + b.v, a.d + b.d); }
static inline tl operator-(const tl &a, const tl &b) { return tl(a.v - b.v, a.d - b.d); }
static inline tl operator-(const tl &a) { return tl(-a.v, -a.d); }
static inline tl operator+(const tl &a) { return a; }
static inline tl operator*(const tl &a, const tl &b) { return tl(a.v * b.v, a.d * b.v + a.v * b.d); }
static inline tl operator/(const tl &a, const tl &b)
{
    const double q = a.v / b.v;
    return tl(q, (a.d - q * b.d) / b.v);
}
static inline tl operator+(const tl &a, double b) { return tl(a.v + b, a.d); }
static inline tl operator+(double a, const tl &b) { return tl(a + b.v, b.d); }
static inline tl operator-(const tl &a, double b) { return tl(a.v - b, a.d); }
static inline tl operator-(double a, const tl &b) { return tl(a - b.v, -b.d); }
static inline tl operator*(const tl &a, double b) { return tl(a.v * b, a.d * b); }
static inline tl operator*(double a, const tl &b) { return tl(a * b.v, a * b.d); }
static inline tl operator/(const tl &a, double b) { return tl(a.v / b, a.d / b); }
static inline tl operator/(double a, const tl &b)
{
    const double q = a / b.v;
    return tl(q, -q * b.d / b.v);
}

#define TL_CMP(op)                                                                    \
    static inline bool operator op(const tl &a, const tl &b) { return a.v op b.v; }    \
    static inline bool operator op(const tl &a, double b) { return a.v op b; }         \
    static inline bool operator op(double a, const tl &b) { return a op b.v; }
TL_CMP(<)
TL_CMP(>)
TL_CMP(<=)
TL_CMP(>=)
TL_CMP(==)
TL_CMP(!=)
#undef TL_CMP

static inline tl sqrt(const tl &a)
{
    const double s = sqrt(a.v);
    return tl(s, a.d / (2.0 * s));
}
static inline tl fabs(const tl &a) { return a.v < 0.0 ? -a : a; }
static inline tl fmax(const tl &a, const tl &b) { return a.v >= b.v ? a : b; }
static inline tl fmin(const tl &a, const tl &b) { return a.v <= b.v ? a : b; }
static inline tl exp(const tl &a)
{
    const double e = exp(a.v);
    return tl(e, e * a.d);
}
static inline tl log(const tl &a) { return tl(log(a.v), a.d / a.v); }
static inline tl tanh(const tl &a)
{
    const double t = tanh(a.v);
    return tl(t, (1.0 - t * t) * a.d);
}
/* x^y for a constant exponent y (and x > 0 where y is not an integer) */
static inline tl pow(const tl &a, double y)
{
    const double p = pow(a.v, y);
    return tl(p, y == 0.0 ? 0.0 : y * pow(a.v, y - 1.0) * a.d);
}
/* finiteness of the value: the value path is that of the plain build */
static inline bool isfinite(const tl &a) { return std::isfinite(a.v); }

#endif
