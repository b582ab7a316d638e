// FP64 exp, expm1, log and log1p for the FP64 property paths, written for
// fewer FP64-pipe operations than general library calls: the FP64 pipe is
// the scarce unit of these kernels (2 operations per clock per SM on GB300),
// and the exponentials and logarithms of Chung's correlation and of the
// departure functions take about a third of its slots.
//
// exp: Tang's table-driven method (P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point
// arithmetic", ACM TOMS 15 (1989) 144-157) with 64 table points: x =
// (64 m + j) ln2/64 + r, |r| <= ln2/128, exp(x) = 2^m 2^(j/64) e^r, the
// reduction in double-double by FMA, e^r - 1 by its Taylor polynomial to r^5
// (the next term is below 3.4e-17 of the result; to r^7 for expm1, whose
// result can be of the size of r), 2^(j/64) as a double-double table, 2^m
// added to the exponent field.  11 FP64 operations (expm1: 15).
// log: Tang's table-driven logarithm (ACM TOMS 16 (1990) 378-400) with
// F = 1 + j/128 nearest the significand m: ln x = e ln2 + ln F + ln(1 + r),
// r = (m - F)/F (m - F exact; 1/F from a table and one correction step),
// ln(1 + r) by its Taylor polynomial to r^8 (|r| <= 1/256).  18 FP64
// operations.
// Valid for finite positive normal x; exp for |x| < 512 (larger |x|, NaN and
// infinities go to CUDA's exp).  Errors on the tested ranges
// (tests/test_gpu_math64.py, extended-precision references): exp 0.75 ulp,
// expm1 1.44, log 1.00, log1p 1.46 at most (CUDA's: 0.85, 1.05, 0.50, 1.46).
#pragma once

#include <cuda_runtime.h>

#include "math64_tables.h"

namespace m64 {

// round-to-nearest integer of x * 64/ln2 via the 1.5 * 2^52 shifter
constexpr double kShift = 6755399441055744.0;

// |x| < 512, from the exponent field of the high word (integer pipe)
__device__ __forceinline__ bool exp_in_range(double x)
{
    return ((__double2hiint(x) >> 20) & 0x7FF) < 1023 + 9;
}

// e^r - 1 for |r| <= ln2/128, to the r^5 term: the truncation is below
// 3.4e-17 of 1 + p, enough for exp
__device__ __forceinline__ double expm1_small(double r)
{
    const double r2 = r * r;
    double q = fma(r, 1.0 / 120.0, 1.0 / 24.0);
    q = fma(q, r, 1.0 / 6.0);
    q = fma(q, r, 0.5);
    return fma(q, r2, r);
}

// the same to the r^7 term: the truncation is below 5e-18 of p itself, as
// expm1 needs when its result is of the size of r
__device__ __forceinline__ double expm1_small_rel(double r)
{
    const double r2 = r * r;
    double q = fma(r, 1.0 / 5040.0, 1.0 / 720.0);
    q = fma(q, r, 1.0 / 120.0);
    q = fma(q, r, 1.0 / 24.0);
    q = fma(q, r, 1.0 / 6.0);
    q = fma(q, r, 0.5);
    return fma(q, r2, r);
}

__device__ __forceinline__ double exp(double x)
{
    if (!exp_in_range(x)) return ::exp(x);
    const double t = fma(x, k64OverLn2, kShift);
    const double kd = t - kShift;
    const int k = __double2loint(t);
    double r = fma(-kd, kLn2Over64Hi, x);
    r = fma(-kd, kLn2Over64Lo, r);
    const double p = expm1_small(r);
    const int j = k & 63, m = k >> 6;
    const double th = __ldg(&kExp2Hi[j]), tl = __ldg(&kExp2Lo[j]);
    const double v = th + fma(th, p, tl);
    return __hiloint2double(__double2hiint(v) + (m << 20), __double2loint(v));
}

// e^x - 1: as exp, with the 1 taken off before the scaled table value is
// rounded, so that small x keep their relative accuracy
__device__ __forceinline__ double expm1(double x)
{
    if (!exp_in_range(x)) return ::expm1(x);
    const double t = fma(x, k64OverLn2, kShift);
    const double kd = t - kShift;
    const int k = __double2loint(t);
    double r = fma(-kd, kLn2Over64Hi, x);
    r = fma(-kd, kLn2Over64Lo, r);
    const double p = expm1_small_rel(r);
    const int j = k & 63, m = k >> 6;
    if (k == 0) return p;
    const double s = __hiloint2double((1023 + m) << 20, 0);   // 2^m
    const double th = __ldg(&kExp2Hi[j]) * s, tl = __ldg(&kExp2Lo[j]) * s;
    // 2^m 2^(j/64) (1 + p) - 1 = (th - 1) + (th p + tl); th - 1 is exact while th is within [1/2, 2]
    return (th - 1.0) + fma(th, p, tl);
}

// ln(1 + r) for |r| <= 1/256, to the r^8 term (the truncation is below
// 2^-64 / 9 of r: near x = 1 the logarithm is of the size of r)
__device__ __forceinline__ double log1p_small(double r)
{
    const double r2 = r * r;
    double q = fma(r, -1.0 / 8.0, 1.0 / 7.0);
    q = fma(q, r, -1.0 / 6.0);
    q = fma(q, r, 0.2);
    q = fma(q, r, -0.25);
    q = fma(q, r, 1.0 / 3.0);
    q = fma(q, r, -0.5);
    return fma(q, r2, r);
}

// ln x for finite positive normal x
__device__ __forceinline__ double log(double x)
{
    const int hx = __double2hiint(x), lx = __double2loint(x);
    const int ex = (hx >> 20) & 0x7FF;
    if (ex == 0 || ex == 0x7FF || hx < 0) return ::log(x);
    // significand m in [1, 2); j: its leading 7 fraction bits, rounded
    const double m = __hiloint2double((hx & 0x000FFFFF) | 0x3FF00000, lx);
    const int j = ((hx & 0x000FFFFF) + (1 << 12)) >> 13;       // 0..128
    const double F = __hiloint2double(0x3FF00000 + (j << 13), 0);   // 1 + j/128 (2 for j = 128)
    // r = (m - F) / F: the product with the rounded 1/F, then one correction
    // step from the exact residual (m - F) - r F
    const double f = m - F, iF = __ldg(&kInvF[j]);
    double r = f * iF;
    r = fma(fma(-r, F, f), iF, r);
    const double lp = log1p_small(r);
    const double e = (double)(ex - 1023);
    const double hi = fma(e, kLn2Hi, __ldg(&kLogFHi[j]));
    const double lo = fma(e, kLn2Lo, __ldg(&kLogFLo[j]));
    return hi + (lp + lo);
}

// ln(1 + z) for z > -1: ln u of the rounded u = 1 + z, plus the rounding
// error of u over u (a tiny correction, taken with a single-precision 1/u)
__device__ __forceinline__ double log1p(double z)
{
    const double u = 1.0 + z;
    const double c = z - (u - 1.0);
    return log(u) + c * (double)__frcp_rn((float)u);
}

}  // namespace m64
