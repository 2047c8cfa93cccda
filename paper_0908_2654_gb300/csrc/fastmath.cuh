// Table-driven FP64 exp and log for the rate fits of the Newton evaluation kernel.
//
// GB300 issues two FP64 FMA per clock per SM, so the transcendental functions of the rate
// fits dominate the cost of the cell-local equations.  These follow the table-driven methods
// of P. T. P. Tang, "Table-driven implementation of the exponential function in IEEE
// floating-point arithmetic", ACM TOMS 15 (1989), and "Table-driven implementation of the
// logarithm function in IEEE floating-point arithmetic", ACM TOMS 16 (1990):
//
//  exp: x = (64 m + j) ln2/64 + r with |r| <= ln2/128, so exp(x) = 2^m 2^(j/64) e^r; e^r - 1 by
//       its Taylor polynomial to r^5 (truncation below 4e-17 relative); 2^(j/64) from a table.
//  log: x = 2^k m, m in [0.75, 1.5); F = j/128 the nearest 1/128 step to m; then
//       log x = k ln2 + log F + log1p(r), r = (m - F)/F with |r| <= 1/192, log1p(r) by its
//       Taylor polynomial to r^8; log F (as a high and a low part) and 1/F from tables.  r is
//       carried as r0 + r1 (an FMA correction of the rounded quotient) and the leading sum
//       k ln2 + log F + r0 is formed with Knuth's two-sum, so that results near x = 1 keep
//       full relative accuracy.
// Both are accurate to about one unit in the last place (checked against the CUDA library
// and NumPy by tests/test_gpu_fastmath.py).  Special values (NaN, +-inf, zero, negative
// arguments of log, results beyond the double range) are handled explicitly.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "fastmath_tables.cuh"

__device__ __forceinline__ double rt_exp(double x) {
    if (!(x < 709.782712893384)) return x != x ? x : __longlong_as_double(0x7ff0000000000000LL);
    if (x < -745.1332191019412) return 0.0;
    const double magic = 6755399441055744.0;             // 1.5 * 2^52: rounds to an integer
    const double t = fma(x, kInvLn2x64, magic);
    const double Nd = t - magic;                          // nearest integer to x 64/ln2
    const int N = (int)(__double_as_longlong(t) - __double_as_longlong(magic));
    const double r = fma(-Nd, kLn2By64Lo, fma(-Nd, kLn2By64Hi, x));
    const int j = N & 63;
    const int m = (N - j) / 64;
    double q = fma(r, 1.0 / 120.0, 1.0 / 24.0);
    q = fma(q, r, 1.0 / 6.0);
    q = fma(q, r, 0.5);
    q = fma(q, r, 1.0);
    const double T = kExpTable[j];
    const double v = fma(T, q * r, T);                    // 2^(j/64) e^r
    if (m > 1023) return (v * 2.0) * __longlong_as_double((long long)(1023 + 1023) << 52);
    if (m >= -1022) return v * __longlong_as_double((long long)(m + 1023) << 52);
    // subnormal result: scale in two steps
    return (v * __longlong_as_double((long long)(m + 54 + 1023) << 52)) * 5.551115123125783e-17;  // 2^-54
}

__device__ __forceinline__ double rt_log(double x) {
    if (!(x > 0.0)) return x == 0.0 ? __longlong_as_double(0xfff0000000000000LL) : __longlong_as_double(0x7ff8000000000000LL);
    long long bits = __double_as_longlong(x);
    if (bits >= 0x7ff0000000000000LL) return x;           // +inf
    int k = (int)(bits >> 52) - 1023;
    if (k == -1023) {                                      // subnormal: bring into the normal range
        bits = __double_as_longlong(x * 18014398509481984.0);   // 2^54
        k = (int)(bits >> 52) - 1023 - 54;
    }
    double m = __longlong_as_double((bits & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
    if (m >= 1.5) {                                        // m in [0.75, 1.5): no cancellation of k ln2
        m *= 0.5;                                          // against ln F for x just below 1
        k += 1;
    }
    const int j = __double2int_rn(m * 128.0);              // F = j/128 nearest m, j in [96, 192]
    const int i = j - kLogJ0;
    const double F = j * (1.0 / 128.0);
    const double f = m - F;                                // exact: m and F are within a factor 2
    const double inv = kLogInv[i];
    const double r0 = f * inv;
    const double r1 = fma(-r0, F, f) * inv;                // r0 + r1 = f/F to well below an ulp of r0
    // log1p(r) - r = r^2 (-1/2 + r/3 - ... - r^6/8), |r| <= 1/192
    double q = fma(r0, -1.0 / 8.0, 1.0 / 7.0);
    q = fma(q, r0, -1.0 / 6.0);
    q = fma(q, r0, 1.0 / 5.0);
    q = fma(q, r0, -0.25);
    q = fma(q, r0, 1.0 / 3.0);
    q = fma(q, r0, -0.5);
    const double p = q * r0 * r0;
    const double kd = (double)k;
    // k ln2_hi is exact and at least |ln F| unless k = 0: fast two-sum (Dekker) gives A + eA exactly
    const double kh = kd * kLn2Hi;
    const double A = kh + kLogHi[i];
    const double eA = kLogHi[i] - (A - kh);
    const double s = A + r0;                               // two-sum (Knuth): s + e = A + r0 exactly
    const double bb = s - A;
    const double e = (A - (s - bb)) + (r0 - bb);
    return s + ((((fma(kd, kLn2Lo, kLogLo[i]) + r1) + p) + eA) + e);
}
