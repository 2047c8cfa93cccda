// Forward-mode dual numbers: value plus K partial derivatives, used to obtain the exact
// cell-local Jacobian blocks of the residual (the derivatives of S_e and S_n) in the same
// pass that evaluates them.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#define RT_HD __host__ __device__ __forceinline__

template <int K>
struct Dual {
    double v;
    double d[K];
};

template <int K>
RT_HD Dual<K> dconst(double v) {
    Dual<K> r;
    r.v = v;
#pragma unroll
    for (int i = 0; i < K; ++i) r.d[i] = 0.0;
    return r;
}

template <int K>
RT_HD Dual<K> dvar(double v, int which) {
    Dual<K> r = dconst<K>(v);
    r.d[which] = 1.0;
    return r;
}

// r = a*v' + b*w' chain helper: value f, derivative scale s (f' = s * x')
template <int K>
RT_HD Dual<K> dchain(const Dual<K>& x, double f, double s) {
    Dual<K> r;
    r.v = f;
#pragma unroll
    for (int i = 0; i < K; ++i) r.d[i] = s * x.d[i];
    return r;
}

template <int K>
RT_HD Dual<K> operator+(const Dual<K>& a, const Dual<K>& b) {
    Dual<K> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int i = 0; i < K; ++i) r.d[i] = a.d[i] + b.d[i];
    return r;
}
template <int K>
RT_HD Dual<K> operator-(const Dual<K>& a, const Dual<K>& b) {
    Dual<K> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int i = 0; i < K; ++i) r.d[i] = a.d[i] - b.d[i];
    return r;
}
template <int K>
RT_HD Dual<K> operator-(const Dual<K>& a) {
    Dual<K> r;
    r.v = -a.v;
#pragma unroll
    for (int i = 0; i < K; ++i) r.d[i] = -a.d[i];
    return r;
}
template <int K>
RT_HD Dual<K> operator*(const Dual<K>& a, const Dual<K>& b) {
    Dual<K> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int i = 0; i < K; ++i) r.d[i] = fma(a.d[i], b.v, a.v * b.d[i]);
    return r;
}
template <int K>
RT_HD Dual<K> operator/(const Dual<K>& a, const Dual<K>& b) {
    const double inv = 1.0 / b.v;
    Dual<K> r;
    r.v = a.v * inv;
#pragma unroll
    for (int i = 0; i < K; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * inv;
    return r;
}
template <int K>
RT_HD Dual<K> operator+(const Dual<K>& a, double s) { Dual<K> r = a; r.v += s; return r; }
template <int K>
RT_HD Dual<K> operator+(double s, const Dual<K>& a) { return a + s; }
template <int K>
RT_HD Dual<K> operator-(const Dual<K>& a, double s) { Dual<K> r = a; r.v -= s; return r; }
template <int K>
RT_HD Dual<K> operator-(double s, const Dual<K>& a) { return (-a) + s; }
template <int K>
RT_HD Dual<K> operator*(const Dual<K>& a, double s) {
    Dual<K> r;
    r.v = a.v * s;
#pragma unroll
    for (int i = 0; i < K; ++i) r.d[i] = a.d[i] * s;
    return r;
}
template <int K>
RT_HD Dual<K> operator*(double s, const Dual<K>& a) { return a * s; }
template <int K>
RT_HD Dual<K> operator/(const Dual<K>& a, double s) { return a * (1.0 / s); }
template <int K>
RT_HD Dual<K> operator/(double s, const Dual<K>& b) {
    const double inv = 1.0 / b.v;
    return dchain(b, s * inv, -s * inv * inv);
}

template <int K>
RT_HD Dual<K> sqrt(const Dual<K>& a) {
    const double s = ::sqrt(a.v);
    return dchain(a, s, s > 0.0 ? 0.5 / s : 0.0);
}
template <int K>
RT_HD Dual<K> exp(const Dual<K>& a) {
    const double e = ::exp(a.v);
    return dchain(a, e, e);
}
template <int K>
RT_HD Dual<K> expm1(const Dual<K>& a) {
    const double e = ::expm1(a.v);
    return dchain(a, e, e + 1.0);
}
template <int K>
RT_HD Dual<K> log(const Dual<K>& a) { return dchain(a, ::log(a.v), 1.0 / a.v); }
template <int K>
RT_HD Dual<K> log1p(const Dual<K>& a) { return dchain(a, ::log1p(a.v), 1.0 / (1.0 + a.v)); }
template <int K>
RT_HD Dual<K> pow(const Dual<K>& a, double p) {
    const double v = ::pow(a.v, p);
    return dchain(a, v, p * v / a.v);
}

RT_HD double value(double x) { return x; }
template <int K>
RT_HD double value(const Dual<K>& x) { return x.v; }
