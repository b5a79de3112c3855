// mts_dual.cuh -- forward-mode dual numbers for the per-particle stress
// derivatives of the adjoint.  A Dual<T, N> carries a value and its
// derivatives along N seeded input directions; the stress laws in
// mts_device.cuh are templates on the real type, so instantiating them with a
// Dual evaluates the law and N columns of its Jacobian in one pass (chain
// rule applied operation by operation).  Comparisons and branches use the
// value, so a derivative is that of the branch the value takes.
#pragma once

#include <cmath>

namespace mts {

template <class T, int N>
struct Dual {
    T v;
    T d[N];
    __device__ __forceinline__ Dual() {}
    __device__ __forceinline__ Dual(T x) : v(x) {
#pragma unroll
        for (int i = 0; i < N; ++i) d[i] = T(0);
    }
};

#define MTS_DUAL_T template <class T, int N>
#define MTS_D Dual<T, N>

MTS_DUAL_T __device__ __forceinline__ MTS_D operator+(const MTS_D &a, const MTS_D &b) {
    MTS_D r;
    r.v = a.v + b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
    return r;
}
MTS_DUAL_T __device__ __forceinline__ MTS_D operator-(const MTS_D &a, const MTS_D &b) {
    MTS_D r;
    r.v = a.v - b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
    return r;
}
MTS_DUAL_T __device__ __forceinline__ MTS_D operator-(const MTS_D &a) {
    MTS_D r;
    r.v = -a.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
    return r;
}
MTS_DUAL_T __device__ __forceinline__ MTS_D operator*(const MTS_D &a, const MTS_D &b) {
    MTS_D r;
    r.v = a.v * b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
MTS_DUAL_T __device__ __forceinline__ MTS_D operator/(const MTS_D &a, const MTS_D &b) {
    MTS_D r;
    const T ib = T(1) / b.v;
    r.v = a.v * ib;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
    return r;
}
MTS_DUAL_T __device__ __forceinline__ MTS_D &operator+=(MTS_D &a, const MTS_D &b) { return a = a + b; }
MTS_DUAL_T __device__ __forceinline__ MTS_D &operator-=(MTS_D &a, const MTS_D &b) { return a = a - b; }
MTS_DUAL_T __device__ __forceinline__ MTS_D &operator*=(MTS_D &a, const MTS_D &b) { return a = a * b; }
MTS_DUAL_T __device__ __forceinline__ bool operator<(const MTS_D &a, const MTS_D &b) { return a.v < b.v; }
MTS_DUAL_T __device__ __forceinline__ bool operator>(const MTS_D &a, const MTS_D &b) { return a.v > b.v; }
MTS_DUAL_T __device__ __forceinline__ bool operator<=(const MTS_D &a, const MTS_D &b) { return a.v <= b.v; }
MTS_DUAL_T __device__ __forceinline__ bool operator>=(const MTS_D &a, const MTS_D &b) { return a.v >= b.v; }

// sqrt, with a zero derivative at 0 (the norm of a vanishing deviator)
MTS_DUAL_T __device__ __forceinline__ MTS_D dsqrt(const MTS_D &a) {
    MTS_D r;
    r.v = sqrt(a.v);
    const T f = r.v > T(0) ? T(0.5) / r.v : T(0);
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = f * a.d[i];
    return r;
}
MTS_DUAL_T __device__ __forceinline__ MTS_D dexp(const MTS_D &a) {
    MTS_D r;
    r.v = exp(a.v);
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = r.v * a.d[i];
    return r;
}
// x^(-1/3): derivative -x^(-4/3)/3 = -r / (3 x)
MTS_DUAL_T __device__ __forceinline__ MTS_D drcbrt(const MTS_D &a) {
    MTS_D r;
    r.v = rcbrt(a.v);
    const T f = -r.v / (T(3) * a.v);
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = f * a.d[i];
    return r;
}
MTS_DUAL_T __device__ __forceinline__ MTS_D dabs(const MTS_D &a) { return a.v < T(0) ? -a : a; }

#undef MTS_D
#undef MTS_DUAL_T

// Newton tolerance of the return mapping for a real type (FP64 / FP32) and
// for duals over it
template <class R> struct NewtonTol { static constexpr double value = sizeof(R) == 8 ? 1e-13 : 1e-6; };
template <class T, int N> struct NewtonTol<Dual<T, N>> { static constexpr double value = NewtonTol<T>::value; };

}  // namespace mts
