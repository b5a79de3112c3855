// mts_device.cuh -- device helpers: vector loads, 3x3 algebra, constitutive laws.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace mts {

template <int D> struct Pad { static constexpr int v = (D == 2) ? 2 : 4; };
template <int D> struct MatS { static constexpr int v = (D == 2) ? 4 : 12; };

// Conversions between IEEE 754 binary32 and binary64 done on the integer
// pipe.  On this GPU a conversion to or from FP64 occupies the FP64 pipe like
// an FP64 operation, and the FP64 pipe is the drift kernel's bound; these give
// the same bits as the hardware conversions (round to nearest, ties to even)
// from the formats' definitions: sign, biased exponent (bias 127 / 1023),
// fraction (23 / 52 bits), subnormals at exponent field 0, infinities and
// NaNs at the all-ones field (NaNs come out quiet).  mts_selftest_conversions
// checks them against the hardware on random and edge-case bit patterns.
__device__ __forceinline__ double f2d_bits(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t s = b & 0x80000000u, e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
    uint32_t hi, lo;
    if (e - 1u < 254u) {                       // normal
        hi = s | ((e + 896u) << 20) | (m >> 3);
        lo = m << 29;
    } else if (e == 0u) {
        if (m == 0u) {                         // signed zero
            hi = s;
            lo = 0u;
        } else {                               // subnormal m 2^-149: normal in binary64
            const int p = 31 - __clz(m);       // leading one at bit p (0..22)
            const unsigned long long man = (unsigned long long)(m & ~(1u << p)) << (52 - p);
            hi = s | ((uint32_t)(p + 874) << 20) | (uint32_t)(man >> 32);
            lo = (uint32_t)man;
        }
    } else {                                   // infinity or NaN
        hi = s | 0x7ff00000u | (m >> 3) | (m ? 0x80000u : 0u);
        lo = m << 29;
    }
    return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ float d2f_bits(double d) {
    const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
    const uint32_t s = hi & 0x80000000u;
    const int E = (int)((hi >> 20) & 0x7ffu);
    const uint32_t mh = hi & 0xfffffu;
    if (E == 0x7ff) {                          // infinity or NaN
        const uint32_t nan = (mh | lo) ? (0x400000u | (mh << 3) | (lo >> 29)) : 0u;
        return __uint_as_float(s | 0x7f800000u | nan);
    }
    const int ef = E - 896;                    // binary32 exponent field of a normal result
    if (ef >= 255) return __uint_as_float(s | 0x7f800000u);
    if (ef >= 1) {                             // keep 23 fraction bits, round on the other 29
        const uint32_t keep = (mh << 3) | (lo >> 29), rem = lo & 0x1fffffffu;
        const uint32_t up = (rem > 0x10000000u || (rem == 0x10000000u && (keep & 1u))) ? 1u : 0u;
        return __uint_as_float(s | ((((uint32_t)ef << 23) | keep) + up));   // a carry may reach infinity
    }
    if (E == 0) return __uint_as_float(s);     // |d| < 2^-1022: rounds to zero
    // subnormal (or zero) result: the 53-bit significand times 2^(E - 1075),
    // in units of 2^-149, is sig >> (30 - ef)
    const int sh = 30 - ef;
    if (sh >= 54) return __uint_as_float(s);   // below half the smallest subnormal
    const unsigned long long sig = ((unsigned long long)(mh | 0x100000u) << 32) | lo;
    const unsigned long long q = sig >> sh, rem = sig & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    const uint32_t up = (rem > half || (rem == half && (q & 1ull))) ? 1u : 0u;
    return __uint_as_float(s | ((uint32_t)q + up));
}

// ------------------------------------------------------------------ loads
template <class R> struct Vec2;
template <> struct Vec2<float> { using T = float2; };
template <> struct Vec2<double> { using T = double2; };

// read-only vector load of N consecutive reals (N = 2 or 4), 8/16-byte aligned
template <class R, int N>
__device__ __forceinline__ void ldg_vec(R (&o)[N], const R *p) {
    if constexpr (sizeof(R) == 4 && N == 4) {
        float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    } else if constexpr (sizeof(R) == 4 && N == 2) {
        float2 t = __ldg(reinterpret_cast<const float2 *>(p));
        o[0] = t.x; o[1] = t.y;
    } else if constexpr (sizeof(R) == 8 && N == 2) {
        double2 t = __ldg(reinterpret_cast<const double2 *>(p));
        o[0] = t.x; o[1] = t.y;
    } else {
        static_assert(sizeof(R) == 8 && N == 4, "unsupported vector load");
        double2 t0 = __ldg(reinterpret_cast<const double2 *>(p));
        double2 t1 = __ldg(reinterpret_cast<const double2 *>(p) + 1);
        o[0] = t0.x; o[1] = t0.y; o[2] = t1.x; o[3] = t1.y;
    }
}

// Programmatic dependent launch (sm_90+): chain_trigger lets the next kernel
// of a substep chain be scheduled once every block of this one has started;
// chain_wait blocks until the previous kernel of the chain has completed and
// its writes are visible.  Both are no-ops for an ordinary launch.
__device__ __forceinline__ void chain_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void chain_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <class R, int N>
__device__ __forceinline__ void ld_vec(R (&o)[N], const R *p) {
    if constexpr (sizeof(R) == 4 && N == 4) {
        float4 t = *reinterpret_cast<const float4 *>(p);
        o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    } else if constexpr (sizeof(R) == 4 && N == 2) {
        float2 t = *reinterpret_cast<const float2 *>(p);
        o[0] = t.x; o[1] = t.y;
    } else if constexpr (sizeof(R) == 8 && N == 2) {
        double2 t = *reinterpret_cast<const double2 *>(p);
        o[0] = t.x; o[1] = t.y;
    } else {
        double2 t0 = reinterpret_cast<const double2 *>(p)[0];
        double2 t1 = reinterpret_cast<const double2 *>(p)[1];
        o[0] = t0.x; o[1] = t0.y; o[2] = t1.x; o[3] = t1.y;
    }
}

template <class R, int N>
__device__ __forceinline__ void st_vec(R *p, const R (&o)[N]) {
    if constexpr (sizeof(R) == 4 && N == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(o[0], o[1], o[2], o[3]);
    } else if constexpr (sizeof(R) == 4 && N == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(o[0], o[1]);
    } else if constexpr (sizeof(R) == 8 && N == 2) {
        *reinterpret_cast<double2 *>(p) = make_double2(o[0], o[1]);
    } else {
        reinterpret_cast<double2 *>(p)[0] = make_double2(o[0], o[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(o[2], o[3]);
    }
}

// store of a velocity slot to shared memory as one access of the slot's
// width: FP32 3D slots as a single 16-byte st.shared (left to itself, the
// compiler splits some of these stores, and a split 16-byte store costs
// more bank-conflict wavefronts than one 16-byte store)
template <class R, int N>
__device__ __forceinline__ void st_smem_vec(R *p, const R (&o)[N]) {
    if constexpr (sizeof(R) == 4 && N == 4) {
        const unsigned a = (unsigned)__cvta_generic_to_shared(p);
        asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(o[0]), "f"(o[1]),
                     "f"(o[2]), "f"(o[3])
                     : "memory");
    } else {
        st_vec<R, N>(p, o);
    }
}

// load a D x D matrix stored with rows padded to Pad<D>
template <class R, int D>
__device__ __forceinline__ void ldg_mat(R (&M)[D][D], const R *p) {
    if constexpr (D == 2) {
        R t[4];
        ldg_vec<R, 4>(t, p);
        M[0][0] = t[0]; M[0][1] = t[1]; M[1][0] = t[2]; M[1][1] = t[3];
    } else {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            R t[4];
            ldg_vec<R, 4>(t, p + 4 * r);
            M[r][0] = t[0]; M[r][1] = t[1]; M[r][2] = t[2];
        }
    }
}

template <class R, int D>
__device__ __forceinline__ void st_mat(R *p, const R (&M)[D][D]) {
    if constexpr (D == 2) {
        R t[4] = {M[0][0], M[0][1], M[1][0], M[1][1]};
        st_vec<R, 4>(p, t);
    } else {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            R t[4] = {M[r][0], M[r][1], M[r][2], R(0)};
            st_vec<R, 4>(p + 4 * r, t);
        }
    }
}

// ------------------------------------------------------------------ async copies
// cp.async global -> shared (non-blocking; completion by cp_async_wait_all)
__device__ __forceinline__ void cp_async(void *smem, const void *gmem, int bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if (bytes == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
    else if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
// copy N reals (N * sizeof(R) a multiple of 8, both ends aligned to min(16, N*sizeof(R)))
template <class R, int N>
__device__ __forceinline__ void cp_async_reals(R *smem, const R *gmem) {
    constexpr int B = N * (int)sizeof(R);
    if constexpr (B <= 16) {
        cp_async(smem, gmem, B);
    } else {
#pragma unroll
        for (int o = 0; o < B / 16; ++o)
            cp_async(reinterpret_cast<char *>(smem) + 16 * o, reinterpret_cast<const char *>(gmem) + 16 * o, 16);
    }
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// close this thread's current group of copies
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N of this thread's committed groups are still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// bulk prefetch of [g, g + bytes) into L2 (no completion to wait for; g and
// bytes multiples of 16)
// L2 prefetch of the line holding p (a hint: L2 is coherent, so it may be
// issued before the data's producer has finished)
__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
__device__ __forceinline__ void prefetch_l2_bulk(const void *g, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(__cvta_generic_to_global(g)),
                 "r"(bytes)
                 : "memory");
}

// ------------------------------------------------------------------ math
__device__ __forceinline__ float fma_r(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_r(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float dsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double dsqrt(double x) { return sqrt(x); }
// square root for the neighbour loops: the hardware approximation in FP32
// (mixed precision), IEEE in FP64; exact 0 for the zero-distance padding
__device__ __forceinline__ float nsqrt(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double nsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float dexp(float x) { return expf(x); }
__device__ __forceinline__ double dexp(double x) { return exp(x); }
__device__ __forceinline__ float drcbrt(float x) { return rcbrtf(x); }
__device__ __forceinline__ double drcbrt(double x) { return rcbrt(x); }
__device__ __forceinline__ float dabs(float x) { return fabsf(x); }
__device__ __forceinline__ double dabs(double x) { return fabs(x); }

template <class R>
__device__ __forceinline__ void m3_mul(const R (&A)[3][3], const R (&B)[3][3], R (&C)[3][3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) C[i][j] = A[i][0] * B[0][j] + A[i][1] * B[1][j] + A[i][2] * B[2][j];
}

// C = A B^T
template <class R>
__device__ __forceinline__ void m3_mul_bt(const R (&A)[3][3], const R (&B)[3][3], R (&C)[3][3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) C[i][j] = A[i][0] * B[j][0] + A[i][1] * B[j][1] + A[i][2] * B[j][2];
}

template <class R>
__device__ __forceinline__ R m3_det(const R (&A)[3][3]) {
    return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
           A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
           A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

// cofactor matrix: cof(A) = det(A) A^-T
template <class R>
__device__ __forceinline__ void m3_cof(const R (&A)[3][3], R (&C)[3][3]) {
    C[0][0] = A[1][1] * A[2][2] - A[1][2] * A[2][1];
    C[0][1] = A[1][2] * A[2][0] - A[1][0] * A[2][2];
    C[0][2] = A[1][0] * A[2][1] - A[1][1] * A[2][0];
    C[1][0] = A[0][2] * A[2][1] - A[0][1] * A[2][2];
    C[1][1] = A[0][0] * A[2][2] - A[0][2] * A[2][0];
    C[1][2] = A[0][1] * A[2][0] - A[0][0] * A[2][1];
    C[2][0] = A[0][1] * A[1][2] - A[0][2] * A[1][1];
    C[2][1] = A[0][2] * A[1][0] - A[0][0] * A[1][2];
    C[2][2] = A[0][0] * A[1][1] - A[0][1] * A[1][0];
}

// ------------------------------------------------------------------ laws
struct MatConst;

// St Venant-Kirchhoff (elastic reading of App. B.2): S = lambda tr(E) I + 2 mu E,
// E = (F^T F - I)/2, P = F S.
template <class R>
__device__ __forceinline__ void stress_svk(const R (&F)[3][3], R lambda, R mu, R (&P)[3][3]) {
    R E[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            E[i][j] = R(0.5) * (F[0][i] * F[0][j] + F[1][i] * F[1][j] + F[2][i] * F[2][j]);
    E[0][0] -= R(0.5); E[1][1] -= R(0.5); E[2][2] -= R(0.5);
    R tr = E[0][0] + E[1][1] + E[2][2];
    R S[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) S[i][j] = R(2) * mu * E[i][j];
    S[0][0] += lambda * tr; S[1][1] += lambda * tr; S[2][2] += lambda * tr;
    m3_mul(F, S, P);
}

// Newton tolerance of the return mapping for a real type (FP64 / FP32)
template <class R> struct NewtonTol { static constexpr double value = sizeof(R) == 8 ? 1e-13 : 1e-6; };

template <class R>
__device__ __forceinline__ R hard_k(R al, R s0, R sinf, R delta, R H) {
    return s0 + (sinf - s0) * (R(1) - dexp(-delta * al)) + H * al;
}
template <class R>
__device__ __forceinline__ R hard_dk(R al, R s0, R sinf, R delta, R H) {
    return (sinf - s0) * delta * dexp(-delta * al) + H;
}

// Alg. 1 (App. A.4): J2 return mapping with saturation hardening.  cp holds
// C_p^-1 as (xx,yy,zz,xy,yz,xz) and alpha; updated in place when plastic.
template <class R>
__device__ __forceinline__ void stress_j2(const R (&F)[3][3], R (&cp)[7], R K, R mu, R s0,
                                          R sinf, R delta, R H, R (&P)[3][3]) {
    const R r23 = R(0.816496580927726);  // sqrt(2/3)
    R J = m3_det(F);
    R sc = drcbrt(J);
    R Fb[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Fb[i][j] = sc * F[i][j];
    R Cp[3][3] = {{cp[0], cp[3], cp[5]}, {cp[3], cp[1], cp[4]}, {cp[5], cp[4], cp[2]}};
    R T[3][3], bpre[3][3];
    m3_mul(Fb, Cp, T);
    m3_mul_bt(T, Fb, bpre);
    R trb = bpre[0][0] + bpre[1][1] + bpre[2][2];
    R s[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) s[i][j] = mu * bpre[i][j];
    R m3 = mu * trb / R(3);
    s[0][0] -= m3; s[1][1] -= m3; s[2][2] -= m3;
    R sn = R(0);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) sn += s[i][j] * s[i][j];
    sn = dsqrt(sn);
    R al = cp[6];
    R kal = hard_k(al, s0, sinf, delta, H);
    R f = sn - r23 * kal;
    if (f > R(0)) {
        R mubar = mu * trb / R(3);
        R dg = R(0);
        const R tol = R(NewtonTol<R>::value);
        for (int it = 0; it < 30; ++it) {
            R g = sn - r23 * hard_k(al + r23 * dg, s0, sinf, delta, H) - R(2) * mubar * dg;
            if (dabs(g) <= tol * r23 * kal) break;
            R dgd = -(R(2) / R(3)) * hard_dk(al + r23 * dg, s0, sinf, delta, H) - R(2) * mubar;
            dg -= g / dgd;
        }
        R fac = R(1) - R(2) * mubar * dg / sn;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) s[i][j] *= fac;
        cp[6] = al + r23 * dg;
        // b_e = s/mu + tr(b_pre)/3 I;  C_p^-1 = Fb^-1 b_e Fb^-T  (det Fb = 1)
        R be[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) be[i][j] = s[i][j] / mu;
        be[0][0] += trb / R(3); be[1][1] += trb / R(3); be[2][2] += trb / R(3);
        R Ci[3][3], Fi[3][3];
        m3_cof(Fb, Ci);                 // cof(Fb) = det(Fb) Fb^-T
        R idet = R(1) / m3_det(Fb);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) Fi[i][j] = Ci[j][i] * idet;   // Fb^-1
        R T2[3][3], Cn[3][3];
        m3_mul(Fi, be, T2);
        m3_mul_bt(T2, Fi, Cn);
        cp[0] = Cn[0][0]; cp[1] = Cn[1][1]; cp[2] = Cn[2][2];
        cp[3] = R(0.5) * (Cn[0][1] + Cn[1][0]);
        cp[4] = R(0.5) * (Cn[1][2] + Cn[2][1]);
        cp[5] = R(0.5) * (Cn[0][2] + Cn[2][0]);
    }
    // tau = K/2 (J^2 - 1) I + s;  P = tau F^-T = tau cof(F) / J
    R pv = R(0.5) * K * (J * J - R(1));
    s[0][0] += pv; s[1][1] += pv; s[2][2] += pv;
    R Cf[3][3];
    m3_cof(F, Cf);
    R iJ = R(1) / J;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            P[i][j] = (s[i][0] * Cf[0][j] + s[i][1] * Cf[1][j] + s[i][2] * Cf[2][j]) * iJ;
}

// swelling (App. B.2): P -= p J F^-T = p cof(F)
template <class R>
__device__ __forceinline__ void add_swelling(const R (&F)[3][3], R p, R (&P)[3][3]) {
    R Cf[3][3];
    m3_cof(F, Cf);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) P[i][j] -= p * Cf[i][j];
}

// ------------------------------------------------------------------ reductions
template <class T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}
template <class T>
__device__ __forceinline__ T warp_max(T x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

}  // namespace mts
