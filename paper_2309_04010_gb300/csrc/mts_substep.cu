// mts_substep.cu -- the substep hot path and the slow-step kernels.
//
// One substep (Sec. 4.2 inner loop) is, in launch order:
//   k_stress  F_a = I + (sum_b V (u_b - u_a) (x) grad W_ab) B0_a (Sec. 2.1, 3.1),
//             stress (SVK, or Alg. 1 return mapping), swelling, store P B0;
//   k_force   dv_a/dt = (1/rho0) sum_b V (PB_a + PB_b) grad_a W_ab (Sec. 3.1),
//             kick of the free axes, block partials of max|a| and of the
//             reported end force;
//   k_damp    pairwise implicit viscous damping (Sec. 4.3), symmetric sweep:
//             colours 0..C-1 forward with dt/2, then C-1..0 in reverse with
//             dt/2; one warp per owner block, velocities of the 2^d touched
//             blocks staged in shared memory, one level (sub-colour) per step;
//   k_drift   BC (fixed axes v = 0, u = ramp u_unit) and drift u += dt v in
//             FP64; FP64 block partials of E_k and |v|max; the last block to
//             finish reduces all partials in a fixed order, applies the
//             kinetic-energy stop (Sec. 4.2) and sets the next dt (Sec. 4.1).
// Every kernel returns at once when the device stop flag is set, so a captured
// chunk of substeps can run past convergence without changing the state.
#include <algorithm>
#include <cmath>

#include "mts_device.cuh"
#include "mts_internal.cuh"

namespace mts {

namespace {

inline unsigned grid_of(long long n) { return (unsigned)((n + kBlock - 1) / kBlock); }

// --------------------------------------------------------------------- F
// F_a = I + (sum_b V (u_b - u_a) (x) grad_a W_ab) B0_a, 3x3 with F_zz = 1 in 2D.
template <class R, int D>
__device__ __forceinline__ void compute_F(const Args<R> &A, long long i, R (&F)[3][3]) {
    constexpr int P = Pad<D>::v;
    R xa[P], ua[P];
    ldg_vec<R, P>(xa, A.X + i * P);
    ldg_vec<R, P>(ua, A.uf + i * P);
    R G[D][D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) G[r][c] = R(0);
    const long long s = i >> 5;
    const int32_t *row = A.ell + A.slice_off[s] + (i & 31);
    const int w = A.slice_w[s];
    for (int j = 0; j < w; ++j) {
        const int b = __ldg(row + 32 * j);
        R xb[P], ub[P];
        ldg_vec<R, P>(xb, A.X + (long long)b * P);
        ldg_vec<R, P>(ub, A.uf + (long long)b * P);
        R d[D], r2 = R(0);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            d[k] = xa[k] - xb[k];
            r2 += d[k] * d[k];
        }
        const R t = R(1) - R(0.5) * dsqrt(r2) * A.inv_h;
        const R f = A.kcoef * t * t * t;   // V W'(r)/r
#pragma unroll
        for (int r = 0; r < D; ++r) {
            const R du = (ub[r] - ua[r]) * f;
#pragma unroll
            for (int c = 0; c < D; ++c) G[r][c] += du * d[c];
        }
    }
    R B[D][D];
    ldg_mat<R, D>(B, A.B0 + i * MatS<D>::v);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) F[r][c] = r == c ? R(1) : R(0);
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) {
            R acc = R(0);
#pragma unroll
            for (int k = 0; k < D; ++k) acc += G[r][k] * B[k][c];
            F[r][c] += acc;
        }
}

// --------------------------------------------------------------------- K_A
template <class R, int D, int MAT>
__global__ void __launch_bounds__(kBlock) k_stress(Args<R> A) {
    if (A.ctrl->done) return;
    const long long i = blockIdx.x * (long long)kBlock + threadIdx.x;
    if (i >= A.n) return;
    R F[3][3];
    compute_F<R, D>(A, i, F);
    R P[3][3];
    if constexpr (MAT == MTS_ELASTIC_SVK) {
        stress_svk<R>(F, A.lambda, A.mu, P);
    } else {
        R cp[8];
        ld_vec<R, 4>(*reinterpret_cast<R(*)[4]>(cp), A.cp + i * 8);
        ld_vec<R, 4>(*reinterpret_cast<R(*)[4]>(cp + 4), A.cp + i * 8 + 4);
        R c7[7] = {cp[0], cp[1], cp[2], cp[3], cp[4], cp[5], cp[6]};
        stress_j2<R>(F, c7, A.K, A.mu, A.s0, A.sinf, A.delta, A.Hlin, P);
        if (c7[6] != cp[6]) {
            R o0[4] = {c7[0], c7[1], c7[2], c7[3]};
            R o1[4] = {c7[4], c7[5], c7[6], R(0)};
            st_vec<R, 4>(A.cp + i * 8, o0);
            st_vec<R, 4>(A.cp + i * 8 + 4, o1);
        }
    }
    if (A.swelling) add_swelling<R>(F, A.swell * (A.c[i] - A.c0), P);
    R B[D][D];
    ldg_mat<R, D>(B, A.B0 + i * MatS<D>::v);
    R PB[D][D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) {
            R acc = R(0);
#pragma unroll
            for (int k = 0; k < D; ++k) acc += P[r][k] * B[k][c];
            PB[r][c] = acc;
        }
    st_mat<R, D>(A.PB + i * MatS<D>::v, PB);
}

// --------------------------------------------------------------------- K_B
template <class R, int D>
__global__ void __launch_bounds__(kBlock) k_force(Args<R> A) {
    if (A.ctrl->done) return;
    constexpr int P = Pad<D>::v;
    const long long i = blockIdx.x * (long long)kBlock + threadIdx.x;
    double amax = 0.0, fm[3] = {0.0, 0.0, 0.0};
    if (i < A.n) {
        R xa[P];
        ldg_vec<R, P>(xa, A.X + i * P);
        R Pa[D][D];
        ldg_mat<R, D>(Pa, A.PB + i * MatS<D>::v);
        R acc[D];
#pragma unroll
        for (int k = 0; k < D; ++k) acc[k] = R(0);
        const long long s = i >> 5;
        const int32_t *row = A.ell + A.slice_off[s] + (i & 31);
        const int w = A.slice_w[s];
        for (int j = 0; j < w; ++j) {
            const int b = __ldg(row + 32 * j);
            R xb[P];
            ldg_vec<R, P>(xb, A.X + (long long)b * P);
            R Pb[D][D];
            ldg_mat<R, D>(Pb, A.PB + (long long)b * MatS<D>::v);
            R d[D], r2 = R(0);
#pragma unroll
            for (int k = 0; k < D; ++k) {
                d[k] = xa[k] - xb[k];
                r2 += d[k] * d[k];
            }
            const R t = R(1) - R(0.5) * dsqrt(r2) * A.inv_h;
            const R f = A.kcoef * t * t * t;
#pragma unroll
            for (int r = 0; r < D; ++r) {
                R sr = R(0);
#pragma unroll
                for (int c = 0; c < D; ++c) sr += (Pa[r][c] + Pb[r][c]) * d[c];
                acc[r] += sr * f;
            }
        }
        const uint8_t fx = A.flags[i];
        const R dt = (R)A.ctrl->dt;
        R v[P];
        ld_vec<R, P>(v, A.v + i * P);
        R ao[P];
        double a2 = 0.0;
#pragma unroll
        for (int k = 0; k < P; ++k) ao[k] = R(0);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            ao[k] = acc[k] * A.inv_rho0;
            if (!((fx >> k) & 1)) {
                v[k] += dt * ao[k];
                a2 += (double)ao[k] * (double)ao[k];
            }
            if (fx & kForceBit) fm[k] = A.mass * (double)ao[k];
        }
        st_vec<R, P>(A.v + i * P, v);
        st_vec<R, P>(A.acc + i * P, ao);
        amax = sqrt(a2);
    }
    // block partials (fixed tree order: deterministic)
    __shared__ double sh[4][kBlock / 32];
    amax = warp_max(amax);
    double f0 = warp_sum(fm[0]), f1 = warp_sum(fm[1]), f2 = warp_sum(fm[2]);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sh[0][wid] = amax; sh[1][wid] = f0; sh[2][wid] = f1; sh[3][wid] = f2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0, s0 = 0, s1 = 0, s2 = 0;
        for (int q = 0; q < kBlock / 32; ++q) {
            m = fmax(m, sh[0][q]); s0 += sh[1][q]; s1 += sh[2][q]; s2 += sh[3][q];
        }
        double *o = A.part_force + blockIdx.x * 4;
        o[0] = m; o[1] = s0; o[2] = s1; o[3] = s2;
    }
}

// --------------------------------------------------------------------- K_C
template <class R, int D>
__device__ __forceinline__ void damp_pair(const Args<R> &A, long long p, R *sv, const uint8_t *sf,
                                          R hdt, R im) {
    constexpr int P = Pad<D>::v;
    const uint32_t ab = __ldg(A.pair_ab + p);
    const int la = (int)(ab & 0xffffu), lb = (int)(ab >> 16);
    const R c = A.eta * __ldg(A.pair_g + p) * hdt;
    const uint8_t fa = sf[la], fb = sf[lb];
    R *va = sv + la * P, *vb = sv + lb * P;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const R ia = ((fa >> k) & 1) ? R(0) : im;
        const R ib = ((fb >> k) & 1) ? R(0) : im;
        const R wn = (va[k] - vb[k]) / (R(1) + c * (ia + ib));
        va[k] -= c * wn * ia;
        vb[k] += c * wn * ib;
    }
}

template <class R, int D>
__global__ void __launch_bounds__(kDampWarps * 32) k_damp(Args<R> A, long long g_begin,
                                                         long long g_end, int mode) {
    if (A.ctrl->done) return;
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int P = Pad<D>::v;
    constexpr int NB = 1 << D;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long g = g_begin + (long long)blockIdx.x * kDampWarps + warp;
    if (g >= g_end) return;
    const int mb = A.mb;
    R *sv = reinterpret_cast<R *>(smem) + (size_t)warp * NB * mb * P;
    uint8_t *sf = reinterpret_cast<uint8_t *>(reinterpret_cast<R *>(smem) +
                                              (size_t)kDampWarps * NB * mb * P) +
                  (size_t)warp * NB * mb;
    int ts[NB], tc[NB];
#pragma unroll
    for (int e = 0; e < NB; ++e) {
        ts[e] = __ldg(A.touch_start + g * NB + e);
        tc[e] = __ldg(A.touch_cnt + g * NB + e);
    }
#pragma unroll
    for (int e = 0; e < NB; ++e)
        for (int t = lane; t < tc[e]; t += 32) {
            R vv[P];
            ld_vec<R, P>(vv, A.v + (long long)(ts[e] + t) * P);
            st_vec<R, P>(sv + (e * mb + t) * P, vv);
            sf[e * mb + t] = A.flags[ts[e] + t];
        }
    __syncwarp();
    const R hdt = (R)(0.5 * A.ctrl->dt);
    const R im = (R)(1.0 / A.mass);
    const int l0 = __ldg(A.grp_lvl + g), l1 = __ldg(A.grp_lvl + g + 1);
    if (mode & 1) {
        for (int l = l0; l < l1; ++l) {
            const long long p1 = __ldg(A.lvl_pair + l + 1);
            for (long long p = __ldg(A.lvl_pair + l) + lane; p < p1; p += 32)
                damp_pair<R, D>(A, p, sv, sf, hdt, im);
            __syncwarp();
        }
    }
    if (mode & 2) {
        for (int l = l1 - 1; l >= l0; --l) {
            const long long p1 = __ldg(A.lvl_pair + l + 1);
            for (long long p = __ldg(A.lvl_pair + l) + lane; p < p1; p += 32)
                damp_pair<R, D>(A, p, sv, sf, hdt, im);
            __syncwarp();
        }
    }
#pragma unroll
    for (int e = 0; e < NB; ++e)
        for (int t = lane; t < tc[e]; t += 32) {
            R vv[P];
            ld_vec<R, P>(vv, sv + (e * mb + t) * P);
            st_vec<R, P>(A.v + (long long)(ts[e] + t) * P, vv);
        }
}

// --------------------------------------------------------------------- drift
template <class R, int D>
__global__ void __launch_bounds__(kBlock) k_drift(Args<R> A) {
    Control *C = A.ctrl;
    if (C->done) return;
    constexpr int P = Pad<D>::v;
    const long long i = blockIdx.x * (long long)kBlock + threadIdx.x;
    double ke = 0.0, vmax = 0.0;
    if (i < A.n) {
        const double dt = C->dt, ramp = C->ramp;
        const uint8_t fx = A.flags[i];
        R v[P];
        ld_vec<R, P>(v, A.v + i * P);
        double u[P];
        ld_vec<double, P>(u, A.u + i * P);
        double v2 = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            if ((fx >> k) & 1) {
                v[k] = R(0);
                u[k] = ramp * A.u_unit[i * P + k];
            } else {
                u[k] += dt * (double)v[k];
            }
            v2 += (double)v[k] * (double)v[k];
        }
        st_vec<R, P>(A.v + i * P, v);
        st_vec<double, P>(A.u + i * P, u);
        if constexpr (sizeof(R) == 4) {
            R uf[P];
#pragma unroll
            for (int k = 0; k < P; ++k) uf[k] = (R)u[k];
            st_vec<R, P>(A.uf + i * P, uf);
        }
        ke = 0.5 * A.mass * v2;
        vmax = sqrt(v2);
    }
    __shared__ double sh[2][kBlock / 32];
    __shared__ int is_last;
    ke = warp_sum(ke);
    vmax = warp_max(vmax);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sh[0][wid] = ke;
        sh[1][wid] = vmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0, m = 0;
        for (int q = 0; q < kBlock / 32; ++q) {
            s += sh[0][q];
            m = fmax(m, sh[1][q]);
        }
        A.part_drift[blockIdx.x * 2] = s;
        A.part_drift[blockIdx.x * 2 + 1] = m;
        __threadfence();
        is_last = atomicAdd(&C->counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    // last block: fixed-order reduction of every block's partials
    double s_ke = 0, s_v = 0, s_a = 0, s_f[3] = {0, 0, 0};
    for (unsigned q = threadIdx.x; q < gridDim.x; q += kBlock) {
        s_ke += __ldcg(A.part_drift + q * 2);
        s_v = fmax(s_v, __ldcg(A.part_drift + q * 2 + 1));
        s_a = fmax(s_a, __ldcg(A.part_force + q * 4));
        for (int k = 0; k < 3; ++k) s_f[k] += __ldcg(A.part_force + q * 4 + 1 + k);
    }
    __shared__ double red[6][kBlock];
    red[0][threadIdx.x] = s_ke; red[1][threadIdx.x] = s_v; red[2][threadIdx.x] = s_a;
    red[3][threadIdx.x] = s_f[0]; red[4][threadIdx.x] = s_f[1]; red[5][threadIdx.x] = s_f[2];
    __syncthreads();
    for (int w = kBlock / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            red[0][threadIdx.x] += red[0][threadIdx.x + w];
            red[1][threadIdx.x] = fmax(red[1][threadIdx.x], red[1][threadIdx.x + w]);
            red[2][threadIdx.x] = fmax(red[2][threadIdx.x], red[2][threadIdx.x + w]);
            for (int k = 3; k < 6; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double KE = red[0][0], VM = red[1][0], AM = red[2][0];
        C->ke = KE;
        C->vmax = VM;
        C->amax = AM;
        for (int k = 0; k < 3; ++k) C->end_force[k] = -red[3 + k][0];
        C->dt_last = C->dt;
        C->nsub += 1;
        if (!isfinite(KE)) {
            C->status = MTS_ERR_NONFINITE;
            C->done = 1;
        } else {
            const double crit = C->ke_mode == 1 ? KE / C->volume : KE;
            if (C->use_tol && crit <= C->ke_thr) {
                C->done = 1;
                C->converged = 1;
            } else if (C->nsub >= C->max_sub) {
                C->done = 1;
            }
        }
        if (C->dt_fixed > 0.0) {
            C->dt = C->dt_fixed;
        } else {
            // Sec. 4.1: dt_s = 0.6 min(h/(c_s + |v|max), sqrt(h/|dv/dt|max))
            const double t1 = A.h / (A.cs + VM);
            const double t2 = sqrt(A.h / AM);
            C->dt = 0.6 * fmin(t1, t2);
        }
        C->counter = 0;
    }
}

// --------------------------------------------------------------------- slow step
__global__ void k_reset_ctrl(Control *C, double dt, double dt_fixed, double ramp,
                             long long max_sub, double ke_thr, int ke_mode, int use_tol,
                             double volume) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    C->dt = dt; C->dt_fixed = dt_fixed; C->ramp = ramp;
    C->max_sub = max_sub; C->ke_thr = ke_thr; C->ke_mode = ke_mode; C->use_tol = use_tol;
    C->volume = volume;
    C->nsub = 0; C->done = 0; C->converged = 0; C->status = 0; C->counter = 0;
    C->ke = 0; C->vmax = 0; C->amax = 0; C->dt_last = 0;
    C->end_force[0] = C->end_force[1] = C->end_force[2] = 0;
}

// load increment (Sec. 4.1 dt_l): prescribed axes jump to ramp * u_unit, v = 0
template <class R, int D>
__global__ void k_load(Args<R> A) {
    constexpr int P = Pad<D>::v;
    const long long i = blockIdx.x * (long long)kBlock + threadIdx.x;
    if (i >= A.n) return;
    const uint8_t fx = A.flags[i];
    if (!(fx & kFixMask)) return;
    const double ramp = A.ctrl->ramp;
    for (int k = 0; k < D; ++k)
        if ((fx >> k) & 1) {
            A.u[i * P + k] = ramp * A.u_unit[i * P + k];
            A.v[i * P + k] = R(0);
            if constexpr (sizeof(R) == 4) A.uf[i * P + k] = (R)A.u[i * P + k];
        }
}

// explicit diffusion (Sec. 2.2 Fick's law as a scalar; Jacobi update)
template <class R, int D>
__global__ void __launch_bounds__(kBlock) k_diffuse(Args<R> A, R dt) {
    constexpr int P = Pad<D>::v;
    const long long i = blockIdx.x * (long long)kBlock + threadIdx.x;
    if (i >= A.n) return;
    if (A.flags[i] & kCHeldBit) {
        A.c_tmp[i] = A.c_held[i];
        return;
    }
    R xa[P];
    ldg_vec<R, P>(xa, A.X + i * P);
    const R ca = A.c[i];
    R s = R(0);
    const long long sl = i >> 5;
    const int32_t *row = A.ell + A.slice_off[sl] + (i & 31);
    const int w = A.slice_w[sl];
    for (int j = 0; j < w; ++j) {
        const int b = __ldg(row + 32 * j);
        R xb[P];
        ldg_vec<R, P>(xb, A.X + (long long)b * P);
        R r2 = R(0);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const R d = xa[k] - xb[k];
            r2 += d * d;
        }
        const R t = R(1) - R(0.5) * dsqrt(r2) * A.inv_h;
        s += (ca - A.c[b]) * t * t * t;
    }
    A.c_tmp[i] = ca + dt * A.dcoef * s;
}

template <class R>
__global__ void k_copy(const R *src, R *dst, long long n) {
    const long long i = blockIdx.x * (long long)kBlock + threadIdx.x;
    if (i < n) dst[i] = src[i];
}

// stable diffusion bound: max_i sum_j 2 D V |W'_ij| / r_ij (FP64, CSR)
template <int D>
__global__ void k_diff_bound(const double *X64, const long long *off, const int32_t *idx,
                             long long n, double h, double kabs, double *part) {
    constexpr int P = Pad<D>::v;
    const long long i = blockIdx.x * (long long)kBlock + threadIdx.x;
    double s = 0.0;
    if (i < n) {
        for (long long p = off[i]; p < off[i + 1]; ++p) {
            const double *xa = X64 + i * P, *xb = X64 + (long long)idx[p] * P;
            double r2 = 0;
            for (int k = 0; k < D; ++k) {
                const double d = xa[k] - xb[k];
                r2 += d * d;
            }
            const double q = sqrt(r2) / h, t = 1.0 - 0.5 * q;
            s += kabs * t * t * t;
        }
    }
    s = warp_max(s);
    __shared__ double sh[kBlock / 32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0;
        for (int q = 0; q < kBlock / 32; ++q) m = fmax(m, sh[q]);
        part[blockIdx.x] = m;
    }
}

// --------------------------------------------------------------------- reads
template <class R, int D>
__global__ void k_defgrad(Args<R> A, double *out) {
    const long long i = blockIdx.x * (long long)kBlock + threadIdx.x;
    if (i >= A.n) return;
    R F[3][3];
    compute_F<R, D>(A, i, F);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) out[i * 9 + r * 3 + c] = (double)F[r][c];
}

// sorted field -> scratch in original order (doubles)
template <class R, int D>
__global__ void k_field_out(Args<R> A, int field, const long long *perm, const double *X64,
                            double *out) {
    constexpr int P = Pad<D>::v;
    const long long s = blockIdx.x * (long long)kBlock + threadIdx.x;
    if (s >= A.n) return;
    const long long i = perm[s];
    switch (field) {
    case MTS_F_U: for (int k = 0; k < D; ++k) out[i * D + k] = A.u[s * P + k]; break;
    case MTS_F_X: for (int k = 0; k < D; ++k) out[i * D + k] = X64[s * P + k]; break;
    case MTS_F_V: for (int k = 0; k < D; ++k) out[i * D + k] = (double)A.v[s * P + k]; break;
    case MTS_F_ACC: for (int k = 0; k < D; ++k) out[i * D + k] = (double)A.acc[s * P + k]; break;
    case MTS_F_PB:
        for (int r = 0; r < D; ++r)
            for (int c = 0; c < D; ++c)
                out[i * D * D + r * D + c] = (double)A.PB[s * MatS<D>::v + r * P + c];
        break;
    case MTS_F_C: out[i] = (double)A.c[s]; break;
    case MTS_F_ALPHA: out[i] = (double)A.cp[s * 8 + 6]; break;
    case MTS_F_CPINV: for (int k = 0; k < 6; ++k) out[i * 6 + k] = (double)A.cp[s * 8 + k]; break;
    default: break;
    }
}

template <class R, int D>
__global__ void k_field_in(Args<R> A, int field, const long long *perm, const double *in) {
    constexpr int P = Pad<D>::v;
    const long long s = blockIdx.x * (long long)kBlock + threadIdx.x;
    if (s >= A.n) return;
    const long long i = perm[s];
    switch (field) {
    case MTS_F_U:
        for (int k = 0; k < D; ++k) {
            A.u[s * P + k] = in[i * D + k];
            if constexpr (sizeof(R) == 4) A.uf[s * P + k] = (R)in[i * D + k];
        }
        break;
    case MTS_F_V: for (int k = 0; k < D; ++k) A.v[s * P + k] = (R)in[i * D + k]; break;
    case MTS_F_C: A.c[s] = (R)in[i]; break;
    case MTS_F_ALPHA: A.cp[s * 8 + 6] = (R)in[i]; break;
    case MTS_F_CPINV: for (int k = 0; k < 6; ++k) A.cp[s * 8 + k] = (R)in[i * 6 + k]; break;
    default: break;
    }
}

// defgrad in sorted order -> original order
__global__ void k_perm_rows(const double *in, const long long *perm, long long n, int w,
                            double *out) {
    const long long s = blockIdx.x * (long long)kBlock + threadIdx.x;
    if (s >= n) return;
    const long long i = perm[s];
    for (int k = 0; k < w; ++k) out[i * w + k] = in[s * w + k];
}

// tip deflection: block partial sums of u over the tip set (and count)
template <int D>
__global__ void k_tip(const double *u, const uint8_t *flags, long long n, double *part) {
    constexpr int P = Pad<D>::v;
    const long long i = blockIdx.x * (long long)kBlock + threadIdx.x;
    double s[4] = {0, 0, 0, 0};
    if (i < n && (flags[i] & kTipBit)) {
        for (int k = 0; k < D; ++k) s[k] = u[i * P + k];
        s[3] = 1.0;
    }
    __shared__ double sh[4][kBlock / 32];
    for (int k = 0; k < 4; ++k) {
        double t = warp_sum(s[k]);
        if ((threadIdx.x & 31) == 0) sh[k][threadIdx.x >> 5] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) {
            double t = 0;
            for (int q = 0; q < kBlock / 32; ++q) t += sh[k][q];
            part[blockIdx.x * 4 + k] = t;
        }
}

__global__ void k_tip_final(const double *part, int nblk, double *out) {
    if (threadIdx.x != 0) return;
    double s[4] = {0, 0, 0, 0};
    for (int b = 0; b < nblk; ++b)
        for (int k = 0; k < 4; ++k) s[k] += part[b * 4 + k];
    for (int k = 0; k < 3; ++k) out[k] = s[3] > 0 ? s[k] / s[3] : 0.0;
}

// --------------------------------------------------------------------- args
template <class R>
Args<R> make_args(mts_body *b) {
    Args<R> A{};
    A.n = b->n;
    A.dim = b->dim;
    A.ell = b->ell;
    A.slice_off = b->slice_off;
    A.slice_w = b->slice_w;
    A.X = (const R *)b->X;
    A.B0 = (const R *)b->B0;
    A.u = b->u;
    A.uf = sizeof(R) == 8 ? (R *)b->u : (R *)b->uf;
    A.v = (R *)b->v;
    A.acc = (R *)b->acc;
    A.PB = (R *)b->PB;
    A.cp = (R *)b->cp;
    A.c = (R *)b->c;
    A.c_tmp = (R *)b->c_tmp;
    A.flags = b->flags;
    A.u_unit = b->u_unit;
    A.c_held = (const R *)b->c_held;
    const double alpha = kernel_alpha(b->dim, b->h);
    A.inv_h = (R)(1.0 / b->h);
    A.kcoef = (R)(b->V * (-5.0 * alpha / (b->h * b->h)));
    A.inv_rho0 = (R)(1.0 / b->rho0);
    A.lambda = (R)b->lambda; A.mu = (R)b->mu; A.K = (R)b->K;
    A.s0 = (R)b->s0; A.sinf = (R)b->sinf; A.delta = (R)b->delta; A.Hlin = (R)b->Hlin;
    A.swelling = b->has_diff && b->beta != 0.0;
    A.swell = (R)(3.0 * b->K * b->beta);
    A.c0 = (R)b->c0;
    A.dcoef = (R)(2.0 * b->D * b->V * (-5.0 * alpha / (b->h * b->h)));
    A.mass = b->rho0 * b->V;
    A.h = b->h;
    A.cs = std::sqrt(b->K / b->rho0);
    A.eta = (R)b->eta;
    A.pair_ab = b->pair_ab;
    A.pair_g = (const R *)b->pair_g;
    A.lvl_pair = b->lvl_pair;
    A.grp_lvl = b->grp_lvl;
    A.touch_start = b->touch_start;
    A.touch_cnt = b->touch_cnt;
    A.mb = b->mb;
    A.ctrl = b->ctrl;
    A.part_force = b->part_force;
    A.part_drift = b->part_drift;
    return A;
}

template <class R, int D>
mts_status stress_t(mts_body *b) {
    Args<R> A = make_args<R>(b);
    if (b->model == MTS_NEOHOOKE_J2)
        k_stress<R, D, MTS_NEOHOOKE_J2><<<grid_of(b->n), kBlock, 0, b->ctx->stream>>>(A);
    else
        k_stress<R, D, MTS_ELASTIC_SVK><<<grid_of(b->n), kBlock, 0, b->ctx->stream>>>(A);
    MTS_CUDA(cudaGetLastError());
    return MTS_OK;
}

template <class R, int D>
mts_status force_t(mts_body *b) {
    k_force<R, D><<<grid_of(b->n), kBlock, 0, b->ctx->stream>>>(make_args<R>(b));
    MTS_CUDA(cudaGetLastError());
    return MTS_OK;
}

template <class R, int D>
size_t damp_smem(const mts_body *b) {
    return (size_t)kDampWarps * (1 << D) * b->mb * (Pad<D>::v * sizeof(R) + 1) + 16;
}

template <class R, int D>
mts_status damping_t(mts_body *b, long long *nlaunch) {
    if (nlaunch) *nlaunch = 0;
    if (b->eta == 0.0 || b->npairs == 0) return MTS_OK;
    Args<R> A = make_args<R>(b);
    const size_t smem = damp_smem<R, D>(b);
    const int ncol = 1 << D;
    auto launch = [&](int c, int mode) -> mts_status {
        const long long g0 = b->col_off[c], g1 = b->col_off[c + 1];
        if (g1 <= g0) return MTS_OK;
        const unsigned grid = (unsigned)((g1 - g0 + kDampWarps - 1) / kDampWarps);
        k_damp<R, D><<<grid, kDampWarps * 32, smem, b->ctx->stream>>>(A, g0, g1, mode);
        MTS_CUDA(cudaGetLastError());
        if (nlaunch) ++*nlaunch;
        return MTS_OK;
    };
    // symmetric sweep: forward 0..C-2, fused forward+reverse on C-1, reverse C-2..0
    for (int c = 0; c < ncol - 1; ++c) MTS_TRY(launch(c, 1));
    MTS_TRY(launch(ncol - 1, 3));
    for (int c = ncol - 2; c >= 0; --c) MTS_TRY(launch(c, 2));
    return MTS_OK;
}

// raise the dynamic shared-memory limit of the damping kernel (outside any
// stream capture)
template <class R, int D>
mts_status prepare_t(mts_body *b) {
    const size_t smem = damp_smem<R, D>(b);
    if (smem > 227 * 1024) {
        set_error("damping blocks hold too many particles (%d) for shared memory", b->mb);
        return MTS_ERR_INVALID_ARG;
    }
    MTS_CUDA(cudaFuncSetAttribute(k_damp<R, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)std::max<size_t>(smem, 48 * 1024)));
    return MTS_OK;
}

template <class R, int D>
mts_status drift_t(mts_body *b) {
    k_drift<R, D><<<grid_of(b->n), kBlock, 0, b->ctx->stream>>>(make_args<R>(b));
    MTS_CUDA(cudaGetLastError());
    return MTS_OK;
}

template <class R, int D>
mts_status load_t(mts_body *b) {
    k_load<R, D><<<grid_of(b->n), kBlock, 0, b->ctx->stream>>>(make_args<R>(b));
    MTS_CUDA(cudaGetLastError());
    return MTS_OK;
}

template <class R, int D>
mts_status diffuse_t(mts_body *b, double dt) {
    Args<R> A = make_args<R>(b);
    k_diffuse<R, D><<<grid_of(b->n), kBlock, 0, b->ctx->stream>>>(A, (R)dt);
    k_copy<R><<<grid_of(b->n), kBlock, 0, b->ctx->stream>>>((const R *)b->c_tmp, (R *)b->c, b->n);
    MTS_CUDA(cudaGetLastError());
    return MTS_OK;
}

template <class R, int D>
mts_status defgrad_t(mts_body *b, double *out_sorted) {
    k_defgrad<R, D><<<grid_of(b->n), kBlock, 0, b->ctx->stream>>>(make_args<R>(b), out_sorted);
    MTS_CUDA(cudaGetLastError());
    return MTS_OK;
}

template <class R, int D>
mts_status field_out_t(mts_body *b, int field) {
    if (field == MTS_F_DEFGRAD) {
        double *tmp = b->scratch + (size_t)b->n * 9;
        k_defgrad<R, D><<<grid_of(b->n), kBlock, 0, b->ctx->stream>>>(make_args<R>(b), tmp);
        k_perm_rows<<<grid_of(b->n), kBlock, 0, b->ctx->stream>>>(tmp, b->perm, b->n, 9, b->scratch);
    } else {
        k_field_out<R, D><<<grid_of(b->n), kBlock, 0, b->ctx->stream>>>(make_args<R>(b), field,
                                                                        b->perm, b->X64, b->scratch);
    }
    MTS_CUDA(cudaGetLastError());
    return MTS_OK;
}

template <class R, int D>
mts_status field_in_t(mts_body *b, int field) {
    k_field_in<R, D><<<grid_of(b->n), kBlock, 0, b->ctx->stream>>>(make_args<R>(b), field, b->perm,
                                                                   b->scratch);
    MTS_CUDA(cudaGetLastError());
    return MTS_OK;
}

#define DISPATCH(fn, ...)                                                        \
    (b->precision == MTS_FP64                                                    \
         ? (b->dim == 2 ? fn<double, 2>(__VA_ARGS__) : fn<double, 3>(__VA_ARGS__)) \
         : (b->dim == 2 ? fn<float, 2>(__VA_ARGS__) : fn<float, 3>(__VA_ARGS__)))

}  // namespace

mts_status launch_stress(mts_body *b) { return DISPATCH(stress_t, b); }
mts_status launch_force(mts_body *b) { return DISPATCH(force_t, b); }
mts_status launch_damping(mts_body *b, long long *launches) { return DISPATCH(damping_t, b, launches); }
mts_status launch_drift(mts_body *b) { return DISPATCH(drift_t, b); }
mts_status prepare_kernels(mts_body *b) { return DISPATCH(prepare_t, b); }
mts_status launch_slow_begin(mts_body *b) { return DISPATCH(load_t, b); }
mts_status launch_diffusion(mts_body *b, double dt) { return DISPATCH(diffuse_t, b, dt); }
mts_status launch_defgrad(mts_body *b, double *out_sorted) { return DISPATCH(defgrad_t, b, out_sorted); }
mts_status field_to_scratch(mts_body *b, int field) { return DISPATCH(field_out_t, b, field); }
mts_status scratch_to_field(mts_body *b, int field) { return DISPATCH(field_in_t, b, field); }

mts_status launch_reset_ctrl(mts_body *b, double dt, double dt_fixed, double ramp,
                             long long max_sub, double ke_thr, int ke_mode, int use_tol) {
    k_reset_ctrl<<<1, 32, 0, b->ctx->stream>>>(b->ctrl, dt, dt_fixed, ramp, max_sub, ke_thr, ke_mode,
                                               use_tol, (double)b->n * b->V);
    MTS_CUDA(cudaGetLastError());
    return MTS_OK;
}

mts_status diffusion_bound(mts_body *b, double *amax_sum) {
    const double alpha = kernel_alpha(b->dim, b->h);
    const double kabs = 2.0 * b->D * b->V * 5.0 * alpha / (b->h * b->h);
    const unsigned g = grid_of(b->n);
    double *part = b->scratch;
    if (b->dim == 2)
        k_diff_bound<2><<<g, kBlock, 0, b->ctx->stream>>>(b->X64, b->nb_off, b->nb_idx, b->n, b->h, kabs, part);
    else
        k_diff_bound<3><<<g, kBlock, 0, b->ctx->stream>>>(b->X64, b->nb_off, b->nb_idx, b->n, b->h, kabs, part);
    MTS_CUDA(cudaGetLastError());
    std::vector<double> h(g);
    MTS_CUDA(cudaMemcpyAsync(h.data(), part, g * sizeof(double), cudaMemcpyDeviceToHost, b->ctx->stream));
    MTS_CUDA(cudaStreamSynchronize(b->ctx->stream));
    double m = 0;
    for (double x : h) m = std::max(m, x);
    *amax_sum = m;
    return MTS_OK;
}

mts_status launch_tip(mts_body *b, double *out3) {
    const unsigned g = grid_of(b->n);
    double *part = b->scratch;
    if (b->dim == 2)
        k_tip<2><<<g, kBlock, 0, b->ctx->stream>>>(b->u, b->flags, b->n, part);
    else
        k_tip<3><<<g, kBlock, 0, b->ctx->stream>>>(b->u, b->flags, b->n, part);
    k_tip_final<<<1, 32, 0, b->ctx->stream>>>(part, (int)g, part + (size_t)g * 4);
    MTS_CUDA(cudaGetLastError());
    MTS_CUDA(cudaMemcpyAsync(out3, part + (size_t)g * 4, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                             b->ctx->stream));
    MTS_CUDA(cudaStreamSynchronize(b->ctx->stream));
    return MTS_OK;
}

int field_width(const mts_body *b, int field) {
    switch (field) {
    case MTS_F_U: case MTS_F_X: case MTS_F_V: case MTS_F_ACC: return b->dim;
    case MTS_F_DEFGRAD: return 9;
    case MTS_F_PB: return b->dim * b->dim;
    case MTS_F_C: case MTS_F_ALPHA: return 1;
    case MTS_F_CPINV: return 6;
    default: return -1;
    }
}

}  // namespace mts
