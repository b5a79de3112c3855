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
//             kinetic-energy stop (Sec. 4.2; tested once E_k has passed its
//             peak after the slow step's event) and sets the next dt (Sec. 4.1).
// Every kernel returns at once when the device stop flag is set, so a captured
// chunk of substeps can run past convergence without changing the state.
#include <algorithm>
#include <cstdlib>
#include <vector>
#include <cmath>

#include "mts_device.cuh"
#include "mts_internal.cuh"
#include "mts_tiles.cuh"

namespace mts {

namespace {

inline unsigned grid_of(long long n) { return (unsigned)((n + kBlock - 1) / kBlock); }
// the drift kernel's grid: four particles per thread
inline unsigned drift_grid(long long n) { return (unsigned)((n + 4LL * kBlock - 1) / (4LL * kBlock)); }

// F_a = I + (sum_b V (u_b - u_a) (x) grad_a W_ab) B0_a, 3x3 with F_zz = 1 in 2D;
// X and u of the halo are in shared memory.
template <class R, int D>
__device__ __forceinline__ void compute_F(const Args<R> &A, const R *sX, const R *sU, long long i,
                                          R (&F)[3][3]) {
    constexpr int P = Pad<D>::v;
    const long long t = blockIdx.x;
    const int li = A.lself[i];
    R xa[P], ua[P];
    ld_vec<R, P>(xa, sX + li * P);
    ld_vec<R, P>(ua, sU + li * P);
    R G[D][D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) G[r][c] = R(0);
    const int T = A.T;
    const uint16_t *row = A.lell + A.lell_off[t] + threadIdx.x;
    const int w = A.tile_w[t];
    // per neighbour V W'(r)/r = kcoef (1 - r/(2h))^3: the factor kcoef is
    // applied once to the sum, and 1 - r/(2h) is one fused multiply-add
    const R mhalf_inv_h = R(-0.5) * A.inv_h;   // exact: a power-of-two scaling
    auto accumulate = [&](const R (&xb)[P], const R (&ub)[P]) {
        R d[D], r2 = R(0);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            d[k] = xa[k] - xb[k];
            r2 += d[k] * d[k];
        }
        const R tt = fma_r(nsqrt(r2), mhalf_inv_h, R(1));
        const R f = tt * tt * tt;
#pragma unroll
        for (int r = 0; r < D; ++r) {
            const R du = (ub[r] - ua[r]) * f;
#pragma unroll
            for (int c = 0; c < D; ++c) G[r][c] += du * d[c];
        }
    };
    for_each_neighbour_chunks(row, T, w, [&](int l) {
        R xb[P], ub[P];
        ld_vec<R, P>(xb, sX + l * P);
        ld_vec<R, P>(ub, sU + l * P);
        accumulate(xb, ub);
    });
    {
        const R kcoef = A.kcoef;
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
            for (int c = 0; c < D; ++c) G[r][c] *= kcoef;
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

// Anisotropic kernel: the gathers run on scaled positions X~ = s (.) X, where
// the kernel is isotropic; the real deformation gradient is
// F = I + (F~ - I) diag(s) (the corrected gradient maps back column by column).
template <class R, int D>
__device__ __forceinline__ void unscale_F(const Args<R> &A, R (&F)[3][3]) {
    if (!A.aniso) return;
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) F[r][c] = (r == c ? R(1) : R(0)) + (F[r][c] - (r == c ? R(1) : R(0))) * A.sk[c];
}

// --------------------------------------------------------------------- K_A
template <class R, int D, int MAT>
__global__ void __launch_bounds__(TileThreads<R>::v) k_stress(Args<R> A) {
    chain_trigger();
    {
        // this particle's per-particle inputs, read after the F gather: into
        // L2 while the previous kernel drains
        const long long ip = blockIdx.x * (long long)A.T + threadIdx.x;
        if (ip < A.n) {
            prefetch_l2(A.B0 + ip * MatS<D>::v);
            if (D == 3) prefetch_l2(A.X + ip * Pad<D>::v);
            if (MAT != MTS_ELASTIC_SVK) prefetch_l2(A.cp + ip * 8);
            if (A.swelling) prefetch_l2(A.c + ip);
        }
    }
    constexpr int P = Pad<D>::v;
    extern __shared__ __align__(16) unsigned char smem[];
    R *sX = reinterpret_cast<R *>(smem);
    R *sU = reinterpret_cast<R *>(smem + second_off<R, P>(A.max_halo));
    // the halo's positions (set-up data) before the wait, u after it; the
    // tile's neighbour slots (set-up data) into L2 meanwhile
    if (threadIdx.x == 0 && A.tile_w[blockIdx.x] > 0)
        prefetch_l2_bulk(A.lell + A.lell_off[blockIdx.x], (unsigned)(A.tile_w[blockIdx.x] * A.T * 2));
    const HaloPre<R> hp = stage_halo_pre<R, P>(A, sX);
    chain_wait();
    if (A.ctrl->done) {
        cp_async_wait_all();
        return;
    }
    stage_halo_post<R, P, P>(A, hp, sX, sU, A.uf);
    const long long i = blockIdx.x * (long long)A.T + threadIdx.x;
    if (i >= A.n) return;
    R F[3][3];
    compute_F<R, D>(A, sX, sU, i, F);
    unscale_F<R, D>(A, F);
    R P3[3][3];
    if constexpr (MAT == MTS_ELASTIC_SVK) {
        stress_svk<R>(F, A.lambda, A.mu, P3);
    } else {
        R cp[8];
        ld_vec<R, 4>(*reinterpret_cast<R(*)[4]>(cp), A.cp + i * 8);
        ld_vec<R, 4>(*reinterpret_cast<R(*)[4]>(cp + 4), A.cp + i * 8 + 4);
        R c7[7] = {cp[0], cp[1], cp[2], cp[3], cp[4], cp[5], cp[6]};
        stress_j2<R>(F, c7, A.K, A.mu, A.s0, A.sinf, A.delta, A.Hlin, P3);
        if (c7[6] != cp[6]) {
            R o0[4] = {c7[0], c7[1], c7[2], c7[3]};
            R o1[4] = {c7[4], c7[5], c7[6], R(0)};
            st_vec<R, 4>(A.cp + i * 8, o0);
            st_vec<R, 4>(A.cp + i * 8 + 4, o1);
        }
    }
    if (A.swelling) add_swelling<R>(F, A.swell * (A.c[i] - A.c0), P3);
    R B[D][D];
    ldg_mat<R, D>(B, A.B0 + i * MatS<D>::v);
    // P B0^T (the variational force of F = I + sum (u_b - u_a) (x) B0^T grad W;
    // B0 is symmetric for an isotropic kernel); anisotropic: P diag(s) B0~^T
    R PB[D][D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) {
            R acc = R(0);
#pragma unroll
            for (int k = 0; k < D; ++k) acc += P3[r][k] * (A.aniso ? A.sk[k] : R(1)) * B[c][k];
            PB[r][c] = acc;
        }
    if constexpr (D == 3) {
        // force record: X then P B0 row-major, 12 reals (three 16-byte rows);
        // X relative to the body's corner (one origin for every particle: the
        // force gathers records of particles from many tiles)
        R rec[12];
        ldg_vec<R, 4>(*reinterpret_cast<R(*)[4]>(rec), A.X + i * P);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) rec[3 + 3 * r + c] = PB[r][c];
        st_vec<R, 4>(A.PB + i * 12, *reinterpret_cast<const R(*)[4]>(rec));
        st_vec<R, 4>(A.PB + i * 12 + 4, *reinterpret_cast<const R(*)[4]>(rec + 4));
        st_vec<R, 4>(A.PB + i * 12 + 8, *reinterpret_cast<const R(*)[4]>(rec + 8));
    } else {
        st_mat<R, D>(A.PB + i * MatS<D>::v, PB);
    }
}

// L2 prefetch of the level slots [m0, m1) of one owner group: a damping
// launch prefetches the next launch's groups, so their slots stream from HBM
// while its own chains run instead of at the start of the next launch
template <class R>
__device__ __forceinline__ void prefetch_group_levels(const Args<R> &A, int m0, int m1) {
    if (m1 > m0) {
        prefetch_l2_bulk(A.pair_ab + 32LL * m0, 128u * (unsigned)(m1 - m0));
        prefetch_l2_bulk(A.pair_g + 32LL * m0, 32u * (unsigned)sizeof(R) * (unsigned)(m1 - m0));
    }
}

// --------------------------------------------------------------------- K_B
template <class R, int D>
__global__ void __launch_bounds__(TileThreads<R>::v) k_force(Args<R> A) {
    chain_trigger();
    constexpr int P = Pad<D>::v;
    constexpr int MS = MatS<D>::v;
    extern __shared__ __align__(16) unsigned char smem[];
    // 3D: one 12-real record per halo particle (X, then P B0 row-major);
    // 2D: X and P B0 in two arrays
    R *sX = reinterpret_cast<R *>(smem);
    R *sP = D == 3 ? sX : reinterpret_cast<R *>(smem + second_off<R, P>(A.max_halo));
    // the halo indices (and 2D positions) before the wait, P B0 after it
    // (an L2 prefetch of the tile's neighbour slots, as in the stress kernel,
    // made this kernel slower: 433 -> 439 us on the plate)
    const HaloPre<R> hp = stage_halo_pre<R, P>(A, D == 3 ? nullptr : sX);
    chain_wait();
    if (A.ctrl->done) {
        cp_async_wait_all();
        return;
    }
    stage_halo_post<R, P, MS>(A, hp, D == 3 ? nullptr : sX, sP, A.PB);
    const long long t = blockIdx.x;
    const long long i = t * A.T + threadIdx.x;
    double amax = 0.0, fm[3] = {0.0, 0.0, 0.0};
    if (i < A.n) {
        const int li = A.lself[i];
        R xa[P];
        R Pa[D][D];
        if constexpr (D == 2) {
            ld_vec<R, P>(xa, sX + li * P);
            R q[4];
            ld_vec<R, 4>(q, sP + li * 4);
            Pa[0][0] = q[0]; Pa[0][1] = q[1]; Pa[1][0] = q[2]; Pa[1][1] = q[3];
        } else {
            R q[12];
            ld_vec<R, 4>(*reinterpret_cast<R(*)[4]>(q), sP + li * 12);
            ld_vec<R, 4>(*reinterpret_cast<R(*)[4]>(q + 4), sP + li * 12 + 4);
            ld_vec<R, 4>(*reinterpret_cast<R(*)[4]>(q + 8), sP + li * 12 + 8);
#pragma unroll
            for (int k = 0; k < 3; ++k) xa[k] = q[k];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) Pa[r][c] = q[3 + 3 * r + c];
        }
        // a_a = (PB_a sum_b g_ab + sum_b PB_b g_ab) / rho0, g_ab = V grad_a W_ab
        R acc[D], gs[D];
#pragma unroll
        for (int k = 0; k < D; ++k) acc[k] = gs[k] = R(0);
        const int T = A.T;
        const uint16_t *row = A.lell + A.lell_off[t] + threadIdx.x;
        const int w = A.tile_w[t];
        const R inv_h = A.inv_h, kcoef = A.kcoef;
        auto load_rec = [&](int l, R (&q)[12]) {
            if constexpr (D == 2) {
                ld_vec<R, 2>(*reinterpret_cast<R(*)[2]>(q), sX + l * 2);
                ld_vec<R, 4>(*reinterpret_cast<R(*)[4]>(q + 3), sP + l * 4);
            } else {
                ld_vec<R, 4>(*reinterpret_cast<R(*)[4]>(q), sP + l * 12);
                ld_vec<R, 4>(*reinterpret_cast<R(*)[4]>(q + 4), sP + l * 12 + 4);
                ld_vec<R, 4>(*reinterpret_cast<R(*)[4]>(q + 8), sP + l * 12 + 8);
            }
        };
        auto accumulate = [&](const R (&q)[12]) {
            R d[D], r2 = R(0);
#pragma unroll
            for (int k = 0; k < D; ++k) {
                d[k] = xa[k] - q[k];
                r2 += d[k] * d[k];
            }
            const R tt = R(1) - R(0.5) * nsqrt(r2) * inv_h;
            const R f = kcoef * tt * tt * tt;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                d[k] *= f;
                gs[k] += d[k];
            }
#pragma unroll
            for (int r = 0; r < D; ++r) {
                R sum = R(0);
#pragma unroll
                for (int c = 0; c < D; ++c) sum += q[3 + D * r + c] * d[c];
                acc[r] += sum;
            }
        };
        for_each_neighbour(row, T, w, [&](int l) {
            R q[12];
            load_rec(l, q);
            accumulate(q);
        });
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
            for (int c = 0; c < D; ++c) acc[r] += Pa[r][c] * gs[c];
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
                if constexpr (sizeof(R) == 4) {
                    const double ad = f2d_bits(ao[k]);   // exact widening on the integer pipe
                    a2 += ad * ad;
                } else {
                    a2 += (double)ao[k] * (double)ao[k];
                }
            }
            if (fx & kForceBit) fm[k] = A.mass * (double)ao[k];
        }
        st_vec<R, P>(A.v + i * P, v);
        st_vec<R, P>(A.acc + i * P, ao);
        amax = a2;                       // max |a|^2; the square root is taken once, at the end
    }
    // block partials (fixed tree order: deterministic)
    __shared__ double sh[4][TileThreads<R>::v / 32];
    amax = warp_max(amax);
    // end-force sums only in warps that hold a reported particle
    double f0 = 0.0, f1 = 0.0, f2 = 0.0;
    if (__any_sync(0xffffffffu, fm[0] != 0.0 || fm[1] != 0.0 || fm[2] != 0.0)) {
        f0 = warp_sum(fm[0]);
        f1 = warp_sum(fm[1]);
        f2 = warp_sum(fm[2]);
    }
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sh[0][wid] = amax; sh[1][wid] = f0; sh[2][wid] = f1; sh[3][wid] = f2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0, s0 = 0, s1 = 0, s2 = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            m = fmax(m, sh[0][q]); s0 += sh[1][q]; s1 += sh[2][q]; s2 += sh[3][q];
        }
        double *o = A.part_force + blockIdx.x * 4;
        o[0] = m; o[1] = s0; o[2] = s1; o[3] = s2;
    }
}

// --------------------------------------------------------------------- K_C
// shared-memory layout of one damping warp: the velocities of the 2^d touched
// blocks (+1 dummy slot, padded to a whole group of eight slots, 16-byte
// aligned for cp.async), then the level slots; the pair words carry the
// constrained axes, so no flags are staged
constexpr int kDampChunk = 4;    // levels per chunk of the damping warp's level ring
template <class R, int D>
struct DampSmem {
    __host__ __device__ static size_t vbytes(int mb) {
        return (((size_t)damp_slot_count((1 << D) * mb) * Pad<D>::v * sizeof(R)) + 15) &
               ~size_t(15);
    }
    // + the level slots (word, coefficient) x 32 per level: every level of the
    // group (RING = false) or a ring of two chunks of kDampChunk levels
    __host__ __device__ static size_t bytes(int mb, int maxl, bool ring) {
        const size_t lv = ring ? (size_t)2 * kDampChunk : (size_t)maxl;
        return (vbytes(mb) + lv * 32 * (4 + sizeof(R)) + 15) & ~size_t(15);
    }
};

// One backward-Euler update of the pair ODE m dv_a/dt = -B (v_a - v_b) with
// x = (dt/2) B: w' = w / (1 + x (1/m_a + 1/m_b)), v_a -= x w' / m_a, v_b += x w' / m_b.
// Layout of a level slot: the pair word holds the byte offsets of v_a and v_b
// in the staged velocities (low / high 16 bits); the coefficient g = B/eta is
// stored negative for a pair with a constrained axis (1/m = 0 on that axis),
// which takes the per-axis path.  Free-free pairs (equal masses):
// v_a -= f w, v_b += f w with f = x/m / (1 + 2 x/m).  An empty slot points
// both offsets at a dummy velocity slot and has g = 0.
template <class R> __device__ __forceinline__ R fast_div(R a, R b) { return a / b; }
template <> __device__ __forceinline__ float fast_div<float>(float a, float b) { return __fdividef(a, b); }

template <class R, int D>
__device__ __forceinline__ void damp_apply(R *pa, R *pb, R g, const uint8_t *sf, uint32_t ia,
                                           uint32_t ib, R hcim, bool transpose = false) {
    constexpr int P = Pad<D>::v;
    R va[P], vb[P];
    ld_vec<R, P>(va, pa);
    ld_vec<R, P>(vb, pb);
    if (g >= R(0)) {
        const R xm = hcim * g;
        const R f2 = fast_div<R>(xm, R(1) + R(2) * xm);
#pragma unroll
        for (int q = 0; q < D; ++q) {
            const R d = va[q] - vb[q];
            va[q] -= f2 * d;
            vb[q] += f2 * d;
        }
    } else {
        // on an axis where one particle is constrained the free one moves by
        // x/m / (1 + x/m) w; a constrained one does not move
        const R xm = -hcim * g;
        const R f2 = fast_div<R>(xm, R(1) + R(2) * xm);
        const R f1 = fast_div<R>(xm, R(1) + xm);
        const uint8_t fa = sf[ia], fb = sf[ib];
#pragma unroll
        for (int q = 0; q < D; ++q) {
            const bool a_free = !((fa >> q) & 1), b_free = !((fb >> q) & 1);
            const R ca = a_free ? (b_free ? f2 : f1) : R(0);
            const R cb = b_free ? (a_free ? f2 : f1) : R(0);
            if (transpose) {    // the transposed 2x2 update (adjoint sweep)
                const R t = ca * va[q] - cb * vb[q];
                va[q] -= t;
                vb[q] += t;
            } else {
                const R d = va[q] - vb[q];
                va[q] -= ca * d;
                vb[q] += cb * d;
            }
        }
    }
    st_vec<R, P>(pa, va);
    st_vec<R, P>(pb, vb);
}

// The free-free branch of damp_apply alone (no lane of the level holds a
// constrained pair): the same arithmetic, nothing else on the level's chain.
template <class R, int D>
__device__ __forceinline__ void damp_pair_free(uint32_t w, R g, unsigned char *svb, R hcim) {
    constexpr int P = Pad<D>::v;
    R *pa = reinterpret_cast<R *>(svb + (w & 0xffffu));
    R *pb = reinterpret_cast<R *>(svb + (w >> 16));
    R va[P], vb[P];
    ld_vec<R, P>(va, pa);
    ld_vec<R, P>(vb, pb);
    const R xm = hcim * g;
    const R f2 = fast_div<R>(xm, R(1) + R(2) * xm);
#pragma unroll
    for (int q = 0; q < D; ++q) {
        const R d = va[q] - vb[q];
        va[q] -= f2 * d;
        vb[q] += f2 * d;
    }
    // an empty slot (coefficient 0, both offsets on the dummy slot) stores
    // nothing: several empty lanes of a quarter-warp would store to one
    // address and replay; loads of one address are a broadcast
    if (g != R(0)) {
        st_smem_vec<R, P>(pa, va);
        st_smem_vec<R, P>(pb, vb);
    }
}

// damp_apply for the warp-per-group kernel, where the pair word carries the
// constrained axes of both particles in the low three bits of each byte
// offset (velocity slots are at least 8 bytes, so those bits are free; they
// are zero for a free pair).  Branch-free: both factors are formed and each
// axis selects its coefficients, so every lane of a level runs the same
// instructions (a free pair takes ca = cb = f2 and the d form, exactly the
// free-free branch; data-dependent branches here cost more than the second
// division).  TR: the transposed 2x2 update for constrained pairs (adjoint).
template <class R, int D, bool TR>
__device__ __forceinline__ void damp_pair_coded(uint32_t w, R g, unsigned char *svb, R hcim) {
    constexpr int P = Pad<D>::v;
    const uint32_t fa = w & 7u, fb = (w >> 16) & 7u;
    R *pa = reinterpret_cast<R *>(svb + ((w & 0xffffu) & ~7u));
    R *pb = reinterpret_cast<R *>(svb + ((w >> 16) & ~7u));
    R va[P], vb[P];
    ld_vec<R, P>(va, pa);
    ld_vec<R, P>(vb, pb);
    const bool cons = g < R(0);
    const R xm = hcim * (cons ? -g : g);
    const R f2 = fast_div<R>(xm, R(1) + R(2) * xm);
    const R f1 = fast_div<R>(xm, R(1) + xm);
#pragma unroll
    for (int q = 0; q < D; ++q) {
        const bool a_free = !((fa >> q) & 1u), b_free = !((fb >> q) & 1u);
        const R ca = a_free ? (b_free ? f2 : f1) : R(0);
        const R cb = b_free ? (a_free ? f2 : f1) : R(0);
        const R d = va[q] - vb[q];
        if constexpr (TR) {
            const R t = ca * va[q] - cb * vb[q];
            const R na = cons ? va[q] - t : va[q] - ca * d;
            const R nb = cons ? vb[q] + t : vb[q] + cb * d;
            va[q] = na;
            vb[q] = nb;
        } else {
            va[q] -= ca * d;
            vb[q] += cb * d;
        }
    }
    if (g != R(0)) {        // empty slots store nothing (see damp_pair_free)
        st_smem_vec<R, P>(pa, va);
        st_smem_vec<R, P>(pb, vb);
    }
}

// One half-sweep of a warp over its group's levels (forward or reverse).  The
// level slots (lane-indexed: lane k only ever reads slot k of a level) stream
// through a per-warp ring of two chunks of kDampChunk levels in shared memory:
// each lane copies its own slots with cp.async a chunk ahead of the one being
// applied, so the ring needs no barrier and the warp's shared memory stays
// small (more warps per SM than staging every level would allow).  primed:
// the caller has already issued chunks 0 and 1 of this sweep.  CONS: the
// group touches a constrained particle, so every level takes the coded update.
template <class R>
__device__ __forceinline__ void damp_stage_chunk(int c, int nl, bool fwd, const uint32_t *gab,
                                                 const R *gg, uint32_t *rw, R *rg, int lane) {
    const int b = c & 1;
#pragma unroll 4
    for (int j = 0; j < kDampChunk; ++j) {
        const int k = c * kDampChunk + j;
        if (k < nl) {
            const int l = fwd ? k : nl - 1 - k;
            cp_async(rw + (b * kDampChunk + j) * 32 + lane, gab + 32 * l + lane, 4);
            cp_async(rg + (b * kDampChunk + j) * 32 + lane, gg + 32 * l + lane, (int)sizeof(R));
        }
    }
    cp_async_commit();
}

template <class R, int D, bool CONS, bool FWD, bool TR>
__device__ __forceinline__ void damp_sweep(int nl, const uint32_t *gab, const R *gg, int lane,
                                           unsigned char *svb, R hcim, uint32_t *rw, R *rg,
                                           bool primed) {
    if (!primed) {
        damp_stage_chunk<R>(0, nl, FWD, gab, gg, rw, rg, lane);
        damp_stage_chunk<R>(1, nl, FWD, gab, gg, rw, rg, lane);
    }
    const int nch = (nl + kDampChunk - 1) / kDampChunk;
    for (int c = 0; c < nch; ++c) {
        cp_async_wait_group<1>();           // chunk c has landed (c + 1 may be in flight)
        const int b = c & 1;
        const int kend = min(kDampChunk, nl - c * kDampChunk);
        for (int j = 0; j < kend; ++j) {
            const uint32_t w = rw[(b * kDampChunk + j) * 32 + lane];
            const R gc = rg[(b * kDampChunk + j) * 32 + lane];
            if constexpr (CONS)
                damp_pair_coded<R, D, TR>(w, gc, svb, hcim);
            else
                damp_pair_free<R, D>(w, gc, svb, hcim);
            __syncwarp();
        }
        // this lane has consumed its slots of buffer b: refill it with chunk c + 2
        damp_stage_chunk<R>(c + 2, nl, FWD, gab, gg, rw, rg, lane);
    }
    cp_async_wait_all();
}

// The same half-sweep with every level of the group already in shared memory
// (sab, sg: 32 slots per level), prefetching the next level's slot off the
// velocity chain.
template <class R, int D, bool CONS, bool FWD, bool TR>
__device__ __forceinline__ void damp_sweep_staged(int nl, const uint32_t *sab, const R *sg, int lane,
                                                  unsigned char *svb, R hcim) {
    int l = FWD ? 0 : nl - 1;
    uint32_t wn = sab[32 * l + lane];
    R gn = sg[32 * l + lane];
    for (int k = 0; k < nl; ++k, l += FWD ? 1 : -1) {
        const uint32_t w = wn;
        const R gc = gn;
        if (k + 1 < nl) {
            const int ln = FWD ? l + 1 : l - 1;
            wn = sab[32 * ln + lane];
            gn = sg[32 * ln + lane];
        }
        if constexpr (CONS)
            damp_pair_coded<R, D, TR>(w, gc, svb, hcim);
        else
            damp_pair_free<R, D>(w, gc, svb, hcim);
        __syncwarp();
    }
}

template <class R, int D, bool CONS, bool TR, bool RING>
__device__ __forceinline__ void damp_sweeps_c(int mode, int nl, const uint32_t *gab, const R *gg,
                                              int lane, unsigned char *svb, R hcim, uint32_t *rw,
                                              R *rg) {
    if constexpr (RING) {
        // the first sweep's chunks 0 and 1 were issued before the chain wait
        if (mode & 1) damp_sweep<R, D, CONS, true, TR>(nl, gab, gg, lane, svb, hcim, rw, rg, true);
        if (mode & 2)
            damp_sweep<R, D, CONS, false, TR>(nl, gab, gg, lane, svb, hcim, rw, rg, !(mode & 1));
    } else {
        if (mode & 1) damp_sweep_staged<R, D, CONS, true, TR>(nl, rw, rg, lane, svb, hcim);
        if (mode & 2) damp_sweep_staged<R, D, CONS, false, TR>(nl, rw, rg, lane, svb, hcim);
    }
}

template <class R, int D, bool TR, bool RING>
__device__ __forceinline__ void damp_sweeps(bool cons, int mode, int nl, const uint32_t *gab,
                                            const R *gg, int lane, unsigned char *svb, R hcim,
                                            uint32_t *rw, R *rg) {
    if (cons)
        damp_sweeps_c<R, D, true, TR, RING>(mode, nl, gab, gg, lane, svb, hcim, rw, rg);
    else
        damp_sweeps_c<R, D, false, TR, RING>(mode, nl, gab, gg, lane, svb, hcim, rw, rg);
}

// RING: the level slots stream through the two-chunk ring (small shared
// memory per warp: many warps per SM, for bodies with many groups per colour);
// otherwise every level of the group is staged before the chain wait (the
// shortest chain, for bodies with few groups per SM).
template <class R, int D, bool RING>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? 6 : 4) k_damp(Args<R> A, long long g_begin, long long g_end,
                                                                         int mode, long long n_begin, long long n_end) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int P = Pad<D>::v;
    constexpr int NB = 1 << D;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long g = g_begin + (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    chain_trigger();
    if (g >= g_end) return;
    // every scalar the group needs, issued together (one memory latency)
    int ts[NB], tc[NB];
#pragma unroll
    for (int e = 0; e < NB; ++e) {
        ts[e] = __ldg(A.touch_start + g * NB + e);
        tc[e] = __ldg(A.touch_cnt + g * NB + e);
    }
    const int l0 = __ldg(A.grp_lvl + g), l1 = __ldg(A.grp_lvl + g + 1);
    const bool cons = __ldg(A.grp_cons + g) != 0;
    const int nl = l1 - l0;
    const int mb = A.mb;
    // the next launch's group of the same rank, prefetched into L2 while this
    // warp's chain runs (n_begin = n_end: none)
    const long long h = n_begin + (g - g_begin);
    int m0 = 0, m1 = 0;
    if (lane == 0 && h < n_end) {
        m0 = __ldg(A.grp_lvl + h);
        m1 = __ldg(A.grp_lvl + h + 1);
    }
    unsigned char *base =
        smem + (size_t)warp * DampSmem<R, D>::bytes(mb, A.max_group_levels, RING);
    R *sv = reinterpret_cast<R *>(base);
    uint32_t *rw = reinterpret_cast<uint32_t *>(base + DampSmem<R, D>::vbytes(mb));
    R *rg = reinterpret_cast<R *>(rw + 32 * (RING ? 2 * kDampChunk : A.max_group_levels));
    // 32 slots per level: pair word and coefficient (set-up data, so they are
    // issued before the chain wait and may overlap the previous kernel: the
    // first two chunks of the first sweep, or every level)
    const uint32_t *gab = A.pair_ab + 32LL * l0;
    const R *gg = A.pair_g + 32LL * l0;
    if constexpr (RING) {
        damp_stage_chunk<R>(0, nl, (mode & 1) != 0, gab, gg, rw, rg, lane);
        damp_stage_chunk<R>(1, nl, (mode & 1) != 0, gab, gg, rw, rg, lane);
    } else {
        for (int k = 4 * lane; k < 32 * nl; k += 128) cp_async(rw + k, gab + k, 16);
        constexpr int GPER = 16 / (int)sizeof(R);
        for (int k = GPER * lane; k < 32 * nl; k += 32 * GPER) cp_async(rg + k, gg + k, 16);
    }
    chain_wait();
    const int done = A.ctrl->done;
    const double dt = A.ctrl->dt;
    if (done) {
        cp_async_wait_all();
        return;
    }
    // the touched blocks' velocities, once the previous kernel has completed
    constexpr int SB = P * (int)sizeof(R);   // bytes per velocity slot
#pragma unroll
    for (int e = 0; e < NB; ++e)
        for (int t = lane; t < tc[e]; t += 32)
            cp_async_reals<R, P>(sv + (size_t)damp_slot_pos(e * mb + t, SB) * P,
                                 A.v + (size_t)(ts[e] + t) * P);
    if (lane == 0) {
        R z[P];
#pragma unroll
        for (int q = 0; q < P; ++q) z[q] = R(0);
        // dummy slot of the empty level slots
        st_vec<R, P>(sv + (size_t)damp_slot_pos(NB * mb, SB) * P, z);
    }
    cp_async_wait_all();
    __syncwarp();
    if (lane == 0) prefetch_group_levels<R>(A, m0, m1);
    const R im = (R)(1.0 / A.mass);
    const R hcim = (R)(0.5 * dt) * A.eta * im;   // (dt/2) eta / m
    const bool tr = A.transpose != 0;
    unsigned char *svb = reinterpret_cast<unsigned char *>(sv);
    // a group that touches no constrained particle has no negative
    // coefficient and runs the free-pair loop alone
    if (nl > 0) {
        if (tr)
            damp_sweeps<R, D, true, RING>(cons, mode, nl, gab, gg, lane, svb, hcim, rw, rg);
        else
            damp_sweeps<R, D, false, RING>(cons, mode, nl, gab, gg, lane, svb, hcim, rw, rg);
    }
#pragma unroll
    for (int e = 0; e < NB; ++e)
        for (int t = lane; t < tc[e]; t += 32) {
            R vv[P];
            ld_vec<R, P>(vv, sv + (size_t)damp_slot_pos(e * mb + t, SB) * P);
            st_vec<R, P>(A.v + (long long)(ts[e] + t) * P, vv);
        }
    // a next launch with more groups than this one: the rest, after this
    // warp's own work
    if (lane == 0)
        for (long long hh = h + (g_end - g_begin); hh < n_end; hh += g_end - g_begin)
            prefetch_group_levels<R>(A, __ldg(A.grp_lvl + hh), __ldg(A.grp_lvl + hh + 1));
}

// ------------------------------------------------- damping, one launch
// The symmetric sweep as one launch (BLOCKS layout).  The multi-launch form
// runs one launch per colour (forward on all but the last colour, forward and
// reverse fused on the last, then reverse), with the whole GPU between two
// launches.  Here every (launch, group) pair of that sequence is a task, taken
// by a warp from a queue in sweep order; before it touches the velocities, a
// task waits until every earlier task touching one of its 2^d blocks has
// finished (a per-block count of finished tasks, written with release and
// read with acquire semantics).  Each task then computes exactly what its
// group computes in the multi-launch form, on the same velocities, so the
// results are bit for bit the same.  Tasks are taken in sweep order and wait
// only on earlier tasks, all held by running warps, so the queue always
// progresses; a wait that exceeds kPersistWaitNs nonetheless gives up, flags
// MTS_ERR_TIMEOUT in the control block and stops the slow step.
constexpr unsigned long long kPersistWaitNs = 2000000000ull;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

struct PersistArgs {
    const int32_t *blk;    // per group x 2^d
    const uint8_t *req;    // per task x 2^d
    unsigned *done;        // per block; done[nblocks] = the task queue
    long long nblocks, ntasks;
    int nph;
    long long off[17], goff[16];
    int mode[16];
};

__global__ void k_persist_reset(unsigned *done, long long count) {
    chain_trigger();
    chain_wait();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        done[i] = 0u;
}

// velocity slot in, bypassing L1 (another SM may have written it in this launch)
template <class R, int P>
__device__ __forceinline__ void stage_velocity_l2(R *s, const R *g) {
    if constexpr (P * sizeof(R) == 8) {
        const float2 t = __ldcg(reinterpret_cast<const float2 *>(g));
        *reinterpret_cast<float2 *>(s) = t;
    } else {
        cp_async_reals<R, P>(s, g);      // 16-byte copies: cp.async.cg, L2 only
    }
}

template <class R, int D, bool RING>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? 6 : 4) k_damp_persist(Args<R> A, PersistArgs Q) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int P = Pad<D>::v;
    constexpr int NB = 1 << D;
    constexpr int SB = P * (int)sizeof(R);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    chain_trigger();
    chain_wait();
    if (A.ctrl->done) return;
    const double dt = A.ctrl->dt;
    const int mb = A.mb;
    unsigned char *base =
        smem + (size_t)warp * DampSmem<R, D>::bytes(mb, A.max_group_levels, RING);
    R *sv = reinterpret_cast<R *>(base);
    uint32_t *rw = reinterpret_cast<uint32_t *>(base + DampSmem<R, D>::vbytes(mb));
    R *rg = reinterpret_cast<R *>(rw + 32 * (RING ? 2 * kDampChunk : A.max_group_levels));
    const R im = (R)(1.0 / A.mass);
    const R hcim = (R)(0.5 * dt) * A.eta * im;
    unsigned char *svb = reinterpret_cast<unsigned char *>(sv);
    unsigned *queue = Q.done + Q.nblocks;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(queue, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if ((long long)t >= Q.ntasks) break;
        int p = 0;
        while (p + 1 < Q.nph && (long long)t >= Q.off[p + 1]) ++p;
        const long long g = Q.goff[p] + ((long long)t - Q.off[p]);
        const int mode = Q.mode[p];
        int ts[NB], tc[NB], bk[NB];
#pragma unroll
        for (int e = 0; e < NB; ++e) {
            ts[e] = __ldg(A.touch_start + g * NB + e);
            tc[e] = __ldg(A.touch_cnt + g * NB + e);
            bk[e] = __ldg(Q.blk + g * NB + e);
        }
        const int l0 = __ldg(A.grp_lvl + g), l1 = __ldg(A.grp_lvl + g + 1);
        const bool cons = __ldg(A.grp_cons + g) != 0;
        const int nl = l1 - l0;
        const uint32_t *gab = A.pair_ab + 32LL * l0;
        const R *gg = A.pair_g + 32LL * l0;
        // set-up data first: it does not depend on the earlier tasks (the
        // ring's later chunks stream from L2 once this prefetch has landed)
        if constexpr (RING) {
            damp_stage_chunk<R>(0, nl, (mode & 1) != 0, gab, gg, rw, rg, lane);
            damp_stage_chunk<R>(1, nl, (mode & 1) != 0, gab, gg, rw, rg, lane);
        } else {
            for (int k = 4 * lane; k < 32 * nl; k += 128) cp_async(rw + k, gab + k, 16);
            constexpr int GPER = 16 / (int)sizeof(R);
            for (int k = GPER * lane; k < 32 * nl; k += 32 * GPER) cp_async(rg + k, gg + k, 16);
        }
        // lane e < 2^d looks after touched block e
        int my_tc = 0, my_bk = 0;
#pragma unroll
        for (int e = 0; e < NB; ++e)
            if (lane == e) {
                my_tc = tc[e];
                my_bk = bk[e];
            }
        // wait for the earlier tasks on this group's blocks
        if (lane < NB && my_tc > 0) {
            const unsigned need = __ldg(Q.req + t * NB + lane);
            const unsigned *cnt = Q.done + my_bk;
            if (ld_acquire_u32(cnt) < need) {
                const unsigned long long t0 = global_ns();
                while (ld_acquire_u32(cnt) < need) {
                    __nanosleep(64);
                    if (global_ns() - t0 > kPersistWaitNs) {
                        atomicExch(&A.ctrl->status, (int)MTS_ERR_TIMEOUT);
                        atomicExch(&A.ctrl->done, 1);
                        break;
                    }
                }
            }
        }
        __syncwarp();
#pragma unroll
        for (int e = 0; e < NB; ++e)
            for (int k = lane; k < tc[e]; k += 32)
                stage_velocity_l2<R, P>(sv + (size_t)damp_slot_pos(e * mb + k, SB) * P,
                                        A.v + (size_t)(ts[e] + k) * P);
        if (lane == 0) {
            R z[P];
#pragma unroll
            for (int q = 0; q < P; ++q) z[q] = R(0);
            st_vec<R, P>(sv + (size_t)damp_slot_pos(NB * mb, SB) * P, z);
        }
        cp_async_wait_all();
        __syncwarp();
        if (nl > 0) damp_sweeps<R, D, false, RING>(cons, mode, nl, gab, gg, lane, svb, hcim, rw, rg);
#pragma unroll
        for (int e = 0; e < NB; ++e)
            for (int k = lane; k < tc[e]; k += 32) {
                R vv[P];
                ld_vec<R, P>(vv, sv + (size_t)damp_slot_pos(e * mb + k, SB) * P);
                st_vec<R, P>(A.v + (long long)(ts[e] + k) * P, vv);
            }
        __syncwarp();
        // release: this warp's velocity stores before the counts the next tasks read
        if (lane < NB && my_tc > 0) {
            __threadfence();
            atomicAdd(Q.done + my_bk, 1u);
        }
        __syncwarp();
    }
}

// ------------------------------------------------- damping, wide layout
// One CTA per owner group.  Shared memory: the touched blocks' velocities and
// flags (gathered through the block-sorted permutation), the group's level
// offsets, and a ring of three level buffers (pair words with 16-bit slot
// indices, signed coefficients) filled by cp.async two levels ahead of the
// level being applied; one barrier per level.
__host__ __device__ inline void wide_offsets(int slots, int maxl, int lc, int P, int rs,
                                             size_t off[4], size_t *total) {
    auto r16 = [](size_t x) { return (x + 15) & ~size_t(15); };
    off[0] = r16((size_t)slots * P * rs);          // flags
    off[1] = off[0] + r16((size_t)slots);           // level offsets
    off[2] = off[1] + r16((size_t)(maxl + 1) * 4);  // ring of pair words
    off[3] = off[2] + r16((size_t)kWideRing * lc * 4);   // ring of coefficients
    *total = off[3] + r16((size_t)kWideRing * lc * rs);
}

template <class R, int D>
__device__ __forceinline__ void wide_sweep(bool fwd, int nl, const int32_t *slv, long long p0,
                                           const uint32_t *gw, const R *gg, uint32_t *sw, R *sgr,
                                           int lc, R *sv, const uint8_t *sf, R hcim,
                                           bool transpose) {
    constexpr int P = Pad<D>::v;
    const int tid = threadIdx.x;
    auto issue = [&](int i) {
        if (i < nl) {
            const int L = fwd ? i : nl - 1 - i;
            const int s0 = slv[L], cnt = slv[L + 1] - s0;
            const int buf = (i % kWideRing) * lc;
            for (int k = tid; k < cnt; k += kWideThreads) {
                cp_async(sw + buf + k, gw + p0 + s0 + k, 4);
                cp_async(sgr + buf + k, gg + p0 + s0 + k, (int)sizeof(R));
            }
        }
        cp_async_commit();
    };
#pragma unroll
    for (int i = 0; i < kWideRing - 1; ++i) issue(i);
    for (int i = 0; i < nl; ++i) {
        cp_async_wait_group<kWideRing - 2>();   // level i has landed (later ones may be in flight)
        __syncthreads();            // ... for every thread; level i - 1 applied everywhere
        issue(i + kWideRing - 1);   // into the buffer level i - 1 used
        const int L = fwd ? i : nl - 1 - i;
        const int cnt = slv[L + 1] - slv[L];
        const int buf = (i % kWideRing) * lc;
        for (int k = tid; k < cnt; k += kWideThreads) {
            const uint32_t w = sw[buf + k];
            const R gc = sgr[buf + k];
            const uint32_t ia = w & 0xffffu, ib = w >> 16;
            damp_apply<R, D>(sv + (size_t)ia * P, sv + (size_t)ib * P, gc, sf, ia, ib, hcim,
                             transpose);
        }
    }
    cp_async_wait_all();
    __syncthreads();
}

template <class R, int D>
__global__ void __launch_bounds__(kWideThreads) k_damp_wide(Args<R> A, long long g_begin, int mode) {
    chain_trigger();
    chain_wait();
    if (A.ctrl->done) return;
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int P = Pad<D>::v;
    constexpr int NB = 1 << D;
    const long long g = g_begin + blockIdx.x;
    const int tid = threadIdx.x;
    const int mb = A.mb, nbw = A.nbw, lc = A.max_level_pairs;
    size_t off[4], smem_total;
    wide_offsets(nbw * mb, A.max_group_levels, lc, P, (int)sizeof(R), off, &smem_total);
    R *sv = reinterpret_cast<R *>(smem);
    uint8_t *sf = smem + off[0];
    int32_t *slv = reinterpret_cast<int32_t *>(smem + off[1]);
    uint32_t *sw = reinterpret_cast<uint32_t *>(smem + off[2]);
    R *sgr = reinterpret_cast<R *>(smem + off[3]);
    // touched blocks, flattened: entry j < total lies in block e with
    // pre[e] <= j < pre[e + 1]
    int ts[NB], pre[NB + 1];
    pre[0] = 0;
#pragma unroll
    for (int e = 0; e < NB; ++e) {
        ts[e] = e < nbw ? __ldg(A.touch_start + g * NB + e) : 0;
        pre[e + 1] = pre[e] + (e < nbw ? __ldg(A.touch_cnt + g * NB + e) : 0);
    }
    const int total = pre[NB];
    auto locate = [&](int j, int &src, int &slot) {
#pragma unroll
        for (int e = 0; e < NB; ++e)
            if (j >= pre[e]) {
                src = ts[e] + (j - pre[e]);
                slot = e * mb + (j - pre[e]);
            }
    };
    const int l0 = __ldg(A.grp_lvl + g), l1 = __ldg(A.grp_lvl + g + 1);
    const int nl = l1 - l0;
    const long long p0 = __ldg(A.lvl_pair + l0);
    // gather in batches of kSB per thread: indices and flags (block-sorted,
    // contiguous) first, then the velocity copies that depend on them
    constexpr int kSB = 8;
    for (int j0 = 0; j0 < total; j0 += kSB * kWideThreads) {
        int pp[kSB], sl[kSB];
        uint8_t ff[kSB];
#pragma unroll
        for (int u = 0; u < kSB; ++u) {
            const int j = j0 + u * kWideThreads + tid;
            sl[u] = -1;
            if (j < total) {
                int src = 0;
                locate(j, src, sl[u]);
                pp[u] = __ldg(A.bperm + src);
                ff[u] = __ldg(A.bflags + src);
            }
        }
#pragma unroll
        for (int u = 0; u < kSB; ++u)
            if (sl[u] >= 0) {
                cp_async_reals<R, P>(sv + (size_t)sl[u] * P, A.v + (long long)pp[u] * P);
                sf[sl[u]] = ff[u];
            }
    }
    for (int t = tid; t <= nl; t += kWideThreads) slv[t] = (int)(__ldg(A.lvl_pair + l0 + t) - p0);
    cp_async_wait_all();
    __syncthreads();
    const R hcim = (R)(0.5 * A.ctrl->dt) * A.eta * (R)(1.0 / A.mass);   // (dt/2) eta / m
    const bool tr = A.transpose != 0;
    if (mode & 1) wide_sweep<R, D>(true, nl, slv, p0, A.pair_ab, A.pair_g, sw, sgr, lc, sv, sf, hcim, tr);
    if (mode & 2) wide_sweep<R, D>(false, nl, slv, p0, A.pair_ab, A.pair_g, sw, sgr, lc, sv, sf, hcim, tr);
    for (int j0 = 0; j0 < total; j0 += kSB * kWideThreads) {
        int pp[kSB], sl[kSB];
#pragma unroll
        for (int u = 0; u < kSB; ++u) {
            const int j = j0 + u * kWideThreads + tid;
            sl[u] = -1;
            if (j < total) {
                int src = 0;
                locate(j, src, sl[u]);
                pp[u] = __ldg(A.bperm + src);
            }
        }
#pragma unroll
        for (int u = 0; u < kSB; ++u)
            if (sl[u] >= 0) {
                R vv[P];
                ld_vec<R, P>(vv, sv + (size_t)sl[u] * P);
                st_vec<R, P>(A.v + (long long)pp[u] * P, vv);
            }
    }
}

// flags in block-sorted order (the wide damping kernel's contiguous reads)
__global__ void k_gather_flags(const uint8_t *flags, const int32_t *bperm, long long n,
                               uint8_t *bflags) {
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s < n) bflags[s] = flags[bperm[s]];
}

// blocks layout: does an owner group touch a particle with a constrained axis
// (its particles are the touched blocks' contiguous ranges)
__global__ void k_group_cons(const int32_t *tstart, const int32_t *tcnt, long long ng, int nb,
                             const uint8_t *flags, int fixmask, uint8_t *cons) {
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g >= ng) return;
    uint8_t any = 0;
    for (int e = 0; e < nb; ++e) {
        const long long s0 = tstart[g * nb + e];
        for (int t = 0; t < tcnt[g * nb + e]; ++t) any |= flags[s0 + t] & fixmask;
    }
    cons[g] = any != 0;
}

// blocks layout: the constrained axes of both particles in the low three bits
// of each byte offset of the padded pair word (low half: pair_a, or pair_b
// where the set-up reversed the pair: kSlotSwapBit of pair_slot)
__global__ void k_pair_fixword(uint32_t *kab, const long long *slot, const int32_t *pa,
                               const int32_t *pb, long long m, const uint8_t *flags, int fixmask) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= m) return;
    const long long s = slot[p];
    uint32_t fa = flags[pa[p]] & fixmask, fb = flags[pb[p]] & fixmask;
    if ((s >> kSlotSwapBit) & 1) {
        const uint32_t t = fa;
        fa = fb;
        fb = t;
    }
    uint32_t &w = kab[s & kSlotMask];
    w = (w & ~(7u | (7u << 16))) | fa | (fb << 16);
}

// pair coefficients: negative when either particle has a constrained axis
template <class R>
__global__ void k_pair_fixsign(R *kg, const long long *slot, const int32_t *pa, const int32_t *pb,
                               long long m, const uint8_t *flags, int fixmask) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= m) return;
    const bool fix = (flags[pa[p]] | flags[pb[p]]) & fixmask;
    R &c = kg[slot[p] & kSlotMask];
    const R a = c < R(0) ? -c : c;
    c = fix ? -a : a;
}

// --------------------------------------------------------------------- drift
// COND: launched inside the conditional WHILE node (sets its condition); the
// other variant carries no conditional-handle code, so profilers can capture
// it inside ordinary graphs
template <class R, int D, bool COND>
__global__ void __launch_bounds__(kBlock) k_drift(Args<R> A) {
    chain_trigger();
    chain_wait();
    Control *C = A.ctrl;
    if (C->done) {
        // defensive: a loop iteration that starts after the stop ends the loop
        if constexpr (COND)
            if (blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(A.cond, 0u);
        return;
    }
    constexpr int P = Pad<D>::v;
    // each thread drifts several particles (grid stride) and keeps FP64
    // partials of sum |v|^2 and max |v|^2; 1/2 m and the square root are
    // applied once, to the totals (max |v| = sqrt(max |v|^2) exactly)
    double v2sum = 0.0, v2max = 0.0;
    R v2maxr = R(0);
    {
        const double dt = C->dt, ramp = C->ramp;
        const long long stride = (long long)gridDim.x * kBlock;
        // the launch gives each thread up to kDriftPer particles (i0, i0 +
        // stride, ...): all their loads are issued before the arithmetic
        constexpr int kDriftPer = 2;
        for (long long i0 = blockIdx.x * (long long)kBlock + threadIdx.x; i0 < A.n;
             i0 += kDriftPer * stride) {
            uint8_t fx[kDriftPer];
            R v[kDriftPer][P];
            double u[kDriftPer][P];
#pragma unroll
            for (int j = 0; j < kDriftPer; ++j) {
                const long long i = i0 + j * stride;
                if (i < A.n) {
                    fx[j] = A.flags[i];
                    ld_vec<R, P>(v[j], A.v + i * P);
                    ld_vec<double, P>(u[j], A.u + i * P);
                }
            }
#pragma unroll
            for (int j = 0; j < kDriftPer; ++j) {
                const long long i = i0 + j * stride;
                if (i >= A.n) break;
                // |v|^2 per particle in the velocity's own precision (in
                // mixed precision a relative rounding of 2^-24 on FP32
                // velocities); summed, maximised and compared in FP64.
                // Mixed precision converts between FP32 and FP64 on the
                // integer pipe: the same bits, off the FP64 pipe.
                R v2r = R(0);
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    if ((fx[j] >> k) & 1) {
                        v[j][k] = R(0);
                        u[j][k] = ramp * A.u_unit[i * P + k];
                    } else {
                        if constexpr (sizeof(R) == 4)
                            u[j][k] += dt * f2d_bits(v[j][k]);
                        else
                            u[j][k] += dt * (double)v[j][k];
                    }
                    v2r += v[j][k] * v[j][k];
                }
                st_vec<R, P>(A.v + i * P, v[j]);
                st_vec<double, P>(A.u + i * P, u[j]);
                if constexpr (sizeof(R) == 4) {
                    R uf[P];
#pragma unroll
                    for (int k = 0; k < P; ++k) uf[k] = k < D ? d2f_bits(u[j][k]) : R(0);   // padding stays 0
                    st_vec<R, P>(A.uf + i * P, uf);
                    v2sum += f2d_bits(v2r);
                    v2maxr = fmaxf(v2maxr, v2r);       // widening is exact and monotonic
                } else {
                    v2sum += (double)v2r;
                    v2max = fmax(v2max, (double)v2r);
                }
            }
        }
    }
    // mixed precision: the warp's max |v|^2 taken in FP32, then widened (the
    // same value: widening is exact and monotonic)
    if constexpr (sizeof(R) == 4) v2max = f2d_bits(warp_max(v2maxr));
    double ke = v2sum, vmax = v2max;
    __shared__ double sh[2][kBlock / 32];
    __shared__ int is_last;
    ke = warp_sum(ke);
    if constexpr (sizeof(R) != 4) vmax = warp_max(vmax);
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
    // last block: fixed-order reduction of every block's partials (loads
    // issued four at a time, accumulated in a fixed order)
    double s_ke = 0, s_v = 0, s_a = 0, s_f[3] = {0, 0, 0};
    for (unsigned q0 = threadIdx.x; q0 < gridDim.x; q0 += 4 * kBlock) {
        double2 t[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const unsigned q = q0 + u * kBlock;
            t[u] = q < gridDim.x ? __ldcg(reinterpret_cast<const double2 *>(A.part_drift) + q)
                                 : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            s_ke += t[u].x;
            s_v = fmax(s_v, t[u].y);
        }
    }
    for (long long q0 = threadIdx.x; q0 < A.ntiles; q0 += 4 * kBlock) {   // one partial per force CTA
        double2 t[4][2];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long long q = q0 + u * kBlock;
            const double2 z = make_double2(0.0, 0.0);
            t[u][0] = q < A.ntiles ? __ldcg(reinterpret_cast<const double2 *>(A.part_force) + 2 * q) : z;
            t[u][1] = q < A.ntiles ? __ldcg(reinterpret_cast<const double2 *>(A.part_force) + 2 * q + 1) : z;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            s_a = fmax(s_a, t[u][0].x);
            s_f[0] += t[u][0].y;
            s_f[1] += t[u][1].x;
            s_f[2] += t[u][1].y;
        }
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
        const double KE = 0.5 * A.mass * red[0][0], VM = sqrt(red[1][0]), AM = sqrt(red[2][0]);
        // Sec. 4.2 with Sec. 5.1/5.3: after the slow step's event E_k rises to a
        // peak, then decays to the criterion; the test is armed from the first
        // substep with E_k(n) <= E_k(n-1) (E_k(0) = 0, the value C->ke is reset to)
        if (KE <= C->ke) C->armed = 1;
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
            if (C->use_tol && C->armed && crit <= C->ke_thr) {
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
        if constexpr (COND) cudaGraphSetConditional(A.cond, C->done ? 0u : 1u);
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
    C->nsub = 0; C->done = 0; C->converged = 0; C->status = 0; C->counter = 0; C->armed = 0;
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
__global__ void __launch_bounds__(TileThreads<R>::v) k_diffuse(Args<R> A, R dt) {
    constexpr int P = Pad<D>::v;
    extern __shared__ __align__(16) unsigned char smem[];
    R *sX = reinterpret_cast<R *>(smem);
    R *sC = reinterpret_cast<R *>(smem + second_off<R, P>(A.max_halo));
    const long long t = blockIdx.x;
    const long long h0 = A.halo_off[t];
    const int nh = (int)(A.halo_off[t + 1] - h0);
    for (int k = threadIdx.x; k < nh; k += blockDim.x) {
        const long long g = __ldg(A.halo_idx + h0 + k);
        R x[P];
        ldg_vec<R, P>(x, A.halo_x + (h0 + k) * P);
        st_vec<R, P>(sX + k * P, x);
        sC[k] = A.c[g];
    }
    __syncthreads();
    const long long i = t * A.T + threadIdx.x;
    if (i >= A.n) return;
    if (A.flags[i] & kCHeldBit) {
        A.c_tmp[i] = A.c_held[i];
        return;
    }
    const int li = A.lself[i];
    R xa[P];
    ld_vec<R, P>(xa, sX + li * P);
    const R ca = sC[li];
    R s = R(0);
    const uint16_t *row = A.lell + A.lell_off[t] + threadIdx.x;
    const int w = A.tile_w[t];
    for (int j = 0; j < w; ++j) {
        const int l = __ldg(row + j * A.T);
        R xb[P];
        ld_vec<R, P>(xb, sX + l * P);
        R r2 = R(0);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const R d = xa[k] - xb[k];
            r2 += d * d;
        }
        const R tt = R(1) - R(0.5) * nsqrt(r2) * A.inv_h;
        s += (ca - sC[l]) * tt * tt * tt;
    }
    A.c_tmp[i] = ca + dt * A.dcoef * s;
}

// Two-stage diffusion in the deformed configuration (Sec. 3.2: flux, then its
// divergence, kernel gradients mapped by F), written in the reference
// configuration through the Piola transform of the flux:
//   stage 1  Q_a = -D J_a C_a^-1 B0_a^T sum_b V (c_b - c_a) grad0_a W_ab,  C = F^T F
//   stage 2  c_a <- c_a - dt sum_b V (Q_a + Q_b) . grad0_a W_ab   (free-c particles)
// Stage 1 stages X, u and c of the tile's halo (F as in the stress kernel).
template <class R, int D>
__device__ __forceinline__ void inv_cauchy_green(const R (&F)[3][3], R (&Ci)[3][3], R &J) {
    R Cm[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Cm[i][j] = F[0][i] * F[0][j] + F[1][i] * F[1][j] + F[2][i] * F[2][j];
    R cof[3][3];
    m3_cof(Cm, cof);                       // symmetric: cof = det(C) C^-1
    const R idet = R(1) / m3_det(Cm);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Ci[i][j] = cof[i][j] * idet;
    J = m3_det(F);
}

template <class R, int D>
__global__ void __launch_bounds__(TileThreads<R>::v) k_diff_flux(Args<R> A) {
    constexpr int P = Pad<D>::v;
    extern __shared__ __align__(16) unsigned char smem[];
    const size_t o1 = second_off<R, P>(A.max_halo);
    R *sX = reinterpret_cast<R *>(smem);
    R *sU = reinterpret_cast<R *>(smem + o1);
    R *sC = reinterpret_cast<R *>(smem + 2 * o1);
    stage_halo<R, P, P>(A, sX, sU, A.uf);
    const long long t = blockIdx.x;
    const long long h0 = A.halo_off[t];
    const int nh = (int)(A.halo_off[t + 1] - h0);
    for (int k = threadIdx.x; k < nh; k += blockDim.x) sC[k] = A.c[__ldg(A.halo_idx + h0 + k)];
    __syncthreads();
    const long long i = t * A.T + threadIdx.x;
    if (i >= A.n) return;
    R F[3][3];
    compute_F<R, D>(A, sX, sU, i, F);
    unscale_F<R, D>(A, F);
    const int li = A.lself[i];
    R xa[P];
    ld_vec<R, P>(xa, sX + li * P);
    const R ca = sC[li];
    R g[D];
#pragma unroll
    for (int k = 0; k < D; ++k) g[k] = R(0);
    const uint16_t *row = A.lell + A.lell_off[t] + threadIdx.x;
    for_each_neighbour(row, A.T, A.tile_w[t], [&](int l) {
        R xb[P];
        ld_vec<R, P>(xb, sX + l * P);
        R d[D], r2 = R(0);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            d[k] = xa[k] - xb[k];
            r2 += d[k] * d[k];
        }
        const R tt = R(1) - R(0.5) * nsqrt(r2) * A.inv_h;
        const R f = A.kcoef * tt * tt * tt * (sC[l] - ca);   // V W'/r (c_b - c_a)
#pragma unroll
        for (int k = 0; k < D; ++k) g[k] += f * d[k];
    });
    R B[D][D];
    ldg_mat<R, D>(B, A.B0 + i * MatS<D>::v);
    R g0[D];   // reference gradient of c: B0^T g (anisotropic: s (.) B0~^T g~)
#pragma unroll
    for (int r = 0; r < D; ++r) {
        R s = R(0);
#pragma unroll
        for (int k = 0; k < D; ++k) s += B[k][r] * g[k];
        g0[r] = A.aniso ? s * A.sk[r] : s;
    }
    R Ci[3][3], J;
    inv_cauchy_green<R, D>(F, Ci, J);
    R q[P];
#pragma unroll
    for (int r = 0; r < P; ++r) {
        R s = R(0);
        if (r < D)
#pragma unroll
            for (int k = 0; k < D; ++k) s += Ci[r][k] * g0[k];
        // stored for the divergence gather on scaled positions: detS s (.) Q
        q[r] = r < D ? -A.diffD * J * s * (A.aniso ? A.detS * A.sk[r] : R(1)) : R(0);
    }
    st_vec<R, P>(A.qflux + i * P, q);
}

template <class R, int D>
__global__ void __launch_bounds__(TileThreads<R>::v) k_diff_div(Args<R> A, R dt) {
    constexpr int P = Pad<D>::v;
    extern __shared__ __align__(16) unsigned char smem[];
    R *sX = reinterpret_cast<R *>(smem);
    R *sQ = reinterpret_cast<R *>(smem + second_off<R, P>(A.max_halo));
    stage_halo<R, P, P>(A, sX, sQ, A.qflux);
    const long long t = blockIdx.x;
    const long long i = t * A.T + threadIdx.x;
    if (i >= A.n) return;
    if (A.flags[i] & kCHeldBit) {
        A.c_tmp[i] = A.c_held[i];
        return;
    }
    const int li = A.lself[i];
    R xa[P], qa[P];
    ld_vec<R, P>(xa, sX + li * P);
    ld_vec<R, P>(qa, sQ + li * P);
    R s = R(0);
    const uint16_t *row = A.lell + A.lell_off[t] + threadIdx.x;
    for_each_neighbour(row, A.T, A.tile_w[t], [&](int l) {
        R xb[P], qb[P];
        ld_vec<R, P>(xb, sX + l * P);
        ld_vec<R, P>(qb, sQ + l * P);
        R d[D], r2 = R(0);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            d[k] = xa[k] - xb[k];
            r2 += d[k] * d[k];
        }
        const R tt = R(1) - R(0.5) * nsqrt(r2) * A.inv_h;
        const R f = A.kcoef * tt * tt * tt;
        R dot = R(0);
#pragma unroll
        for (int k = 0; k < D; ++k) dot += (qa[k] + qb[k]) * d[k];
        s += f * dot;
    });
    A.c_tmp[i] = A.c[i] - dt * s;
}

// Gershgorin bound of the two-stage operator (see the oracle): R_x =
// 2 D |J_x| |C_x^-1 B0_x^T|_inf s1_x with s1_x = sum_b V |grad0 W_xb|_1, then
// max over rows of sum_b V |grad0 W_ab|_1 (R_a + R_b)
template <class R, int D>
__global__ void __launch_bounds__(TileThreads<R>::v) k_ts_rowcoef(Args<R> A, double *Rx) {
    constexpr int P = Pad<D>::v;
    extern __shared__ __align__(16) unsigned char smem[];
    R *sX = reinterpret_cast<R *>(smem);
    R *sU = reinterpret_cast<R *>(smem + second_off<R, P>(A.max_halo));
    stage_halo<R, P, P>(A, sX, sU, A.uf);
    const long long t = blockIdx.x;
    const long long i = t * A.T + threadIdx.x;
    if (i >= A.n) return;
    R F[3][3];
    compute_F<R, D>(A, sX, sU, i, F);
    const int li = A.lself[i];
    R xa[P];
    ld_vec<R, P>(xa, sX + li * P);
    double s1 = 0.0;
    const uint16_t *row = A.lell + A.lell_off[t] + threadIdx.x;
    for_each_neighbour(row, A.T, A.tile_w[t], [&](int l) {
        R xb[P];
        ld_vec<R, P>(xb, sX + l * P);
        R d[D], r2 = R(0), n1 = R(0);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            d[k] = xa[k] - xb[k];
            r2 += d[k] * d[k];
            n1 += (d[k] < R(0) ? -d[k] : d[k]) * (A.aniso ? A.detS * A.sk[k] : R(1));
        }
        const R tt = R(1) - R(0.5) * nsqrt(r2) * A.inv_h;
        const R f = A.kcoef * tt * tt * tt;
        s1 += (double)(f < R(0) ? -f : f) * (double)n1;
    });
    unscale_F<R, D>(A, F);
    R B[D][D];
    ldg_mat<R, D>(B, A.B0 + i * MatS<D>::v);
    R Ci[3][3], J;
    inv_cauchy_green<R, D>(F, Ci, J);
    // real B0^T = diag(s) B0~^T diag(1/s) / detS; real |grad W|_1 = detS sum s_k |grad~_k|
    double nrm = 0.0;
#pragma unroll
    for (int r = 0; r < D; ++r) {
        double rs = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            double m = 0.0;
#pragma unroll
            for (int q = 0; q < D; ++q)
                m += (double)Ci[r][q] * (double)B[k][q] *
                     (A.aniso ? (double)A.sk[q] / ((double)A.sk[k] * (double)A.detS) : 1.0);
            rs += fabs(m);
        }
        nrm = fmax(nrm, rs);
    }
    Rx[i] = 2.0 * (double)A.diffD * fabs((double)J) * nrm * s1;
}

template <class R, int D>
__global__ void __launch_bounds__(TileThreads<R>::v) k_ts_bound(Args<R> A, const double *Rx, double *part) {
    constexpr int P = Pad<D>::v;
    extern __shared__ __align__(16) unsigned char smem[];
    R *sX = reinterpret_cast<R *>(smem);
    double *sR = reinterpret_cast<double *>(smem + second_off<R, P>(A.max_halo));
    stage_halo<R, P, P>(A, sX, nullptr, (const R *)nullptr);
    const long long t = blockIdx.x;
    const long long h0 = A.halo_off[t];
    const int nh = (int)(A.halo_off[t + 1] - h0);
    for (int k = threadIdx.x; k < nh; k += blockDim.x) sR[k] = Rx[__ldg(A.halo_idx + h0 + k)];
    __syncthreads();
    const long long i = t * A.T + threadIdx.x;
    double rowsum = 0.0;
    if (i < A.n) {
        const int li = A.lself[i];
        R xa[P];
        ld_vec<R, P>(xa, sX + li * P);
        const double ra = sR[li];
        const uint16_t *row = A.lell + A.lell_off[t] + threadIdx.x;
        for_each_neighbour(row, A.T, A.tile_w[t], [&](int l) {
            R xb[P];
            ld_vec<R, P>(xb, sX + l * P);
            R d[D], r2 = R(0), n1 = R(0);
#pragma unroll
            for (int k = 0; k < D; ++k) {
                d[k] = xa[k] - xb[k];
                r2 += d[k] * d[k];
                n1 += (d[k] < R(0) ? -d[k] : d[k]) * (A.aniso ? A.detS * A.sk[k] : R(1));
            }
            const R tt = R(1) - R(0.5) * nsqrt(r2) * A.inv_h;
            const R f = A.kcoef * tt * tt * tt;
            rowsum += (double)(f < R(0) ? -f : f) * (double)n1 * (ra + sR[l]);
        });
    }
    rowsum = warp_max(rowsum);
    __shared__ double sh[TileThreads<R>::v / 32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = rowsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) m = fmax(m, sh[q]);
        part[blockIdx.x] = m;
    }
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
__global__ void __launch_bounds__(TileThreads<R>::v) k_defgrad(Args<R> A, double *out) {
    constexpr int P = Pad<D>::v;
    extern __shared__ __align__(16) unsigned char smem[];
    R *sX = reinterpret_cast<R *>(smem);
    R *sU = reinterpret_cast<R *>(smem + second_off<R, P>(A.max_halo));
    stage_halo<R, P, P>(A, sX, sU, A.uf);
    const long long i = blockIdx.x * (long long)A.T + threadIdx.x;
    if (i >= A.n) return;
    R F[3][3];
    compute_F<R, D>(A, sX, sU, i, F);
    unscale_F<R, D>(A, F);
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
    case MTS_F_X:
        for (int k = 0; k < D; ++k) out[i * D + k] = X64[s * P + k] / (A.aniso ? (double)A.sk[k] : 1.0);
        break;
    case MTS_F_V: for (int k = 0; k < D; ++k) out[i * D + k] = (double)A.v[s * P + k]; break;
    case MTS_F_ACC: for (int k = 0; k < D; ++k) out[i * D + k] = (double)A.acc[s * P + k]; break;
    case MTS_F_PB:
        for (int r = 0; r < D; ++r)
            for (int c = 0; c < D; ++c)
                out[i * D * D + r * D + c] =
                    (double)A.PB[s * MatS<D>::v + (D == 3 ? 3 + 3 * r + c : r * P + c)] /
                    (A.aniso ? (double)A.detS * (double)A.sk[c] : 1.0);
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

// all partials summed by one block: strided per thread, then a fixed tree
__global__ void __launch_bounds__(kBlock) k_tip_final(const double *part, int nblk, double *out) {
    __shared__ double red[4][kBlock];
    double s[4] = {0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblk; b += kBlock)
        for (int k = 0; k < 4; ++k) s[k] += part[b * 4 + k];
    for (int k = 0; k < 4; ++k) red[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int w = kBlock / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < 4; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) out[k] = red[3][0] > 0 ? red[k][0] / red[3][0] : 0.0;
}

// --------------------------------------------------------------------- args
}  // namespace

template <class R>
Args<R> make_args(mts_body *b) {
    Args<R> A{};
    A.n = b->n;
    A.dim = b->dim;
    A.T = b->T;
    A.ntiles = b->ntiles;
    A.max_halo = b->max_halo;
    A.halo_off = b->halo_off;
    A.halo_idx = b->halo_idx;
    A.halo_x = (const R *)b->halo_x;
    A.lself = b->lself;
    A.lell = b->lell;
    A.lell_off = b->lell_off;
    A.tile_w = b->tile_w;
    A.max_group_pairs = b->max_group_pairs;
    A.max_group_levels = b->max_group_levels;
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
    A.diffD = (R)b->D;
    A.qflux = (R *)b->qflux;
    A.aniso = b->aniso;
    for (int k = 0; k < 3; ++k) A.sk[k] = (R)b->sk[k];
    A.detS = (R)b->detS;
    A.mass = b->rho0 * b->V;
    A.h = b->h;
    A.cs = std::sqrt(b->K / b->rho0);
    A.eta = (R)b->eta;
    A.pair_ab = b->kpad_ab;
    A.pair_g = (const R *)b->kpad_g;
    A.lvl_pair = b->lvl_pair;
    A.grp_lvl = b->grp_lvl;
    A.grp_cons = b->grp_cons;
    A.touch_start = b->touch_start;
    A.touch_cnt = b->touch_cnt;
    A.bperm = b->bperm;
    A.bflags = b->bflags;
    A.mb = b->mb;
    A.nbw = b->nbw;
    A.max_level_pairs = b->max_level_pairs;
    A.cond = b->cond;
    A.use_cond = b->use_cond;
    A.ctrl = b->ctrl;
    A.part_force = b->part_force;
    A.part_drift = b->part_drift;
    return A;
}

template Args<float> make_args<float>(mts_body *b);
template Args<double> make_args<double>(mts_body *b);

namespace {

template <class R, int D> size_t smem_stress(const mts_body *b) {
    return second_off<R, Pad<D>::v>(b->max_halo) + (size_t)b->max_halo * Pad<D>::v * sizeof(R);
}
template <class R, int D> size_t smem_force(const mts_body *b) {
    if (D == 3) return (size_t)b->max_halo * 12 * sizeof(R);
    return second_off<R, Pad<D>::v>(b->max_halo) + (size_t)b->max_halo * MatS<D>::v * sizeof(R);
}
template <class R, int D> size_t smem_diffuse(const mts_body *b) {
    return second_off<R, Pad<D>::v>(b->max_halo) + (size_t)b->max_halo * sizeof(R);
}
// damping warps (owner groups) per CTA: the requested count, or 4, reduced
// while the CTA's staging does not fit the shared-memory budget
template <class R, int D> int damp_warps(const mts_body *b) {
    const size_t per = DampSmem<R, D>::bytes(b->mb, b->max_group_levels, b->damp_ring);
    int w = b->damp_warps_req > 0 ? b->damp_warps_req : 4;
    while (w > 1 && per * w > 200 * 1024) w >>= 1;
    return w;
}
template <class R, int D> size_t smem_damp(const mts_body *b) {
    return DampSmem<R, D>::bytes(b->mb, b->max_group_levels, b->damp_ring) * damp_warps<R, D>(b);
}

// Launch a kernel of the substep chain.  While a body captures its chain
// (pdl_now), the launch allows programmatic dependent launch: the kernel's
// blocks may be scheduled while the previous kernel drains and run their
// set-up-data prologue; chain_wait() in the kernel orders everything else.
template <typename... KP, typename... AP>
cudaError_t launch_chain(mts_body *b, void (*k)(KP...), unsigned grid, unsigned block,
                         size_t smem, AP &&...args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = b->ctx->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = b->pdl_now ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, std::forward<AP>(args)...);
}

template <class R, int D>
mts_status stress_t(mts_body *b) {
    Args<R> A = make_args<R>(b);
    const size_t sm = smem_stress<R, D>(b);
    if (b->model == MTS_NEOHOOKE_J2)
        k_stress<R, D, MTS_NEOHOOKE_J2><<<(unsigned)b->ntiles, b->T, sm, b->ctx->stream>>>(A);
    else
        k_stress<R, D, MTS_ELASTIC_SVK><<<(unsigned)b->ntiles, b->T, sm, b->ctx->stream>>>(A);
    MTS_CUDA(cudaGetLastError());
    return MTS_OK;
}

template <class R, int D>
mts_status force_t(mts_body *b) {
    MTS_CUDA(launch_chain(b, k_force<R, D>, (unsigned)b->ntiles, (unsigned)b->T,
                          smem_force<R, D>(b), make_args<R>(b)));
    return MTS_OK;
}

// Task tables of the one-launch sweep: the colour launches of the multi-launch
// form in their order, each group of a launch one task; per task and touched
// block, the number of earlier tasks that touch that block.
mts_status build_persist_tables(mts_body *b) {
    const int NB = 1 << b->dim;
    const long long ng = b->n_groups;
    cudaStream_t st = b->ctx->stream;
    std::vector<int32_t> ts((size_t)ng * NB), tc((size_t)ng * NB);
    MTS_CUDA(cudaMemcpyAsync(ts.data(), b->touch_start, ts.size() * 4, cudaMemcpyDeviceToHost, st));
    MTS_CUDA(cudaMemcpyAsync(tc.data(), b->touch_cnt, tc.size() * 4, cudaMemcpyDeviceToHost, st));
    MTS_CUDA(cudaStreamSynchronize(st));
    // a touched block is known by its first particle
    std::vector<int32_t> starts;
    for (size_t q = 0; q < ts.size(); ++q)
        if (tc[q] > 0) starts.push_back(ts[q]);
    std::sort(starts.begin(), starts.end());
    starts.erase(std::unique(starts.begin(), starts.end()), starts.end());
    std::vector<int32_t> blk(ts.size(), -1);
    for (size_t q = 0; q < ts.size(); ++q)
        if (tc[q] > 0)
            blk[q] = (int32_t)(std::lower_bound(starts.begin(), starts.end(), ts[q]) - starts.begin());
    int cols[8], nc = 0;
    for (int c = 0; c < NB; ++c)
        if (b->col_off[c + 1] > b->col_off[c]) cols[nc++] = c;
    int pcol[16], pmode[16], nph = 0;
    for (int i = 0; i < nc - 1; ++i) { pcol[nph] = cols[i]; pmode[nph++] = 1; }
    if (nc > 0) { pcol[nph] = cols[nc - 1]; pmode[nph++] = 3; }
    for (int i = nc - 2; i >= 0; --i) { pcol[nph] = cols[i]; pmode[nph++] = 2; }
    long long ntasks = 0;
    for (int p = 0; p < nph; ++p) {
        b->pd_off[p] = ntasks;
        b->pd_goff[p] = b->col_off[pcol[p]];
        b->pd_mode[p] = pmode[p];
        ntasks += b->col_off[pcol[p] + 1] - b->col_off[pcol[p]];
    }
    b->pd_off[nph] = ntasks;
    std::vector<uint8_t> req((size_t)ntasks * NB, 0);
    std::vector<int> cnt(starts.size(), 0);
    for (int p = 0; p < nph; ++p)
        for (long long t = b->pd_off[p]; t < b->pd_off[p + 1]; ++t) {
            const long long g = b->pd_goff[p] + (t - b->pd_off[p]);
            for (int e = 0; e < NB; ++e) {
                const int32_t k = blk[g * NB + e];
                if (k < 0) continue;
                if (cnt[k] > 255) {
                    set_error("one-launch damping: a block is touched by more than 255 tasks");
                    return MTS_ERR_STATE;
                }
                req[t * NB + e] = (uint8_t)cnt[k]++;   // a launch touches a block at most once
            }
        }
    MTS_TRY(dalloc_t(b->ctx, &b->pd_blk, blk.size()));
    MTS_TRY(dalloc_t(b->ctx, &b->pd_req, std::max<size_t>(req.size(), 1)));
    MTS_TRY(dalloc_t(b->ctx, &b->pd_done, starts.size() + 1));
    MTS_CUDA(cudaMemcpyAsync(b->pd_blk, blk.data(), blk.size() * 4, cudaMemcpyHostToDevice, st));
    if (!req.empty())
        MTS_CUDA(cudaMemcpyAsync(b->pd_req, req.data(), req.size(), cudaMemcpyHostToDevice, st));
    MTS_CUDA(cudaMemsetAsync(b->pd_done, 0, (starts.size() + 1) * 4, st));
    MTS_CUDA(cudaStreamSynchronize(st));
    b->pd_ntasks = ntasks;
    b->pd_nblocks = (long long)starts.size();
    b->pd_nph = nph;
    return MTS_OK;
}

template <class R, int D>
mts_status damping_persist(mts_body *b, const Args<R> &A, long long *nlaunch) {
    PersistArgs Q{};
    Q.blk = b->pd_blk;
    Q.req = b->pd_req;
    Q.done = b->pd_done;
    Q.nblocks = b->pd_nblocks;
    Q.ntasks = b->pd_ntasks;
    Q.nph = b->pd_nph;
    for (int p = 0; p <= b->pd_nph; ++p) Q.off[p] = b->pd_off[p];
    for (int p = 0; p < b->pd_nph; ++p) {
        Q.goff[p] = b->pd_goff[p];
        Q.mode[p] = b->pd_mode[p];
    }
    const int W = damp_warps<R, D>(b);
    const size_t smem = smem_damp<R, D>(b);
    MTS_CUDA(launch_chain(b, k_persist_reset, 1u, 256u, (size_t)0, b->pd_done,
                          b->pd_nblocks + 1));
    if (b->damp_ring)
        MTS_CUDA(launch_chain(b, k_damp_persist<R, D, true>, (unsigned)b->pd_grid,
                              (unsigned)(W * 32), smem, A, Q));
    else
        MTS_CUDA(launch_chain(b, k_damp_persist<R, D, false>, (unsigned)b->pd_grid,
                              (unsigned)(W * 32), smem, A, Q));
    if (nlaunch) *nlaunch = 2;
    return MTS_OK;
}

template <class R, int D>
mts_status damping_run(mts_body *b, const Args<R> &A, long long *nlaunch) {
    if (nlaunch) *nlaunch = 0;
    if (b->eta == 0.0 || b->npairs == 0) return MTS_OK;
    if (b->pd_on && !A.transpose && b->damp_layout != MTS_DAMP_WIDE)
        return damping_persist<R, D>(b, A, nlaunch);
    const bool wide = b->damp_layout == MTS_DAMP_WIDE;
    const size_t smem = wide ? damp_wide_smem(b) : smem_damp<R, D>(b);
    const int W = damp_warps<R, D>(b);
    int cols[8], nc = 0;
    for (int c = 0; c < (1 << D); ++c)
        if (b->col_off[c + 1] > b->col_off[c]) cols[nc++] = c;
    // cn: the colour of the next launch (-1: none), whose level slots the
    // warp-per-group kernel prefetches into L2
    auto launch = [&](int c, int mode, int cn) -> mts_status {
        const long long g0 = b->col_off[c], g1 = b->col_off[c + 1];
        if (wide) {
            MTS_CUDA(launch_chain(b, k_damp_wide<R, D>, (unsigned)(g1 - g0), (unsigned)kWideThreads,
                                  smem, A, g0, mode));
        } else {
            const long long n0 = cn >= 0 ? b->col_off[cn] : 0, n1 = cn >= 0 ? b->col_off[cn + 1] : 0;
            const unsigned grid = (unsigned)((g1 - g0 + W - 1) / W);
            if (b->damp_ring)
                MTS_CUDA(launch_chain(b, k_damp<R, D, true>, grid, (unsigned)(W * 32), smem, A, g0,
                                      g1, mode, n0, n1));
            else
                MTS_CUDA(launch_chain(b, k_damp<R, D, false>, grid, (unsigned)(W * 32), smem, A,
                                      g0, g1, mode, n0, n1));
        }
        if (nlaunch) ++*nlaunch;
        return MTS_OK;
    };
    // symmetric sweep over the non-empty colours: forward on all but the
    // last, forward + reverse fused on the last, then reverse
    if (nc == 0) return MTS_OK;
    for (int i = 0; i < nc - 1; ++i) MTS_TRY(launch(cols[i], 1, cols[i + 1]));
    MTS_TRY(launch(cols[nc - 1], 3, nc >= 2 ? cols[nc - 2] : -1));
    for (int i = nc - 2; i >= 0; --i) MTS_TRY(launch(cols[i], 2, i > 0 ? cols[i - 1] : -1));
    return MTS_OK;
}

template <class R, int D>
mts_status damping_t(mts_body *b, long long *nlaunch) {
    return damping_run<R, D>(b, make_args<R>(b), nlaunch);
}

// transposed sweep on an FP64 adjoint velocity array: the same pair order
// (forward then reverse) with every 2x2 pair update transposed
template <class R, int D>
mts_status damping_adjoint_t(mts_body *b, double *vbar, Control *ctrl) {
    if constexpr (sizeof(R) != 8) {
        set_error("the adjoint runs on FP64 bodies only");
        return MTS_ERR_STATE;
    } else {
        Args<R> A = make_args<R>(b);
        A.v = vbar;
        A.ctrl = ctrl;
        A.transpose = 1;
        return damping_run<R, D>(b, A, nullptr);
    }
}

// Raise the dynamic shared-memory cap of the staging kernels (outside any
// stream capture).  The cap is a per-kernel attribute shared by every body in
// the process, so it is set to what the device allows next to the kernel's
// static shared memory, not to this body's need: a later, smaller body must
// not lower it under an earlier body's captured graphs.
template <class R, int D>
mts_status prepare_t(mts_body *b) {
    int optin = 0;
    MTS_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->ctx->device));
    const bool wide = b->damp_layout == MTS_DAMP_WIDE;
    auto attr = [&](const void *fn, size_t need, const char *what) -> mts_status {
        cudaFuncAttributes fa{};
        MTS_CUDA(cudaFuncGetAttributes(&fa, fn));
        const size_t cap = (size_t)optin - fa.sharedSizeBytes;
        if (need > cap) {
            set_error("%s needs %zu bytes of shared memory, at most %zu fit (halo %d particles, "
                      "damping block %d particles)", what, need, cap, b->max_halo, b->mb);
            return MTS_ERR_INVALID_ARG;
        }
        MTS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap));
        return MTS_OK;
    };
    if (wide) {
        MTS_TRY(attr((const void *)k_damp_wide<R, D>, damp_wide_smem(b), "damping (wide)"));
    } else {
        // Level staging: with every level staged a warp needs room for the
        // group's longest chain, which caps the warps per SM; when a colour has
        // more groups than the SMs can then hold at once, the two-chunk ring
        // (a fraction of the shared memory, several times the warps) wins.
        // Compare the rounds of warps a colour launch needs in each form (the
        // ring's warps run a little slower, so it takes strictly fewer rounds).
        int sms = 0;
        MTS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->ctx->device));
        auto rounds = [&](bool ring) {
            const size_t per = DampSmem<R, D>::bytes(b->mb, b->max_group_levels, ring);
            const long long per_sm = std::max<long long>(1, std::min<long long>(32, (long long)(optin / per)));
            long long gmax = 0;
            for (int c = 0; c < (1 << D); ++c)
                gmax = std::max<long long>(gmax, b->col_off[c + 1] - b->col_off[c]);
            return (gmax + sms * per_sm - 1) / (sms * per_sm);
        };
        const long long rounds_ring = rounds(true);
        b->damp_ring = rounds_ring < rounds(false);
        MTS_TRY(attr((const void *)k_damp<R, D, false>,
                     DampSmem<R, D>::bytes(b->mb, b->max_group_levels, false) * damp_warps<R, D>(b),
                     "damping"));
        MTS_TRY(attr((const void *)k_damp<R, D, true>,
                     DampSmem<R, D>::bytes(b->mb, b->max_group_levels, true) * damp_warps<R, D>(b),
                     "damping"));
        // The one-launch form where a colour launch needs several rounds of warps
        // even in the ring form: there it removes the launch boundaries and the
        // tails of each round (the 2.5 M-particle plate, 3 rounds: 1.05 -> 0.85
        // ms per substep).  With one round per launch the chain of dependent
        // tasks is the critical path and separate launches are faster (the
        // 252,800-particle cylinder: 0.18 vs 0.37 ms; a 625,000-particle plate:
        // 0.37 vs 0.60 ms).  MTS_DAMP_MULTILAUNCH=1 keeps the multi-launch form
        // (for comparisons; the results are the same bits).
        const char *ml = std::getenv("MTS_DAMP_MULTILAUNCH");
        const bool want = !(ml && ml[0] == '1') && b->damp_ring && rounds_ring >= 2 &&
                          b->npairs > 0 && b->n_groups > 0;
        if (want && !b->pd_blk) MTS_TRY(build_persist_tables(b));
        b->pd_on = want;
        if (want) {
            MTS_TRY(attr((const void *)k_damp_persist<R, D, false>,
                         DampSmem<R, D>::bytes(b->mb, b->max_group_levels, false) *
                             damp_warps<R, D>(b), "damping (one launch)"));
            MTS_TRY(attr((const void *)k_damp_persist<R, D, true>,
                         DampSmem<R, D>::bytes(b->mb, b->max_group_levels, true) *
                             damp_warps<R, D>(b), "damping (one launch)"));
            const int W = damp_warps<R, D>(b);
            int per_sm = 0;
            if (b->damp_ring)
                MTS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &per_sm, k_damp_persist<R, D, true>, W * 32, smem_damp<R, D>(b)));
            else
                MTS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &per_sm, k_damp_persist<R, D, false>, W * 32, smem_damp<R, D>(b)));
            const long long need = (b->pd_ntasks + W - 1) / W;
            b->pd_grid = (int)std::max<long long>(1, std::min<long long>(need, (long long)std::max(per_sm, 1) * sms));
        }
    }
    const size_t sa = smem_stress<R, D>(b);
    MTS_TRY(attr((const void *)k_stress<R, D, MTS_ELASTIC_SVK>, sa, "stress"));
    MTS_TRY(attr((const void *)k_stress<R, D, MTS_NEOHOOKE_J2>, sa, "stress"));
    MTS_TRY(attr((const void *)k_defgrad<R, D>, sa, "deformation gradient"));
    MTS_TRY(attr((const void *)k_force<R, D>, smem_force<R, D>(b), "force"));
    MTS_TRY(attr((const void *)k_diffuse<R, D>, smem_diffuse<R, D>(b), "diffusion"));
    const size_t sh2 = 2 * second_off<R, Pad<D>::v>(b->max_halo);
    MTS_TRY(attr((const void *)k_diff_flux<R, D>, 3 * second_off<R, Pad<D>::v>(b->max_halo), "diffusion flux"));
    MTS_TRY(attr((const void *)k_diff_div<R, D>, sh2, "diffusion divergence"));
    MTS_TRY(attr((const void *)k_ts_rowcoef<R, D>, sh2, "diffusion bound"));
    MTS_TRY(attr((const void *)k_ts_bound<R, D>,
                 second_off<R, Pad<D>::v>(b->max_halo) + (size_t)b->max_halo * 8, "diffusion bound"));
    return MTS_OK;
}

template <class R, int D>
mts_status drift_t(mts_body *b) {
    if (b->use_cond)
        MTS_CUDA(launch_chain(b, k_drift<R, D, true>, drift_grid(b->n), (unsigned)kBlock, 0,
                              make_args<R>(b)));
    else
        MTS_CUDA(launch_chain(b, k_drift<R, D, false>, drift_grid(b->n), (unsigned)kBlock, 0,
                              make_args<R>(b)));
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
    MTS_TRY((prepare_t<R, D>(b)));
    if (b->diff_mode == 1) {
        const size_t s1 = 3 * second_off<R, Pad<D>::v>(b->max_halo);
        const size_t s2 = 2 * second_off<R, Pad<D>::v>(b->max_halo);
        k_diff_flux<R, D><<<(unsigned)b->ntiles, b->T, s1, b->ctx->stream>>>(A);
        k_diff_div<R, D><<<(unsigned)b->ntiles, b->T, s2, b->ctx->stream>>>(A, (R)dt);
    } else {
        k_diffuse<R, D><<<(unsigned)b->ntiles, b->T, smem_diffuse<R, D>(b), b->ctx->stream>>>(A, (R)dt);
    }
    k_copy<R><<<grid_of(b->n), kBlock, 0, b->ctx->stream>>>((const R *)b->c_tmp, (R *)b->c, b->n);
    MTS_CUDA(cudaGetLastError());
    return MTS_OK;
}

template <class R, int D>
mts_status ts_bound_t(mts_body *b, double *lambda) {
    MTS_TRY((prepare_t<R, D>(b)));
    Args<R> A = make_args<R>(b);
    double *Rx = b->scratch, *part = b->scratch + b->n;
    const size_t s2 = 2 * second_off<R, Pad<D>::v>(b->max_halo);
    const size_t s3 = second_off<R, Pad<D>::v>(b->max_halo) + (size_t)b->max_halo * 8;
    k_ts_rowcoef<R, D><<<(unsigned)b->ntiles, b->T, s2, b->ctx->stream>>>(A, Rx);
    k_ts_bound<R, D><<<(unsigned)b->ntiles, b->T, s3, b->ctx->stream>>>(A, Rx, part);
    MTS_CUDA(cudaGetLastError());
    std::vector<double> h(b->ntiles);
    MTS_CUDA(cudaMemcpyAsync(h.data(), part, b->ntiles * sizeof(double), cudaMemcpyDeviceToHost,
                             b->ctx->stream));
    MTS_CUDA(cudaStreamSynchronize(b->ctx->stream));
    double m = 0;
    for (double x : h) m = std::max(m, x);
    *lambda = m;
    return MTS_OK;
}

template <class R, int D>
mts_status defgrad_t(mts_body *b, double *out_sorted) {
    MTS_TRY((prepare_t<R, D>(b)));
    k_defgrad<R, D><<<(unsigned)b->ntiles, b->T, smem_stress<R, D>(b), b->ctx->stream>>>(
        make_args<R>(b), out_sorted);
    MTS_CUDA(cudaGetLastError());
    return MTS_OK;
}

template <class R, int D>
mts_status field_out_t(mts_body *b, int field) {
    if (field == MTS_F_DEFGRAD) {
        double *tmp = b->scratch + (size_t)b->n * 9;
        MTS_TRY((defgrad_t<R, D>(b, tmp)));
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

int damp_warps_of(const mts_body *b) {
    if (b->precision == MTS_FP64)
        return b->dim == 2 ? damp_warps<double, 2>(b) : damp_warps<double, 3>(b);
    return b->dim == 2 ? damp_warps<float, 2>(b) : damp_warps<float, 3>(b);
}
mts_status launch_stress(mts_body *b) { return DISPATCH(stress_t, b); }
mts_status launch_force(mts_body *b) { return DISPATCH(force_t, b); }
mts_status launch_damping(mts_body *b, long long *launches) { return DISPATCH(damping_t, b, launches); }
mts_status launch_damping_adjoint(mts_body *b, double *vbar, Control *ctrl) {
    return DISPATCH(damping_adjoint_t, b, vbar, ctrl);
}
mts_status launch_drift(mts_body *b) { return DISPATCH(drift_t, b); }
mts_status prepare_kernels(mts_body *b) { return DISPATCH(prepare_t, b); }

size_t damp_wide_smem(const mts_body *b) {
    size_t off[4], total = 0;
    wide_offsets(b->nbw * b->mb, b->max_group_levels, b->max_level_pairs, b->dim == 2 ? 2 : 4,
                 (int)b->rsize, off, &total);
    return total;
}

mts_status update_pair_fixbits(mts_body *b) {
    if (b->grp_cons && b->n_groups > 0)
        k_group_cons<<<(unsigned)((b->n_groups + 255) / 256), 256, 0, b->ctx->stream>>>(
            b->touch_start, b->touch_cnt, b->n_groups, 1 << b->dim, b->flags, (1 << b->dim) - 1,
            b->grp_cons);
    if (b->grp_cons && b->npairs > 0)
        k_pair_fixword<<<(unsigned)((b->npairs + 255) / 256), 256, 0, b->ctx->stream>>>(
            b->kpad_ab, b->pair_slot, b->pair_a, b->pair_b, b->npairs, b->flags,
            (1 << b->dim) - 1);
    if (b->bflags)
        k_gather_flags<<<(unsigned)((b->n + 255) / 256), 256, 0, b->ctx->stream>>>(
            b->flags, b->bperm, b->n, b->bflags);
    if (b->npairs == 0) return MTS_OK;
    const unsigned grid = (unsigned)((b->npairs + 255) / 256);
    if (b->precision == MTS_FP64)
        k_pair_fixsign<double><<<grid, 256, 0, b->ctx->stream>>>(
            (double *)b->kpad_g, b->pair_slot, b->pair_a, b->pair_b, b->npairs, b->flags,
            (1 << b->dim) - 1);
    else
        k_pair_fixsign<float><<<grid, 256, 0, b->ctx->stream>>>(
            (float *)b->kpad_g, b->pair_slot, b->pair_a, b->pair_b, b->npairs, b->flags,
            (1 << b->dim) - 1);
    MTS_CUDA(cudaGetLastError());
    return MTS_OK;
}
mts_status launch_slow_begin(mts_body *b) { return DISPATCH(load_t, b); }
mts_status launch_diffusion(mts_body *b, double dt) { return DISPATCH(diffuse_t, b, dt); }
mts_status diffusion_bound_two_stage(mts_body *b, double *lambda) { return DISPATCH(ts_bound_t, b, lambda); }
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
    k_tip_final<<<1, kBlock, 0, b->ctx->stream>>>(part, (int)g, part + (size_t)g * 4);
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
