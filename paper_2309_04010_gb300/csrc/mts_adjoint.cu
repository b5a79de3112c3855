// mts_adjoint.cu -- reverse mode of the slow step (FP64 arithmetic; a mixed-
// precision body is reversed on its FP64 twin about its own taped states).
//
// With its substep sizes and count held at the values of the forward run, a
// slow step (Sec. 4.2) is a fixed composition of maps on the state (u, v,
// C-bar_p^-1, alpha, c): the load jump, the diffusion step, then per substep
// F and stress (Sec. 2.1, 3.1, App. A Alg. 1, App. B.2), force and kick
// (Sec. 3.1), the pairwise damping sweep (Sec. 4.3), BC and drift.  The
// adjoint applies the transposes of these maps in reverse order to an adjoint
// state and accumulates the derivatives with respect to the parameters
// (E, sigma_0, sigma_inf, delta, H, D, beta).  With g_ab = V grad_a W_ab
// (antisymmetric in a, b on symmetric neighbour lists) the transposes are:
//   drift    v-bar += dt u-bar on free axes; u-bar = v-bar = 0 on prescribed axes
//   damping  the same sequence of pair updates, each 2x2 update transposed
//   kick     a-bar = dt v-bar on free axes, plus the end-force adjoint
//   force    (P B0^T)-bar_c = -(1/rho0) sum_b (a-bar_b - a-bar_c) (x) g_cb
//   P B0^T   P-bar = (P B0^T)-bar B0
//   stress   one reverse sweep through the constitutive law (mts_vjp.cuh)
//            from the output adjoints (P, C-bar_p^-1', alpha')
//   F        G-bar = F-bar B0^T;  u-bar_c -= sum_b (G-bar_c + G-bar_b) g_cb
//   diffusion  y = c-bar on free-c particles; c-bar = y + dt L(y), L the
//            pairwise Laplacian of the forward step; D-bar from c before it
// The force and F transposes are the F and force gathers of the forward pass
// with the roles of the arrays exchanged, on the same Morton tiles.
#include <cmath>

#include "mts_device.cuh"
#include "mts_vjp.cuh"
#include "mts_internal.cuh"
#include "mts_tiles.cuh"

namespace mts {

namespace {

constexpr int kTh = 8;          // parameter slots: E, s0, sinf, delta, H, D, beta, (spare)

inline unsigned grid_n(long long n) { return (unsigned)((n + kBlock - 1) / kBlock); }

// cp: the plastic state in the forward body's storage precision (a mixed-
// precision body's is FP32; the tape is FP64 either way)
template <class R>
__global__ void k_tape(const double *u, const R *cp, const Control *C, long long n, int pad,
                       long long k, double *tape_u, double *tape_cp, double *tape_dt) {
    const long long i = blockIdx.x * (long long)kBlock + threadIdx.x;
    if (i == 0) tape_dt[k] = C->dt;
    if (i >= n) return;
    for (int q = 0; q < pad; ++q) tape_u[k * n * pad + i * pad + q] = u[i * pad + q];
    for (int q = 0; q < 8; ++q) tape_cp[k * n * 8 + i * 8 + q] = (double)cp[i * 8 + q];
}

template <class R>
__global__ void k_to_double(const R *x, long long n, double *y) {
    const long long i = blockIdx.x * (long long)kBlock + threadIdx.x;
    if (i < n) y[i] = (double)x[i];
}

__global__ void k_adj_setdt(Control *C, const double *tape_dt, long long k) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        C->dt = tape_dt[k];
        C->done = 0;
    }
}

// BC + drift transposed
template <int D>
__global__ void k_adj_drift(const uint8_t *flags, long long n, const Control *C, double *au,
                            double *av) {
    constexpr int P = Pad<D>::v;
    const long long i = blockIdx.x * (long long)kBlock + threadIdx.x;
    if (i >= n) return;
    const double dt = C->dt;
    const uint8_t fx = flags[i];
#pragma unroll
    for (int q = 0; q < D; ++q) {
        if ((fx >> q) & 1) {
            au[i * P + q] = 0.0;
            av[i * P + q] = 0.0;
        } else {
            av[i * P + q] += dt * au[i * P + q];
        }
    }
}

// kick transposed; the end force -sum m a over the force set enters at the
// last substep
template <int D>
__global__ void k_adj_kick(const uint8_t *flags, long long n, const Control *C, double mass,
                           const double *av, double *aa, double f0, double f1, double f2,
                           int last) {
    constexpr int P = Pad<D>::v;
    const long long i = blockIdx.x * (long long)kBlock + threadIdx.x;
    if (i >= n) return;
    const double dt = C->dt;
    const uint8_t fx = flags[i];
    const double fs[3] = {f0, f1, f2};
#pragma unroll
    for (int q = 0; q < P; ++q) {
        double a = 0.0;
        if (q < D) {
            if (!((fx >> q) & 1)) a = dt * av[i * P + q];
            if (last && (fx & kForceBit)) a -= mass * fs[q];
        }
        aa[i * P + q] = a;
    }
}

// sum over neighbours b of (y_b - y_a) (x) g_ab for a staged vector field y
template <int D>
__device__ __forceinline__ void gather_grad(const Args<double> &A, const double *sX, const double *sY,
                                            long long i, double (&G)[D][D]) {
    constexpr int P = Pad<D>::v;
    const long long t = blockIdx.x;
    const int li = A.lself[i];
    double xa[P], ya[P];
    ld_vec<double, P>(xa, sX + li * P);
    ld_vec<double, P>(ya, sY + li * P);
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) G[r][c] = 0.0;
    const uint16_t *row = A.lell + A.lell_off[t] + threadIdx.x;
    const int w = A.tile_w[t];
    for_each_neighbour(row, A.T, w, [&](int l) {
        double xb[P], yb[P];
        ld_vec<double, P>(xb, sX + l * P);
        ld_vec<double, P>(yb, sY + l * P);
        double d[D], r2 = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            d[k] = xa[k] - xb[k];
            r2 += d[k] * d[k];
        }
        const double tt = 1.0 - 0.5 * sqrt(r2) * A.inv_h;
        const double f = A.kcoef * tt * tt * tt;   // V W'(r)/r
#pragma unroll
        for (int r = 0; r < D; ++r) {
            const double dy = (yb[r] - ya[r]) * f;
#pragma unroll
            for (int c = 0; c < D; ++c) G[r][c] += dy * d[c];
        }
    });
}

// Jacobian-transpose product of the stress law at one particle: inputs F
// (d x d free entries), C-bar_p^-1 and alpha (J2), c, and the parameters
// (E, then sigma_0, sigma_inf, delta, H for J2, then beta); outputs P (3x3),
// C-bar_p^-1' and alpha'.  yb = output adjoints (P row-major, then the
// plastic state); xb = input adjoints in the order above.
template <int D, int MAT>
struct StressDirs {
    static constexpr int nF = D * D;
    static constexpr int nCp = MAT == MTS_NEOHOOKE_J2 ? 7 : 0;
    static constexpr int iC = nF + nCp;
    static constexpr int iE = iC + 1;
    static constexpr int iHard = iE + 1;                       // s0, sinf, delta, H (J2)
    static constexpr int iBeta = iHard + (MAT == MTS_NEOHOOKE_J2 ? 4 : 0);
    static constexpr int n = iBeta + 1;
};

template <int D, int MAT>
__device__ void stress_vjp(const Args<double> &A, const double (&F)[3][3], const double (&cp)[7],
                           double c, double beta, double dK, double dmu, const double (&yb)[16],
                           double (&xb)[StressDirs<D, MAT>::n]) {
    using S = StressDirs<D, MAT>;
    const double K = (double)A.K, mu = (double)A.mu;
    double Pb[3][3], Fbar[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            Pb[r][q] = yb[r * 3 + q];
            Fbar[r][q] = 0.0;
        }
    LawBar lb{0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    double cpb_in[7] = {0, 0, 0, 0, 0, 0, 0};
    if constexpr (MAT == MTS_NEOHOOKE_J2) {
        const double cpb_out[7] = {yb[9], yb[10], yb[11], yb[12], yb[13], yb[14], yb[15]};
        stress_j2_vjp(F, cp, K, mu, (double)A.s0, (double)A.sinf, (double)A.delta,
                      (double)A.Hlin, Pb, cpb_out, Fbar, cpb_in, lb);
    } else {
        stress_svk_vjp(F, K - mu * (2.0 / 3.0), mu, Pb, Fbar, lb);
    }
    double cb = 0.0, betab = 0.0;
    if (A.swelling) {
        // P -= p cof(F), p = 3 K beta (c - c0)
        const double dc = c - (double)A.c0;
        const double p = 3.0 * K * beta * dc;
        double Cf[3][3], mPb[3][3], pbar = 0.0;
        m3_cof(F, Cf);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                pbar -= Pb[r][q] * Cf[r][q];
                mPb[r][q] = -p * Pb[r][q];
            }
        cof_vjp(F, mPb, Fbar);
        lb.K += pbar * 3.0 * beta * dc;
        betab = pbar * 3.0 * K * dc;
        cb = pbar * 3.0 * K * beta;
    }
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int q = 0; q < D; ++q) xb[r * D + q] = Fbar[r][q];
    if constexpr (MAT == MTS_NEOHOOKE_J2) {
#pragma unroll
        for (int k = 0; k < 7; ++k) xb[S::nF + k] = cpb_in[k];
        xb[S::iHard] = lb.s0;
        xb[S::iHard + 1] = lb.sinf;
        xb[S::iHard + 2] = lb.delta;
        xb[S::iHard + 3] = lb.H;
    }
    xb[S::iC] = cb;
    xb[S::iE] = lb.K * dK + lb.mu * dmu;
    xb[S::iBeta] = betab;
}

// force transposed + P B0 transposed + stress transposed, at substep k of the
// tape: one Morton tile per CTA, halo X, a-bar and u_k staged
template <int D, int MAT>
__global__ void __launch_bounds__(128) k_adj_stress(Args<double> A, const double *aa,
                                                    const double *tu, const double *tcp,
                                                    double *acp, double *ac, double *aG,
                                                    double *part, double beta, double dK,
                                                    double dmu) {
    constexpr int P = Pad<D>::v;
    constexpr int MS = MatS<D>::v;
    using S = StressDirs<D, MAT>;
    extern __shared__ __align__(16) unsigned char smem[];
    const size_t o1 = second_off<double, P>(A.max_halo);
    double *sX = reinterpret_cast<double *>(smem);
    double *sA = reinterpret_cast<double *>(smem + o1);
    double *sU = reinterpret_cast<double *>(smem + 2 * o1);
    stage_halo<double, P, P>(A, sX, sA, aa);
    stage_halo<double, P, P>(A, nullptr, sU, tu);
    const long long i = blockIdx.x * (long long)A.T + threadIdx.x;
    double th[6] = {0, 0, 0, 0, 0, 0};   // E, s0, sinf, delta, H, beta
    if (i < A.n) {
        double B[D][D];
        ldg_mat<double, D>(B, A.B0 + i * MS);
        double Ga[D][D], Gu[D][D];
        gather_grad<D>(A, sX, sA, i, Ga);
        gather_grad<D>(A, sX, sU, i, Gu);
        double F[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int q = 0; q < 3; ++q) F[r][q] = r == q ? 1.0 : 0.0;
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
            for (int q = 0; q < D; ++q) {
                double s = 0.0;
#pragma unroll
                for (int k = 0; k < D; ++k) s += Gu[r][k] * B[k][q];
                F[r][q] += s;
            }
        // P-bar = (P B0^T)-bar B0 with (P B0^T)-bar = -(1/rho0) G[a-bar]
        double yb[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) yb[k] = 0.0;
        const double irho = -(double)A.inv_rho0;
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
            for (int q = 0; q < D; ++q) {
                double s = 0.0;
#pragma unroll
                for (int k = 0; k < D; ++k) s += Ga[r][k] * B[k][q];
                yb[r * 3 + q] = irho * s;
            }
        double cp7[7];
#pragma unroll
        for (int k = 0; k < 7; ++k) cp7[k] = tcp[i * 8 + k];
        if constexpr (MAT == MTS_NEOHOOKE_J2) {
#pragma unroll
            for (int k = 0; k < 7; ++k) yb[9 + k] = acp[i * 8 + k];
        }
        double xb[S::n];
        stress_vjp<D, MAT>(A, F, cp7, (double)A.c[i], beta, dK, dmu, yb, xb);
        // G-bar = F-bar B0^T
        double *g = aG + i * MS;
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
            for (int q = 0; q < D; ++q) {
                double s = 0.0;
#pragma unroll
                for (int k = 0; k < D; ++k) s += xb[r * D + k] * B[q][k];
                g[r * P + q] = s;
            }
        if constexpr (MAT == MTS_NEOHOOKE_J2) {
#pragma unroll
            for (int k = 0; k < 7; ++k) acp[i * 8 + k] = xb[S::nF + k];
        }
        ac[i] += xb[S::iC];
        th[0] = xb[S::iE];
        if constexpr (MAT == MTS_NEOHOOKE_J2) {
#pragma unroll
            for (int k = 0; k < 4; ++k) th[1 + k] = xb[S::iHard + k];
        }
        th[5] = xb[S::iBeta];
    }
    // tile partials (fixed tree order)
    __shared__ double sh[6][4];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const double v = warp_sum(th[k]);
        if (lane == 0) sh[k][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (int)(blockDim.x >> 5);
        double s[6] = {0, 0, 0, 0, 0, 0};
        for (int q = 0; q < nw; ++q)
            for (int k = 0; k < 6; ++k) s[k] += sh[k][q];
        double *o = part + blockIdx.x * kTh;
        o[0] = s[0]; o[1] = s[1]; o[2] = s[2]; o[3] = s[3]; o[4] = s[4]; o[6] = s[5];
        o[5] = 0.0; o[7] = 0.0;
    }
}

// F transposed: u-bar_c -= sum_b (G-bar_c + G-bar_b) g_cb
template <int D>
__global__ void __launch_bounds__(128) k_adj_grad(Args<double> A, const double *aG, double *au) {
    constexpr int P = Pad<D>::v;
    constexpr int MS = MatS<D>::v;
    extern __shared__ __align__(16) unsigned char smem[];
    double *sX = reinterpret_cast<double *>(smem);
    double *sG = reinterpret_cast<double *>(smem + second_off<double, P>(A.max_halo));
    stage_halo<double, P, MS>(A, sX, sG, aG);
    const long long t = blockIdx.x;
    const long long i = t * A.T + threadIdx.x;
    if (i >= A.n) return;
    const int li = A.lself[i];
    double xa[P];
    ld_vec<double, P>(xa, sX + li * P);
    double Ga[D][D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int q = 0; q < D; ++q) Ga[r][q] = sG[li * MS + r * P + q];
    double s[D];
#pragma unroll
    for (int r = 0; r < D; ++r) s[r] = 0.0;
    const uint16_t *row = A.lell + A.lell_off[t] + threadIdx.x;
    const int w = A.tile_w[t];
    for_each_neighbour(row, A.T, w, [&](int l) {
        double xb[P];
        ld_vec<double, P>(xb, sX + l * P);
        double d[D], r2 = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            d[k] = xa[k] - xb[k];
            r2 += d[k] * d[k];
        }
        const double tt = 1.0 - 0.5 * sqrt(r2) * A.inv_h;
        const double f = A.kcoef * tt * tt * tt;
#pragma unroll
        for (int r = 0; r < D; ++r) {
            double acc = 0.0;
#pragma unroll
            for (int q = 0; q < D; ++q) acc += (Ga[r][q] + sG[l * MS + r * P + q]) * d[q];
            s[r] += f * acc;
        }
    });
#pragma unroll
    for (int r = 0; r < D; ++r) au[i * P + r] -= s[r];
}

// sum the tile partials into the accumulators, in tile order
__global__ void k_adj_theta(const double *part, long long ntiles, double *acc) {
    __shared__ double red[kTh][256];
    double s[kTh];
    for (int k = 0; k < kTh; ++k) s[k] = 0.0;
    for (long long t = threadIdx.x; t < ntiles; t += blockDim.x)
        for (int k = 0; k < kTh; ++k) s[k] += part[t * kTh + k];
    for (int k = 0; k < kTh; ++k) red[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < kTh; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < kTh) acc[threadIdx.x] += red[threadIdx.x][0];
}

__global__ void k_adj_free_c(const uint8_t *flags, long long n, const double *ac, double *y) {
    const long long i = blockIdx.x * (long long)kBlock + threadIdx.x;
    if (i < n) y[i] = (flags[i] & kCHeldBit) ? 0.0 : ac[i];
}

// diffusion transposed: c-bar = y + dt L(y); D-bar = sum y dt L(c_before) / D
template <int D>
__global__ void __launch_bounds__(128) k_adj_diffuse(Args<double> A, const double *y,
                                                     const double *cpre, double dt, double invD,
                                                     double *ac, double *part) {
    constexpr int P = Pad<D>::v;
    extern __shared__ __align__(16) unsigned char smem[];
    const size_t o1 = second_off<double, P>(A.max_halo);
    double *sX = reinterpret_cast<double *>(smem);
    double *sY = reinterpret_cast<double *>(smem + o1);
    double *sC = sY + A.max_halo;
    const long long t = blockIdx.x;
    const long long h0 = A.halo_off[t];
    const int nh = (int)(A.halo_off[t + 1] - h0);
    for (int k = threadIdx.x; k < nh; k += blockDim.x) {
        const long long g = __ldg(A.halo_idx + h0 + k);
        double x[P];
        ldg_vec<double, P>(x, A.halo_x + (h0 + k) * P);
        st_vec<double, P>(sX + k * P, x);
        sY[k] = y[g];
        sC[k] = cpre[g];
    }
    __syncthreads();
    const long long i = t * A.T + threadIdx.x;
    double dpart = 0.0;
    if (i < A.n) {
        const int li = A.lself[i];
        double xa[P];
        ld_vec<double, P>(xa, sX + li * P);
        const double ya = sY[li], ca = sC[li];
        double sy = 0.0, sc = 0.0;
        const uint16_t *row = A.lell + A.lell_off[t] + threadIdx.x;
        const int w = A.tile_w[t];
        for (int j = 0; j < w; ++j) {
            const int l = __ldg(row + j * A.T);
            double xb[P];
            ld_vec<double, P>(xb, sX + l * P);
            double r2 = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const double d = xa[k] - xb[k];
                r2 += d * d;
            }
            const double tt = 1.0 - 0.5 * sqrt(r2) * A.inv_h;
            const double t3 = tt * tt * tt;
            sy += (ya - sY[l]) * t3;
            sc += (ca - sC[l]) * t3;
        }
        ac[i] = ya + dt * (double)A.dcoef * sy;
        dpart = ya * dt * (double)A.dcoef * sc * invD;
    }
    __shared__ double sh[4];
    const double v = warp_sum(dpart);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += sh[q];
        double *o = part + blockIdx.x * kTh;
        for (int k = 0; k < kTh; ++k) o[k] = 0.0;
        o[5] = s;
    }
}

// load jump transposed: prescribed axes are overwritten
template <int D>
__global__ void k_adj_load(const uint8_t *flags, long long n, double *au, double *av) {
    constexpr int P = Pad<D>::v;
    const long long i = blockIdx.x * (long long)kBlock + threadIdx.x;
    if (i >= n) return;
    const uint8_t fx = flags[i];
#pragma unroll
    for (int q = 0; q < D; ++q)
        if ((fx >> q) & 1) au[i * P + q] = av[i * P + q] = 0.0;
}

// seeds: u-bar += u_bar (original order); tip mean adjoint
template <int D>
__global__ void k_adj_seed(const uint8_t *flags, const long long *perm, long long n,
                           const double *ubar_orig, double t0, double t1, double t2, double *au) {
    constexpr int P = Pad<D>::v;
    const long long s = blockIdx.x * (long long)kBlock + threadIdx.x;
    if (s >= n) return;
    const double tb[3] = {t0, t1, t2};
    const bool tip = flags[s] & kTipBit;
#pragma unroll
    for (int q = 0; q < D; ++q) {
        double a = ubar_orig ? ubar_orig[perm[s] * D + q] : 0.0;
        if (tip) a += tb[q];
        au[s * P + q] += a;
    }
}

// adjoint field -> original order (doubles); field as mts_field
template <int D>
__global__ void k_adj_out(long long n, const long long *perm, int field, const double *au,
                          const double *av, const double *acp, const double *ac, double *out) {
    constexpr int P = Pad<D>::v;
    const long long s = blockIdx.x * (long long)kBlock + threadIdx.x;
    if (s >= n) return;
    const long long i = perm[s];
    switch (field) {
    case MTS_F_U: for (int q = 0; q < D; ++q) out[i * D + q] = au[s * P + q]; break;
    case MTS_F_V: for (int q = 0; q < D; ++q) out[i * D + q] = av[s * P + q]; break;
    case MTS_F_C: out[i] = ac[s]; break;
    case MTS_F_ALPHA: out[i] = acp[s * 8 + 6]; break;
    case MTS_F_CPINV: for (int q = 0; q < 6; ++q) out[i * 6 + q] = acp[s * 8 + q]; break;
    default: break;
    }
}

// sum of squares of the (u, v) adjoint: block partials, then one block in
// block order
template <int D>
__global__ void k_adj_norm_part(const double *au, const double *av, long long n, double *part) {
    constexpr int P = Pad<D>::v;
    const long long i = blockIdx.x * (long long)kBlock + threadIdx.x;
    double s = 0.0;
    if (i < n)
#pragma unroll
        for (int q = 0; q < D; ++q) s += au[i * P + q] * au[i * P + q] + av[i * P + q] * av[i * P + q];
    __shared__ double sh[kBlock / 32];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < kBlock / 32; ++q) t += sh[q];
        part[blockIdx.x] = t;
    }
}

__global__ void k_adj_norm_final(const double *part, long long nb, double *out) {
    __shared__ double red[256];
    double s = 0.0;
    for (long long q = threadIdx.x; q < nb; q += blockDim.x) s += part[q];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

template <int D>
size_t smem_adj_stress(const mts_body *b) {
    return 3 * second_off<double, Pad<D>::v>(b->max_halo);
}
template <int D>
size_t smem_adj_grad(const mts_body *b) {
    return second_off<double, Pad<D>::v>(b->max_halo) + (size_t)b->max_halo * MatS<D>::v * 8;
}
template <int D>
size_t smem_adj_diffuse(const mts_body *b) {
    return second_off<double, Pad<D>::v>(b->max_halo) + (size_t)b->max_halo * 16;
}

template <int D>
mts_status prepare_adj(mts_body *b) {
    int optin = 0;
    MTS_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->ctx->device));
    auto attr = [&](const void *fn, size_t need) -> mts_status {
        cudaFuncAttributes fa{};
        MTS_CUDA(cudaFuncGetAttributes(&fa, fn));
        const size_t cap = (size_t)optin - fa.sharedSizeBytes;
        if (need > cap) {
            set_error("adjoint kernel needs %zu bytes of shared memory, at most %zu fit", need, cap);
            return MTS_ERR_INVALID_ARG;
        }
        MTS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap));
        return MTS_OK;
    };
    MTS_TRY(attr((const void *)k_adj_stress<D, MTS_ELASTIC_SVK>, smem_adj_stress<D>(b)));
    MTS_TRY(attr((const void *)k_adj_stress<D, MTS_NEOHOOKE_J2>, smem_adj_stress<D>(b)));
    MTS_TRY(attr((const void *)k_adj_grad<D>, smem_adj_grad<D>(b)));
    MTS_TRY(attr((const void *)k_adj_diffuse<D>, smem_adj_diffuse<D>(b)));
    return MTS_OK;
}

// elastic moduli per unit E at fixed Poisson ratio: K = E/(3(1-2nu)), mu = E/(2(1+nu))
void moduli_seeds(const mts_body *b, double *dK, double *dmu) {
    *dK = 1.0 / (3.0 * (1.0 - 2.0 * b->nu));
    *dmu = 1.0 / (2.0 * (1.0 + b->nu));
}

template <int D>
mts_status adj_substep_t(mts_body *b, long long k, bool last) {
    cudaStream_t st = b->ctx->stream;
    const long long n = b->n;
    constexpr int P = Pad<D>::v;
    Args<double> A = make_args<double>(b);
    k_adj_setdt<<<1, 32, 0, st>>>(b->adj_ctrl, b->tape_dt, k);
    k_adj_drift<D><<<grid_n(n), kBlock, 0, st>>>(b->flags, n, b->adj_ctrl, b->adj_u, b->adj_v);
    MTS_CUDA(cudaGetLastError());
    MTS_TRY(launch_damping_adjoint(b, b->adj_v, b->adj_ctrl));
    k_adj_kick<D><<<grid_n(n), kBlock, 0, st>>>(b->flags, n, b->adj_ctrl, b->rho0 * b->V, b->adj_v,
                                                b->adj_a, b->adj_force_seed[0],
                                                b->adj_force_seed[1], b->adj_force_seed[2],
                                                last ? 1 : 0);
    double dK, dmu;
    moduli_seeds(b, &dK, &dmu);
    const double *tu = b->tape_u + k * n * P, *tcp = b->tape_cp + k * n * 8;
    const size_t ss = smem_adj_stress<D>(b);
    if (b->model == MTS_NEOHOOKE_J2)
        k_adj_stress<D, MTS_NEOHOOKE_J2><<<(unsigned)b->ntiles, b->T, ss, st>>>(
            A, b->adj_a, tu, tcp, b->adj_cp, b->adj_c, b->adj_G, b->adj_part, b->beta, dK, dmu);
    else
        k_adj_stress<D, MTS_ELASTIC_SVK><<<(unsigned)b->ntiles, b->T, ss, st>>>(
            A, b->adj_a, tu, tcp, b->adj_cp, b->adj_c, b->adj_G, b->adj_part, b->beta, dK, dmu);
    MTS_CUDA(cudaGetLastError());
    k_adj_grad<D><<<(unsigned)b->ntiles, b->T, smem_adj_grad<D>(b), st>>>(A, b->adj_G, b->adj_u);
    k_adj_theta<<<1, 256, 0, st>>>(b->adj_part, b->ntiles, b->adj_theta);
    MTS_CUDA(cudaGetLastError());
    return MTS_OK;
}

template <int D>
mts_status adj_diffusion_t(mts_body *b, double dt) {
    cudaStream_t st = b->ctx->stream;
    Args<double> A = make_args<double>(b);
    k_adj_free_c<<<grid_n(b->n), kBlock, 0, st>>>(b->flags, b->n, b->adj_c, b->adj_a);
    k_adj_diffuse<D><<<(unsigned)b->ntiles, b->T, smem_adj_diffuse<D>(b), st>>>(
        A, b->adj_a, b->tape_c, dt, b->D > 0 ? 1.0 / b->D : 0.0, b->adj_c, b->adj_part);
    k_adj_theta<<<1, 256, 0, st>>>(b->adj_part, b->ntiles, b->adj_theta);
    MTS_CUDA(cudaGetLastError());
    return MTS_OK;
}

}  // namespace

mts_status adjoint_prepare(mts_body *b) {
    return b->dim == 2 ? prepare_adj<2>(b) : prepare_adj<3>(b);
}

mts_status adjoint_tape(const mts_body *src, mts_body *dst, long long k) {
    const int pad = src->dim == 2 ? 2 : 4;
    if (src->rsize == 4)
        k_tape<float><<<grid_n(src->n), kBlock, 0, src->ctx->stream>>>(
            src->u, (const float *)src->cp, src->ctrl, src->n, pad, k, dst->tape_u, dst->tape_cp,
            dst->tape_dt);
    else
        k_tape<double><<<grid_n(src->n), kBlock, 0, src->ctx->stream>>>(
            src->u, (const double *)src->cp, src->ctrl, src->n, pad, k, dst->tape_u, dst->tape_cp,
            dst->tape_dt);
    MTS_CUDA(cudaGetLastError());
    return MTS_OK;
}

mts_status copy_c_to_double(const mts_body *src, double *dst) {
    if (src->rsize == 4)
        k_to_double<float><<<grid_n(src->n), kBlock, 0, src->ctx->stream>>>(
            (const float *)src->c, src->n, dst);
    else
        k_to_double<double><<<grid_n(src->n), kBlock, 0, src->ctx->stream>>>(
            (const double *)src->c, src->n, dst);
    MTS_CUDA(cudaGetLastError());
    return MTS_OK;
}

mts_status adjoint_substep(mts_body *b, long long k, bool last) {
    return b->dim == 2 ? adj_substep_t<2>(b, k, last) : adj_substep_t<3>(b, k, last);
}

mts_status adjoint_diffusion(mts_body *b, double dt) {
    return b->dim == 2 ? adj_diffusion_t<2>(b, dt) : adj_diffusion_t<3>(b, dt);
}

mts_status adjoint_load(mts_body *b) {
    if (b->dim == 2)
        k_adj_load<2><<<grid_n(b->n), kBlock, 0, b->ctx->stream>>>(b->flags, b->n, b->adj_u, b->adj_v);
    else
        k_adj_load<3><<<grid_n(b->n), kBlock, 0, b->ctx->stream>>>(b->flags, b->n, b->adj_u, b->adj_v);
    MTS_CUDA(cudaGetLastError());
    return MTS_OK;
}

mts_status adjoint_seed(mts_body *b, const double *ubar_orig_dev, const double tip[3]) {
    const double s = b->tip_count > 0 ? 1.0 / (double)b->tip_count : 0.0;
    const double t0 = tip ? tip[0] * s : 0.0, t1 = tip ? tip[1] * s : 0.0, t2 = tip ? tip[2] * s : 0.0;
    if (b->dim == 2)
        k_adj_seed<2><<<grid_n(b->n), kBlock, 0, b->ctx->stream>>>(b->flags, b->perm, b->n,
                                                                   ubar_orig_dev, t0, t1, t2, b->adj_u);
    else
        k_adj_seed<3><<<grid_n(b->n), kBlock, 0, b->ctx->stream>>>(b->flags, b->perm, b->n,
                                                                   ubar_orig_dev, t0, t1, t2, b->adj_u);
    MTS_CUDA(cudaGetLastError());
    return MTS_OK;
}

// |(u-bar, v-bar)|^2 into out_dev[0]; part_dev holds one double per block of kBlock
mts_status adjoint_norm2(mts_body *b, double *part_dev, double *out_dev) {
    const unsigned g = grid_n(b->n);
    if (b->dim == 2)
        k_adj_norm_part<2><<<g, kBlock, 0, b->ctx->stream>>>(b->adj_u, b->adj_v, b->n, part_dev);
    else
        k_adj_norm_part<3><<<g, kBlock, 0, b->ctx->stream>>>(b->adj_u, b->adj_v, b->n, part_dev);
    k_adj_norm_final<<<1, 256, 0, b->ctx->stream>>>(part_dev, g, out_dev);
    MTS_CUDA(cudaGetLastError());
    return MTS_OK;
}

mts_status adjoint_out(mts_body *b, int field, double *out_dev) {
    if (b->dim == 2)
        k_adj_out<2><<<grid_n(b->n), kBlock, 0, b->ctx->stream>>>(b->n, b->perm, field, b->adj_u,
                                                                  b->adj_v, b->adj_cp, b->adj_c, out_dev);
    else
        k_adj_out<3><<<grid_n(b->n), kBlock, 0, b->ctx->stream>>>(b->n, b->perm, field, b->adj_u,
                                                                  b->adj_v, b->adj_cp, b->adj_c, out_dev);
    MTS_CUDA(cudaGetLastError());
    return MTS_OK;
}

}  // namespace mts
