// mts_setup.cu -- one-time body setup on the GPU (Sec. 3.1: the neighbourhood
// and the correction matrix B0 are fixed in the reference configuration).
//
//   1. Morton order: cell = floor((X - Xmin)/dx), key = bit interleave (x lowest),
//      stable radix sort, so equal keys keep the original index order.
//   2. Neighbour CSR: all j != i with |X_i - X_j|^2 < (2h)^2, evaluated in FP64
//      with explicit round-to-nearest multiply/add (no fused multiply-add), over
//      a dense cell grid; rows sorted ascending with a segmented sort.
//   3. B0_a = (sum_b V (X_b - X_a) (x) grad_a W_ab)^-1 in FP64.
//   4. Morton tiles of T particles with their neighbour halos and 16-bit local
//      neighbour slots (shared-memory staging in the substep kernels).
//   5. Canonical order of the pairwise damping (Sec. 4.3): pairs owned by the
//      componentwise-min block (blocks of 2^s cells, 2^s dx > 2h) of their two
//      particles; block colour = parity bits; greedy sub-colours in ascending
//      (a,b) per owner block, at most 32 pairs per sub-colour; then per-block
//      level lists with block-local
//      particle indices for the shared-memory damping kernel.
#include <cub/cub.cuh>

#include <algorithm>
#include <cmath>
#include <vector>

#include "mts_device.cuh"
#include "mts_internal.cuh"

namespace mts {

namespace {

constexpr int TPB = 256;

inline unsigned grid_for(long long n, int tpb = TPB) {
    return (unsigned)((n + tpb - 1) / tpb);
}

__host__ __device__ inline unsigned long long morton(int dim, long long c0, long long c1,
                                                     long long c2) {
    unsigned long long key = 0;
    long long c[3] = {c0, c1, c2};
    int bits = dim == 2 ? 32 : 21;
    for (int bit = 0; bit < bits; ++bit)
        for (int k = 0; k < dim; ++k)
            key |= (unsigned long long)((c[k] >> bit) & 1) << (bit * dim + k);
    return key;
}

// exact FP64 squared distance (explicit rounding, no contraction)
__device__ inline double dist2_rn(const double *a, const double *b, int dim) {
    double d0 = __dsub_rn(a[0], b[0]);
    double d1 = __dsub_rn(a[1], b[1]);
    double r2 = __dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1));
    if (dim == 3) {
        double d2 = __dsub_rn(a[2], b[2]);
        r2 = __dadd_rn(r2, __dmul_rn(d2, d2));
    }
    return r2;
}

// ---------------------------------------------------------------- extents
__global__ void k_extent_partial(const double *X, long long n, int dim, double *part) {
    __shared__ double smin[3][TPB];
    __shared__ int sbad[TPB];
    double mn[3] = {INFINITY, INFINITY, INFINITY};
    int bad = 0;
    for (long long i = blockIdx.x * (long long)TPB + threadIdx.x; i < n;
         i += (long long)gridDim.x * TPB)
        for (int k = 0; k < dim; ++k) {
            double x = X[i * dim + k];
            if (!isfinite(x)) bad = 1;
            mn[k] = fmin(mn[k], x);
        }
    for (int k = 0; k < 3; ++k) smin[k][threadIdx.x] = mn[k];
    sbad[threadIdx.x] = bad;
    __syncthreads();
    for (int s = TPB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            for (int k = 0; k < 3; ++k)
                smin[k][threadIdx.x] = fmin(smin[k][threadIdx.x], smin[k][threadIdx.x + s]);
            sbad[threadIdx.x] |= sbad[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k < 3; ++k) part[blockIdx.x * 4 + k] = smin[k][0];
        part[blockIdx.x * 4 + 3] = sbad[0];
    }
}

__global__ void k_extent_final(const double *part, int nblk, double *out) {
    if (threadIdx.x != 0) return;
    double mn[3] = {INFINITY, INFINITY, INFINITY};
    double bad = 0;
    for (int b = 0; b < nblk; ++b) {
        for (int k = 0; k < 3; ++k) mn[k] = fmin(mn[k], part[b * 4 + k]);
        bad = fmax(bad, part[b * 4 + 3]);
    }
    for (int k = 0; k < 3; ++k) out[k] = mn[k];
    out[3] = bad;
}

// ---------------------------------------------------------------- Morton keys
__global__ void k_keys(const double *X, long long n, int dim, double x0, double x1, double x2,
                       double dx, unsigned long long *keys, long long *vals,
                       unsigned long long *cmax) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double xm[3] = {x0, x1, x2};
    long long c[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) {
        c[k] = (long long)floor(__ddiv_rn(__dsub_rn(X[i * dim + k], xm[k]), dx));
        atomicMax(cmax + k, (unsigned long long)c[k]);
    }
    keys[i] = morton(dim, c[0], c[1], c[2]);
    vals[i] = i;
}

template <class R, int D>
__global__ void k_apply_perm(const double *Xo, const long long *perm, long long n, double x0,
                             double x1, double x2, double dx, double *X64, R *Xr,
                             long long *rank, int *cell) {
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= n) return;
    constexpr int P = Pad<D>::v;
    long long i = perm[s];
    rank[i] = s;
    double xm[3] = {x0, x1, x2};
    for (int k = 0; k < P; ++k) {
        double x = k < D ? Xo[i * D + k] : 0.0;
        X64[s * P + k] = x;
        Xr[s * P + k] = k < D ? (R)(x - xm[k]) : R(0);
    }
    for (int k = 0; k < 3; ++k)
        cell[s * 3 + k] = k < D ? (int)floor(__ddiv_rn(__dsub_rn(Xo[i * D + k], xm[k]), dx)) : 0;
}

// ---------------------------------------------------------------- cell grid
__global__ void k_cell_ranges(const unsigned long long *keys, const int *cell, long long n,
                              long long g0, long long g1, int *cstart, int *cend) {
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= n) return;
    long long lin = ((long long)cell[s * 3 + 2] * g1 + cell[s * 3 + 1]) * g0 + cell[s * 3 + 0];
    if (s == 0 || keys[s] != keys[s - 1]) cstart[lin] = (int)s;
    if (s == n - 1 || keys[s + 1] != keys[s]) cend[lin] = (int)(s + 1);
}

template <int D, bool FILL>
__global__ void k_neigh(const double *X64, const int *cell, long long n, long long g0,
                        long long g1, long long g2, int reach, double cut2, const int *cstart,
                        const int *cend, long long *cnt, const long long *off, int32_t *out) {
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= n) return;
    constexpr int P = Pad<D>::v;
    const double *xs = X64 + s * P;
    int cx = cell[s * 3], cy = cell[s * 3 + 1], cz = cell[s * 3 + 2];
    long long c = 0;
    long long base = FILL ? off[s] : 0;
    int zr = D == 3 ? reach : 0;
    for (int z = cz - zr; z <= cz + zr; ++z) {
        if (z < 0 || z >= g2) continue;
        for (int y = cy - reach; y <= cy + reach; ++y) {
            if (y < 0 || y >= g1) continue;
            for (int x = cx - reach; x <= cx + reach; ++x) {
                if (x < 0 || x >= g0) continue;
                long long lin = ((long long)z * g1 + y) * g0 + x;
                int a = cstart[lin];
                if (a < 0) continue;
                int e = cend[lin];
                for (int j = a; j < e; ++j) {
                    if (j == s) continue;
                    if (dist2_rn(xs, X64 + (long long)j * P, D) < cut2) {
                        if (FILL) out[base + c] = j;
                        ++c;
                    }
                }
            }
        }
    }
    if (!FILL) cnt[s] = c;
}

// ---------------------------------------------------------------- B0
template <class R, int D>
__global__ void k_b0(const double *X64, const long long *off, const int32_t *idx, long long n,
                     double h, double alpha, double V, R *B0, Control *ctrl) {
    long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (a >= n) return;
    constexpr int P = Pad<D>::v;
    double S[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    const double *xa = X64 + a * P;
    for (long long p = off[a]; p < off[a + 1]; ++p) {
        const double *xb = X64 + (long long)idx[p] * P;
        double d[3] = {0, 0, 0}, r2 = 0;
        for (int k = 0; k < D; ++k) {
            d[k] = xa[k] - xb[k];
            r2 += d[k] * d[k];
        }
        double r = sqrt(r2);
        double q = r / h;
        double t = 1.0 - 0.5 * q;
        double dw = -5.0 * alpha * q * t * t * t / h;   // W'(r)
        for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j) S[i][j] += V * (-d[i]) * (dw * d[j] / r);
    }
    double nrm = 0;
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) nrm += S[i][j] * S[i][j];
    nrm = sqrt(nrm);
    R out[D][D];
    if (D == 2) {
        double det = S[0][0] * S[1][1] - S[0][1] * S[1][0];
        if (!(fabs(det) >= 1e-12 * nrm * nrm) || nrm == 0.0) {
            atomicOr(&ctrl->err, kErrSingular);
            det = 1.0;
        }
        out[0][0] = (R)(S[1][1] / det);
        out[0][1] = (R)(-S[0][1] / det);
        out[1][0] = (R)(-S[1][0] / det);
        out[1][1] = (R)(S[0][0] / det);
    } else {
        double det = S[0][0] * (S[1][1] * S[2][2] - S[1][2] * S[2][1]) -
                     S[0][1] * (S[1][0] * S[2][2] - S[1][2] * S[2][0]) +
                     S[0][2] * (S[1][0] * S[2][1] - S[1][1] * S[2][0]);
        if (!(fabs(det) >= 1e-12 * nrm * nrm * nrm) || nrm == 0.0) {
            atomicOr(&ctrl->err, kErrSingular);
            det = 1.0;
        }
        double C[3][3];
        C[0][0] = S[1][1] * S[2][2] - S[1][2] * S[2][1];
        C[0][1] = S[0][2] * S[2][1] - S[0][1] * S[2][2];
        C[0][2] = S[0][1] * S[1][2] - S[0][2] * S[1][1];
        C[1][0] = S[1][2] * S[2][0] - S[1][0] * S[2][2];
        C[1][1] = S[0][0] * S[2][2] - S[0][2] * S[2][0];
        C[1][2] = S[0][2] * S[1][0] - S[0][0] * S[1][2];
        C[2][0] = S[1][0] * S[2][1] - S[1][1] * S[2][0];
        C[2][1] = S[0][1] * S[2][0] - S[0][0] * S[2][1];
        C[2][2] = S[0][0] * S[1][1] - S[0][1] * S[1][0];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) out[i][j] = (R)(C[i][j] / det);
    }
    R *dst = B0 + a * MatS<D>::v;
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < P; ++j) dst[i * P + j] = j < D ? out[i][j] : R(0);
}

// ---------------------------------------------------------------- damping order
__global__ void k_count_pairs(const long long *off, const int32_t *idx, long long n,
                              long long *cnt) {
    long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (a >= n) return;
    long long c = 0;
    for (long long p = off[a]; p < off[a + 1]; ++p) c += idx[p] > a;
    cnt[a] = c;
}

// owner-block widths per axis: 2^s cells, or the whole axis (s = kWholeAxis)
struct Shifts {
    int s[3];
};
__host__ __device__ inline long long bco(long long c, int s) { return s >= 31 ? 0 : c >> s; }

__global__ void k_fill_pairs(const long long *off, const int32_t *idx, const int *cell,
                             long long n, int dim, Shifts sh, const long long *poff,
                             int32_t *pa, int32_t *pb, unsigned long long *key) {
    long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (a >= n) return;
    long long t = poff[a];
    for (long long p = off[a]; p < off[a + 1]; ++p) {
        int b = idx[p];
        if (b <= a) continue;
        long long ob[3] = {0, 0, 0};
        int col = 0;
        for (int k = 0; k < dim; ++k) {
            long long ba = bco(cell[a * 3 + k], sh.s[k]), bb = bco(cell[(long long)b * 3 + k], sh.s[k]);
            ob[k] = ba < bb ? ba : bb;
            col |= (int)(ob[k] & 1) << k;
        }
        pa[t] = (int32_t)a;
        pb[t] = b;
        key[t] = ((unsigned long long)col << 60) | morton(dim, ob[0], ob[1], ob[2]);
        ++t;
    }
}

template <class T>
__global__ void k_gather(const T *src, const long long *order, long long m, T *dst) {
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p < m) dst[p] = src[order[p]];
}

__global__ void k_iota(long long *v, long long m) {
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p < m) v[p] = p;
}

__global__ void k_run_flags(const unsigned long long *key, long long m, long long *flag) {
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p < m) flag[p] = (p == 0 || key[p] != key[p - 1]) ? 1 : 0;
}

// after an inclusive scan of the flags: id = scan - 1
__global__ void k_run_starts(const long long *scan, long long m, long long *start) {
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= m) return;
    if (p == 0 || scan[p] != scan[p - 1]) start[scan[p] - 1] = p;
}

__global__ void k_block_keys(const int *cell, long long n, int dim, Shifts sh,
                             unsigned long long *bkey) {
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= n) return;
    bkey[s] = morton(dim, bco(cell[s * 3], sh.s[0]), bco(cell[s * 3 + 1], sh.s[1]),
                     bco(cell[s * 3 + 2], sh.s[2]));
}

template <class T>
__global__ void k_inverse(const long long *perm, long long n, T *inv) {
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s < n) inv[perm[s]] = (T)s;
}

__global__ void k_to_i32(const long long *in, long long n, int32_t *out) {
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s < n) out[s] = (int32_t)in[s];
}

__global__ void k_block_table(const long long *bstart, long long nb, long long n,
                              const unsigned long long *bkey_p, unsigned long long *bkey,
                              int *bcnt, unsigned int *mb) {
    long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    long long s = bstart[b];
    long long e = b + 1 < nb ? bstart[b + 1] : n;
    bkey[b] = bkey_p[s];
    bcnt[b] = (int)(e - s);
    atomicMax(mb, (unsigned int)(e - s));
}

__device__ long long find_key(const unsigned long long *keys, long long m, unsigned long long k) {
    long long lo = 0, hi = m;
    while (lo < hi) {
        long long mid = (lo + hi) >> 1;
        if (keys[mid] < k) lo = mid + 1;
        else hi = mid;
    }
    return (lo < m && keys[lo] == k) ? lo : -1;
}

// the blocked axes in ascending order; bit j of a touched-block index is the
// +1 step on the j-th of them
__device__ inline int blocked_axes(const Shifts &sh, int dim, int *ax) {
    int nb = 0;
    for (int k = 0; k < dim; ++k)
        if (sh.s[k] < kWholeAxis) ax[nb++] = k;
    return nb;
}

// per owner group: the touched blocks (owner + steps on the blocked axes),
// their first block-sorted position and particle count
__global__ void k_touch(const long long *gstart, long long ng, const int32_t *pa, const int32_t *pb,
                        const int *cell, int dim, Shifts sh, const unsigned long long *bkey,
                        const long long *bstart, const int *bcnt, long long nblocks,
                        int32_t *tstart, int32_t *tcnt, int32_t *gcol, long long *gkey) {
    long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g >= ng) return;
    long long p = gstart[g];
    int a = pa[p], b = pb[p];
    long long ob[3] = {0, 0, 0};
    int col = 0;
    for (int k = 0; k < dim; ++k) {
        long long ba = bco(cell[(long long)a * 3 + k], sh.s[k]);
        long long bb = bco(cell[(long long)b * 3 + k], sh.s[k]);
        ob[k] = ba < bb ? ba : bb;
        col |= (int)(ob[k] & 1) << k;
    }
    gcol[g] = col;
    gkey[g] = (long long)morton(dim, ob[0], ob[1], ob[2]);
    int ax[3];
    const int nblk = blocked_axes(sh, dim, ax);
    const int nbk = 1 << dim;
    for (int e = 0; e < nbk; ++e) {
        long long bi = -1;
        if (e < (1 << nblk)) {
            long long c[3] = {ob[0], ob[1], ob[2]};
            for (int j = 0; j < nblk; ++j) c[ax[j]] += (e >> j) & 1;
            bi = find_key(bkey, nblocks, morton(dim, c[0], c[1], c[2]));
        }
        tstart[g * nbk + e] = bi >= 0 ? (int32_t)bstart[bi] : 0;
        tcnt[g * nbk + e] = bi >= 0 ? bcnt[bi] : 0;
    }
}

// greedy sub-colouring of one owner group per thread; local particle index =
// e * mb + (block-sorted position - start of touched block e); cap = most
// pairs per sub-colour (0 = no cap)
__global__ void k_greedy(const long long *gstart, long long g0, long long g1, long long ng,
                         long long m, const int32_t *pa, const int32_t *pb, const int *cell,
                         int dim, Shifts sh, const int32_t *tstart, const int32_t *binv, int mb,
                         int nbw, int cap, unsigned long long *used, int32_t *sub, uint32_t *ab,
                         int32_t *nsub, Control *ctrl) {
    long long g = g0 + blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g >= g1) return;
    const int nbk = 1 << dim;
    unsigned long long *U = used + (g - g0) * (long long)nbw * mb * 4;
    long long p0 = gstart[g], p1 = g + 1 < ng ? gstart[g + 1] : m;
    long long ob[3] = {0, 0, 0};
    {
        int a = pa[p0], b = pb[p0];
        for (int k = 0; k < dim; ++k) {
            long long ba = bco(cell[(long long)a * 3 + k], sh.s[k]);
            long long bb = bco(cell[(long long)b * 3 + k], sh.s[k]);
            ob[k] = ba < bb ? ba : bb;
        }
    }
    int ax[3];
    const int nblk = blocked_axes(sh, dim, ax);
    int maxc = -1;
    int count[256];
    for (int c = 0; c < 256; ++c) count[c] = 0;
    for (long long p = p0; p < p1; ++p) {
        int loc[2];
        int pp[2] = {pa[p], pb[p]};
        for (int t = 0; t < 2; ++t) {
            int e = 0;
            for (int j = 0; j < nblk; ++j)
                e |= (int)(bco(cell[(long long)pp[t] * 3 + ax[j]], sh.s[ax[j]]) - ob[ax[j]]) << j;
            loc[t] = e * mb + (binv[pp[t]] - tstart[g * nbk + e]);
        }
        unsigned long long *ua = U + (long long)loc[0] * 4, *ub = U + (long long)loc[1] * 4;
        // smallest sub-colour free at both particles that still has room
        int c = -1;
        for (int w = 0; w < 4 && c < 0; ++w) {
            unsigned long long free_bits = ~(ua[w] | ub[w]);
            while (free_bits) {
                const int cand = w * 64 + __ffsll((long long)free_bits) - 1;
                if (cap == 0 || count[cand] < cap) {
                    c = cand;
                    break;
                }
                free_bits &= free_bits - 1;
            }
        }
        if (c < 0) {
            atomicOr(&ctrl->err, kErrTooMany);
            c = 255;
        }
        ++count[c];
        ua[c >> 6] |= 1ull << (c & 63);
        ub[c >> 6] |= 1ull << (c & 63);
        sub[p] = c;
        ab[p] = (uint32_t)loc[0] | ((uint32_t)loc[1] << 16);
        maxc = max(maxc, c);
    }
    nsub[g] = maxc + 1;
}

// offset class: cell(b) - cell(a), sign-folded, base (2R+1) digits; the greedy
// visits a group's classes in descending order
__global__ void k_pair_class(const int32_t *pa, const int32_t *pb, const long long *gscan,
                             long long m, const int *cell, int dim, int R,
                             unsigned long long *key) {
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= m) return;
    long long o[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k)
        o[k] = (long long)cell[(long long)pb[p] * 3 + k] - cell[(long long)pa[p] * 3 + k];
    int sg = 0;
    for (int k = dim - 1; k >= 0 && sg == 0; --k)
        if (o[k] != 0) sg = o[k] > 0 ? 1 : -1;
    long long c = 0, base = 2 * R + 1;
    for (int k = dim - 1; k >= 0; --k) c = c * base + (sg * o[k] + R);
    // classes in descending order within a group (c < 2^16)
    key[p] = ((unsigned long long)(gscan[p] - 1) << 16) | (unsigned long long)(0xffff - c);
}

template <class T>
__global__ void k_scatter(const T *src, const long long *order, long long m, T *dst) {
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p < m) dst[order[p]] = src[p];
}

// padded kernel layout: level L of the canonical order occupies slots
// [32 L, 32 L + 32); pair p sits at slot 32 L + lane (lane & 31 of k_level_lanes)
// slot words hold byte offsets (slot index * bytes per velocity slot) of the
// two particles in the damping kernel's staged velocities, in the order the
// lane assignment chose (bit 5 of lane: pair_b first)
__global__ void k_fill_slots(const unsigned long long *key2s, long long m, const int32_t *grp_lvl,
                             const long long *lvl_pair, const uint32_t *ab, const int8_t *lane,
                             long long *slot, uint32_t *kab, int bps) {
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= m) return;
    const long long g = (long long)(key2s[p] >> 8);
    const int s = (int)(key2s[p] & 255);
    const long long L = grp_lvl[g] + s;
    const int lv = lane[p];
    const bool sw = (lv & 32) != 0;
    const long long sl = 32 * L + (lv & 31);
    slot[p] = sl | (sw ? (1LL << kSlotSwapBit) : 0LL);
    uint32_t la = (uint32_t)damp_slot_pos((int)(ab[p] & 0xffffu), bps);
    uint32_t lb = (uint32_t)damp_slot_pos((int)(ab[p] >> 16), bps);
    if (sw) {
        const uint32_t t = la;
        la = lb;
        lb = t;
    }
    kab[sl] = (la * (uint32_t)bps) | ((lb * (uint32_t)bps) << 16);
}

// Lane and particle order of each pair inside its level.  A level's pairs
// touch disjoint particles, so any assignment gives the same result, and a
// free pair's update is symmetric in its particles bit for bit.  With 16-byte
// slots a 128-bit shared access is served eight lanes (a quarter-warp) at a
// time, and its cost there is the largest number of lanes whose slots fall in
// one 16-byte bank group (empty lanes of a quarter with a pair read that
// pair's slots: free).  A level step loads and stores both particles, so a
// quarter costs 2 (mA + mB) wavefronts, mA and mB the largest bank-group
// counts of its first and second particles (2 for a quarter without pairs:
// its lanes load one dummy slot).  The pairs are placed greedily, the most
// crowded bank groups first, in the quarter that keeps those counts lowest;
// then a local search over the pairs that share a bank group in their quarter
// tries reversing the pair, then moving it to each lane of the other quarters
// (exchanging with that lane's pair, either in either order) and keeps the
// first change that lowers the cost of the two quarters, up to two passes
// (a third changed the modelled cost by 0.2 %).
// Other slot sizes keep the canonical order.
__device__ __forceinline__ int lanes_max8(const uint8_t *h) {
    int m = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) m = max(m, (int)h[k]);
    return m;
}

__global__ void k_level_lanes(const long long *lvl_pair, long long nlev, const uint32_t *ab,
                              int bps, int8_t *lane) {
    const long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (L >= nlev) return;
    const long long p0 = lvl_pair[L];
    const int n = (int)(lvl_pair[L + 1] - p0);
    if (bps != 16 || n <= 1 || n > 32) {
        for (int k = 0; k < n; ++k) lane[p0 + k] = (int8_t)k;
        return;
    }
    int ga[32], gb[32], ord[32], pos[32];
    for (int k = 0; k < n; ++k) {
        ga[k] = damp_slot_pos((int)(ab[p0 + k] & 0xffffu), bps) & 7;
        gb[k] = damp_slot_pos((int)(ab[p0 + k] >> 16), bps) & 7;
        pos[k] = k;
    }
    if (n > 8) {
        int fa[8] = {0, 0, 0, 0, 0, 0, 0, 0}, fb[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int k = 0; k < n; ++k) {
            ++fa[ga[k]];
            ++fb[gb[k]];
        }
        // visit order: descending fa[ga] + fb[gb], ties by canonical position
        for (int k = 0; k < n; ++k) ord[k] = k;
        for (int i = 1; i < n; ++i) {
            const int x = ord[i], kx = fa[ga[x]] + fb[gb[x]];
            int j = i - 1;
            while (j >= 0 && fa[ga[ord[j]]] + fb[gb[ord[j]]] < kx) {
                ord[j + 1] = ord[j];
                --j;
            }
            ord[j + 1] = x;
        }
        int ca[4][8], cb[4][8], size[4] = {0, 0, 0, 0}, ma[4] = {0, 0, 0, 0}, mxb[4] = {0, 0, 0, 0};
        for (int q = 0; q < 4; ++q)
            for (int k = 0; k < 8; ++k) ca[q][k] = cb[q][k] = 0;
        for (int i = 0; i < n; ++i) {
            const int k = ord[i];
            int best = -1, bc0 = 0, bc1 = 0;
            for (int q = 0; q < 4; ++q) {
                if (size[q] >= 8) continue;
                const int c0 = max(ca[q][ga[k]] + 1, ma[q]) + max(cb[q][gb[k]] + 1, mxb[q]);
                const int c1 = ca[q][ga[k]] + cb[q][gb[k]];
                if (best < 0 || c0 < bc0 || (c0 == bc0 && (c1 < bc1 || (c1 == bc1 && size[q] < size[best])))) {
                    best = q;
                    bc0 = c0;
                    bc1 = c1;
                }
            }
            pos[k] = best * 8 + size[best];
            ++size[best];
            ma[best] = max(ma[best], ++ca[best][ga[k]]);
            mxb[best] = max(mxb[best], ++cb[best][gb[k]]);
        }
    }
    // local search
    int at[32];
    bool fl[32];
    uint8_t hA[4][8], hB[4][8];
    int cnt[4] = {0, 0, 0, 0};
    for (int i = 0; i < 32; ++i) at[i] = -1;
    for (int q = 0; q < 4; ++q)
        for (int k = 0; k < 8; ++k) hA[q][k] = hB[q][k] = 0;
    for (int k = 0; k < n; ++k) {
        at[pos[k]] = k;
        fl[k] = false;
        ++hA[pos[k] >> 3][ga[k]];
        ++hB[pos[k] >> 3][gb[k]];
        ++cnt[pos[k] >> 3];
    }
    auto qcost = [&](int q) { return cnt[q] ? 2 * (lanes_max8(hA[q]) + lanes_max8(hB[q])) : 2; };
    for (int pass = 0; pass < 2; ++pass) {
        bool improved = false;
        for (int i = 0; i < 32; ++i) {
            const int k = at[i];
            if (k < 0) continue;
            const int qi = i >> 3;
            const int a = fl[k] ? gb[k] : ga[k], b = fl[k] ? ga[k] : gb[k];
            if (hA[qi][a] <= 1 && hB[qi][b] <= 1) continue;
            const int base_i = qcost(qi);
            // the pair reversed
            --hA[qi][a]; --hB[qi][b]; ++hA[qi][b]; ++hB[qi][a];
            if (qcost(qi) < base_i) {
                fl[k] = !fl[k];
                improved = true;
                continue;
            }
            --hA[qi][b]; --hB[qi][a]; ++hA[qi][a]; ++hB[qi][b];
            bool done = false;
            for (int j = 0; j < 32 && !done; ++j) {
                const int qj = j >> 3;
                if (qj == qi) continue;
                const int k2 = at[j];
                const int base = base_i + qcost(qj);
                const int a2 = k2 < 0 ? 0 : (fl[k2] ? gb[k2] : ga[k2]);
                const int b2 = k2 < 0 ? 0 : (fl[k2] ? ga[k2] : gb[k2]);
                for (int v = 0; v < (k2 < 0 ? 2 : 4) && !done; ++v) {
                    const bool fi = v & 1, fj = (v >> 1) & 1;
                    const int ai = fi ? b : a, bi = fi ? a : b;
                    const int aj = fj ? b2 : a2, bj = fj ? a2 : b2;
                    --hA[qi][a]; --hB[qi][b]; --cnt[qi];
                    ++hA[qj][ai]; ++hB[qj][bi]; ++cnt[qj];
                    if (k2 >= 0) {
                        --hA[qj][a2]; --hB[qj][b2]; --cnt[qj];
                        ++hA[qi][aj]; ++hB[qi][bj]; ++cnt[qi];
                    }
                    if (qcost(qi) + qcost(qj) < base) {
                        at[i] = k2;
                        at[j] = k;
                        if (fi) fl[k] = !fl[k];
                        if (k2 >= 0 && fj) fl[k2] = !fl[k2];
                        done = improved = true;
                        break;
                    }
                    if (k2 >= 0) {
                        --hA[qi][aj]; --hB[qi][bj]; --cnt[qi];
                        ++hA[qj][a2]; ++hB[qj][b2]; ++cnt[qj];
                    }
                    --hA[qj][ai]; --hB[qj][bi]; --cnt[qj];
                    ++hA[qi][a]; ++hB[qi][b]; ++cnt[qi];
                }
            }
        }
        if (!improved) break;
    }
    for (int i = 0; i < 32; ++i)
        if (at[i] >= 0) lane[p0 + at[i]] = (int8_t)(i | (fl[at[i]] ? 32 : 0));
}

// Empty slots of a quarter-warp that holds a pair take that pair's word
// (coefficient 0: the lane loads what a neighbour lane loads, a broadcast,
// and stores nothing); quarters without a pair keep the dummy slot.
__global__ void k_fill_empty(uint32_t *kab, long long nlev, uint32_t dummy_word) {
    const long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (L >= nlev) return;
    uint32_t *w = kab + 32 * L;
    for (int q = 0; q < 4; ++q) {
        uint32_t first = dummy_word;
        for (int k = 0; k < 8; ++k)
            if (w[8 * q + k] != dummy_word) {
                first = w[8 * q + k];
                break;
            }
        if (first == dummy_word) continue;
        for (int k = 0; k < 8; ++k)
            if (w[8 * q + k] == dummy_word) w[8 * q + k] = first;
    }
}

__global__ void k_fill_dummy(uint32_t *kab, long long ns, uint32_t dummy) {
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k < ns) kab[k] = dummy | (dummy << 16);
}

template <class R>
__global__ void k_fill_slot_g(const R *g, const long long *slot, long long m, R *kg) {
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p < m) kg[slot[p] & kSlotMask] = g[p];
}

__global__ void k_group_of_pair(const long long *gscan, long long m, const int32_t *sub,
                                unsigned long long *key2) {
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p < m) key2[p] = ((unsigned long long)(gscan[p] - 1) << 8) | (unsigned)sub[p];
}

__global__ void k_levels(const unsigned long long *key2, long long m, const int32_t *grp_lvl,
                         long long *lvl_pair, long long nlev) {
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p > m) return;
    if (p == m) {
        lvl_pair[nlev] = m;
        return;
    }
    if (p == 0 || key2[p] != key2[p - 1]) {
        long long g = (long long)(key2[p] >> 8);
        int s = (int)(key2[p] & 255);
        lvl_pair[grp_lvl[g] + s] = p;
    }
}

template <class R, int D>
__global__ void k_pair_coef(const int32_t *pa, const int32_t *pb, long long m, const double *X64,
                            double h, double alpha, double V, R *g) {
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= m) return;
    constexpr int P = Pad<D>::v;
    const double *xa = X64 + (long long)pa[p] * P, *xb = X64 + (long long)pb[p] * P;
    double r2 = 0;
    for (int k = 0; k < D; ++k) {
        double d = xa[k] - xb[k];
        r2 += d * d;
    }
    double r = sqrt(r2);
    double q = r / h, t = 1.0 - 0.5 * q;
    double dw = -5.0 * alpha * q * t * t * t / h;
    g[p] = (R)(-2.0 * V * V * dw / r);   // B_ab / eta
}

// ---------------------------------------------------------------- tiles
// entries of tile t: its own particles and all their CSR neighbours
__global__ void k_tile_entries(const long long *off, const int32_t *idx, long long n, int32_t *vals) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    long long dst = off[i] + i;
    vals[dst] = (int32_t)i;
    for (long long p = off[i]; p < off[i + 1]; ++p) vals[++dst] = idx[p];
}

__global__ void k_tile_seg(const long long *off, long long n, int T, long long ntiles,
                           long long *seg) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t > ntiles) return;
    long long i = t * T < n ? t * T : n;
    seg[t] = off[i] + i;
}

__global__ void k_uniq_flags(const int32_t *v, long long m, long long *flag) {
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k < m) flag[k] = (k == 0 || v[k] != v[k - 1]) ? 1 : 0;
}

__global__ void k_seg_start_flags(const long long *seg, long long ntiles, long long *flag) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < ntiles) flag[seg[t]] = 1;
}

__global__ void k_halo_compact(const int32_t *v, const long long *flag, const long long *scan,
                               long long m, int32_t *halo) {
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k < m && flag[k]) halo[scan[k] - 1] = v[k];
}

__global__ void k_halo_off(const long long *seg, const long long *scan, long long ntiles,
                           long long total, long long *hoff, unsigned int *hmax) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t > ntiles) return;
    hoff[t] = t == ntiles ? total : scan[seg[t]] - 1;
    if (t < ntiles) {
        long long e = t + 1 == ntiles ? total : scan[seg[t + 1]] - 1;
        atomicMax(hmax, (unsigned int)(e - (scan[seg[t]] - 1)));
    }
}

// per halo entry of tile t: X(particle) - X(first particle of the tile), in
// FP64, stored in the storage precision
template <class R, int P>
__global__ void k_halo_x(const long long *hoff, const int32_t *halo, long long ntiles, int T,
                         long long total, const double *X64, R *hx) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= total) return;
    long long lo = 0, hi = ntiles;   // tile of entry e: hoff[t] <= e < hoff[t + 1]
    while (hi - lo > 1) {
        const long long mid = (lo + hi) >> 1;
        if (hoff[mid] <= e) lo = mid;
        else hi = mid;
    }
    const double *o = X64 + lo * T * P, *x = X64 + (long long)halo[e] * P;
#pragma unroll
    for (int k = 0; k < P; ++k) hx[e * P + k] = (R)(x[k] - o[k]);
}

// longest neighbour list whose visiting order is scheduled (longer lists keep
// the CSR order)
constexpr int kEllOrderCap = 128;

__global__ void k_tile_w(const long long *off, long long n, int T, long long ntiles, long long *w,
                         unsigned int *wmax) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    long long m = 0;
    for (long long i = t * T; i < min(n, (t + 1) * T); ++i) m = max(m, off[i + 1] - off[i]);
    w[t] = m * T;
    if (m <= kEllOrderCap) atomicMax(wmax, (unsigned int)m);
}

__device__ int find_slot(const int32_t *h, long long len, int32_t key) {
    long long lo = 0, hi = len;
    while (lo < hi) {
        long long mid = (lo + hi) >> 1;
        if (h[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return (int)lo;
}

// Per tile: the local slot of every particle (lself) and its neighbours' halo
// slots in CSR order, neighbour-major (entry j of tile lane k at j * T + k),
// padded to the tile's width with the particle's own slot (a zero
// contribution: the kernel gradient vanishes at r = 0).  Lanes past the end of
// the body hold slot 0 and are never read.
__global__ void k_local_ell(const long long *off, const int32_t *idx, long long n, int T,
                            long long ntiles, const long long *hoff, const int32_t *halo,
                            const long long *loff, int32_t *tw, uint16_t *lell, uint16_t *lself) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long t = i / T;
    if (t >= ntiles) return;
    int lane = (int)(i - t * T);
    long long width = (loff[t + 1] - loff[t]) / T;
    if (lane == 0) tw[t] = (int32_t)width;
    const int32_t *h = halo + hoff[t];
    long long hl = hoff[t + 1] - hoff[t];
    uint16_t *out = lell + loff[t] + lane;
    if (i >= n) {
        for (long long j = 0; j < width; ++j) out[j * T] = 0;
        return;
    }
    int self = find_slot(h, hl, (int32_t)i);
    lself[i] = (uint16_t)self;
    long long deg = off[i + 1] - off[i];
    for (long long j = 0; j < width; ++j)
        out[j * T] = (uint16_t)(j < deg ? find_slot(h, hl, idx[off[i] + j]) : self);
}

// Visiting order of the gathers.  The order in which a particle visits its
// neighbours is free (it moves only the rounding of the sums).  The 3D gathers
// stage one 16-byte unit (or a 48-byte record of three) per halo slot, so slot s
// sits in bank group s mod 8 (3s + unit mod 8), and a 16-byte shared load is
// served eight lanes at a time: its cost is, over those eight lanes, the
// largest number of DIFFERENT slots that fall in one bank group (lanes reading
// the same slot share one access).  In 2D the positions are 8-byte slots
// served sixteen lanes at a time, residues mod 16.  The eight (sixteen) lanes
// of a group are neighbouring particles whose lists overlap heavily, so the
// schedule builds each step as a set of slots, at most one per residue, that
// every lane of the group holds among its unvisited entries: residues are
// taken in descending remaining demand (the sum over their slots of the
// largest number of visits a lane still owes the slot), and for each the slot
// held by the most lanes not yet served at this step (then the larger
// demand, then the smaller slot).  Each lane takes, among the step's slots it
// holds, the one of the most-demanded residue (then its own larger count, then
// the smaller slot); a lane holding none takes its entry of the most-demanded
// residue (a conflict).  Ties are broken by slot values only, so the order is
// deterministic.  One warp per group; its lanes' lists (CSR order, written by
// k_local_ell) are read into a shared-memory hash table of slot -> per-lane
// counts and then overwritten in place, step by step.  Every lane of the group
// emits exactly the multiset of entries it was given.
struct EllSchedSmem {
    static size_t bytes(int H, int G) {
        return (size_t)H * 2 + (size_t)H * G + (size_t)H + (size_t)H * 2 + 4 * 4 * 17;
    }
};

template <int G>
__device__ __forceinline__ unsigned ell_lane_mask(const uint32_t *cw, int nvalid) {
    unsigned m = 0u;
#pragma unroll
    for (int w = 0; w < G / 4; ++w) {
        const uint32_t x = cw[w];
#pragma unroll
        for (int b = 0; b < 4; ++b)
            if ((x >> (8 * b)) & 0xffu) m |= 1u << (4 * w + b);
    }
    return m & ((1u << nvalid) - 1u);
}

template <int G>
__device__ __forceinline__ int ell_lane_max(const uint32_t *cw) {
    int mx = 0;
#pragma unroll
    for (int w = 0; w < G / 4; ++w) {
        const uint32_t x = cw[w];
#pragma unroll
        for (int b = 0; b < 4; ++b) mx = max(mx, (int)((x >> (8 * b)) & 0xffu));
    }
    return mx;
}

template <int G>
__global__ void __launch_bounds__(32) k_ell_schedule(uint16_t *lell, const long long *loff,
                                                     const int32_t *tw, int T, long long n,
                                                     long long ngroups, int lgH) {
    constexpr int M = G;                 // residues
    constexpr int CW = G / 4;            // count words per table entry
    constexpr uint16_t kEmpty = 0xffffu;
    extern __shared__ __align__(16) unsigned char smem[];
    const int H = 1 << lgH;
    uint32_t *cnt = reinterpret_cast<uint32_t *>(smem);                 // H x CW
    uint16_t *key = reinterpret_cast<uint16_t *>(cnt + (size_t)H * CW); // H
    uint16_t *bidx = key + H;                                           // H (bucketed entries)
    uint8_t *umx = reinterpret_cast<uint8_t *>(bidx + H);               // H
    int *boff = reinterpret_cast<int *>(umx + ((H + 15) & ~15));        // M + 1
    int *bfill = boff + (M + 1);                                        // M
    int *dem = bfill + M;                                               // M
    int *sel = dem + M;                                                 // M
    const int lane = threadIdx.x;
    const unsigned full = 0xffffffffu;
    const int nq = T / G;
    for (long long gq = blockIdx.x; gq < ngroups; gq += gridDim.x) {
        const long long t = gq / nq;
        const int q = (int)(gq - t * nq);
        const int W = tw[t];
        const long long first = t * (long long)T + (long long)q * G;
        const int nvalid = (int)min((long long)G, n - first);
        if (W <= 1 || W > kEllOrderCap || nvalid <= 0) continue;
        uint16_t *base = lell + loff[t] + (long long)q * G;
        for (int h = lane; h < H; h += 32) {
            key[h] = kEmpty;
            umx[h] = 0;
#pragma unroll
            for (int w = 0; w < CW; ++w) cnt[h * CW + w] = 0u;
        }
        if (lane < M) {
            bfill[lane] = 0;
            dem[lane] = 0;
            sel[lane] = -1;
        }
        __syncwarp();
        // lists -> table of slot -> per-lane counts (linear probing; the table
        // holds at least twice the entries, so a free cell always exists)
        const int ne = nvalid * W;
        for (int e = lane; e < ne; e += 32) {
            const int k = e / W, j = e - k * W;
            const uint16_t s = base[(long long)j * T + k];
            unsigned h = ((unsigned)s * 0x9E3779B1u) >> (32 - lgH);
            for (int probe = 0; probe < H; ++probe) {
                const unsigned short old = atomicCAS(reinterpret_cast<unsigned short *>(key + h),
                                                     (unsigned short)kEmpty, (unsigned short)s);
                if (old == kEmpty || old == s) break;
                h = (h + 1) & (unsigned)(H - 1);
            }
            atomicAdd(cnt + h * CW + (k >> 2), 1u << (8 * (k & 3)));
        }
        __syncwarp();
        // bucket the occupied cells by residue; initial demand per residue
        for (int h = lane; h < H; h += 32)
            if (key[h] != kEmpty) atomicAdd(bfill + (key[h] % M), 1);
        __syncwarp();
        if (lane == 0) {
            int acc = 0;
            for (int r = 0; r < M; ++r) {
                boff[r] = acc;
                acc += bfill[r];
                bfill[r] = 0;
            }
            boff[M] = acc;
        }
        __syncwarp();
        for (int h = lane; h < H; h += 32)
            if (key[h] != kEmpty) {
                const int r = key[h] % M;
                bidx[boff[r] + atomicAdd(bfill + r, 1)] = (uint16_t)h;
                const int mx = ell_lane_max<G>(cnt + h * CW);
                umx[h] = (uint8_t)mx;
                atomicAdd(dem + r, mx);
            }
        __syncwarp();
        for (int j = 0; j < W; ++j) {
            int dm[M];
#pragma unroll
            for (int r = 0; r < M; ++r) dm[r] = dem[r];
            unsigned unc = (1u << nvalid) - 1u, taken = 0u;
            // the step's slots: residues by descending demand (then index)
            for (int it = 0; it < M && unc; ++it) {
                int r = -1, best = -1;
#pragma unroll
                for (int rr = 0; rr < M; ++rr)
                    if (!((taken >> rr) & 1u) && dm[rr] > best) {
                        best = dm[rr];
                        r = rr;
                    }
                taken |= 1u << r;
                unsigned bk = 0u, bm = 0u;
                int bh = -1;
                for (int x = boff[r] + lane; x < boff[r + 1]; x += 32) {
                    const int h = bidx[x];
                    const unsigned m = ell_lane_mask<G>(cnt + h * CW, nvalid) & unc;
                    if (!m) continue;
                    const unsigned kk = ((unsigned)__popc(m) << 24) | ((unsigned)umx[h] << 16) |
                                        (unsigned)(0xffffu - key[h]);
                    if (kk > bk) {
                        bk = kk;
                        bh = h;
                        bm = m;
                    }
                }
                const unsigned wk = __reduce_max_sync(full, bk);
                if (wk == 0u) continue;
                const unsigned src = __ffs(__ballot_sync(full, bk == wk)) - 1;
                bh = __shfl_sync(full, bh, src);
                bm = __shfl_sync(full, bm, src);
                if (lane == 0) sel[r] = bh;
                unc &= ~bm;
            }
            __syncwarp();
            // each lane of the group takes its entry of this step
            int pick = -1;
            if (lane < nvalid) {
                const int byte = 8 * (lane & 3), word = lane >> 2;
                unsigned long long bk = 0ull;
#pragma unroll
                for (int r = 0; r < M; ++r) {
                    const int h = sel[r];
                    if (h < 0) continue;
                    const unsigned c = (cnt[h * CW + word] >> byte) & 0xffu;
                    if (!c) continue;
                    const unsigned long long kk = ((unsigned long long)(dm[r] + 1) << 32) |
                                                  ((unsigned long long)c << 16) |
                                                  (unsigned long long)(0xffffu - key[h]);
                    if (kk > bk) {
                        bk = kk;
                        pick = h;
                    }
                }
                if (pick < 0) {   // no slot of this step: a conflict
                    for (int x = 0; x < boff[M]; ++x) {
                        const int h = bidx[x];
                        const unsigned c = (cnt[h * CW + word] >> byte) & 0xffu;
                        if (!c) continue;
                        const unsigned long long kk = ((unsigned long long)(dm[key[h] % M] + 1) << 32) |
                                                      ((unsigned long long)c << 16) |
                                                      (unsigned long long)(0xffffu - key[h]);
                        if (kk > bk) {
                            bk = kk;
                            pick = h;
                        }
                    }
                }
                base[(long long)j * T + lane] = key[pick];
                atomicSub(cnt + pick * CW + word, 1u << byte);
            }
            __syncwarp();
            // new demand of the slots taken (one lane per distinct slot)
            const unsigned same = __match_any_sync(full, pick);
            if (pick >= 0 && lane == __ffs(same) - 1) {
                const int mx = ell_lane_max<G>(cnt + pick * CW);
                const int d = (int)umx[pick] - mx;
                if (d) {
                    umx[pick] = (uint8_t)mx;
                    atomicSub(dem + key[pick] % M, d);
                }
            }
            if (lane < M) sel[lane] = -1;
            __syncwarp();
        }
        __syncwarp();
    }
}

__global__ void k_group_max(const long long *lvl_pair, const int32_t *grp_lvl, long long ng,
                            unsigned int *mx) {
    long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g >= ng) return;
    atomicMax(mx, (unsigned int)(lvl_pair[grp_lvl[g + 1]] - lvl_pair[grp_lvl[g]]));
    atomicMax(mx + 1, (unsigned int)(grp_lvl[g + 1] - grp_lvl[g]));
}

__global__ void k_level_max(const long long *lvl_pair, long long nlev, unsigned int *mx) {
    long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (L < nlev) atomicMax(mx, (unsigned int)(lvl_pair[L + 1] - lvl_pair[L]));
}

__global__ void k_col_off(const int32_t *gcol, long long ng, int ncol, int *col_off) {
    long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g > ng) return;
    int cprev = g == 0 ? -1 : gcol[g - 1];
    int cnow = g == ng ? ncol : gcol[g];
    for (int c = cprev + 1; c <= cnow; ++c) col_off[c] = (int)g;
}

__global__ void k_minus_one(const long long *in, long long m, long long *out) {
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p < m) out[p] = in[p] - 1;
}

// ---------------------------------------------------------------- helpers
struct Tmp {
    mts_ctx *ctx;
    std::vector<void *> ptrs;
    ~Tmp() {
        for (void *p : ptrs) dfree(ctx, p);
    }
    template <class T>
    T *get(size_t count) {
        void *p = dalloc(ctx, count * sizeof(T) + 16);
        if (p && (reinterpret_cast<uintptr_t>(p) & 15u)) {   // see dalloc_into
            dfree(ctx, p);
            p = nullptr;
        }
        if (p) ptrs.push_back(p);
        return (T *)p;
    }
};

#define NEED(p)                                                  \
    do {                                                         \
        if (!(p)) {                                              \
            set_error("device allocation failed (%s)", #p);      \
            return MTS_ERR_OOM;                                  \
        }                                                        \
    } while (0)

template <class T>
mts_status cub_excl_sum(Tmp &tmp, const T *in, T *out, long long m, cudaStream_t st) {
    size_t bytes = 0;
    MTS_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, bytes, in, out, m, st));
    void *t = tmp.get<char>(bytes);
    NEED(t);
    MTS_CUDA(cub::DeviceScan::ExclusiveSum(t, bytes, in, out, m, st));
    return MTS_OK;
}

template <class T>
mts_status cub_incl_sum(Tmp &tmp, const T *in, T *out, long long m, cudaStream_t st) {
    size_t bytes = 0;
    MTS_CUDA(cub::DeviceScan::InclusiveSum(nullptr, bytes, in, out, m, st));
    void *t = tmp.get<char>(bytes);
    NEED(t);
    MTS_CUDA(cub::DeviceScan::InclusiveSum(t, bytes, in, out, m, st));
    return MTS_OK;
}

mts_status cub_sort_pairs(Tmp &tmp, const unsigned long long *kin, unsigned long long *kout,
                          const long long *vin, long long *vout, long long m, int end_bit,
                          cudaStream_t st) {
    size_t bytes = 0;
    MTS_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, bytes, kin, kout, vin, vout, m, 0, end_bit, st));
    void *t = tmp.get<char>(bytes);
    NEED(t);
    MTS_CUDA(cub::DeviceRadixSort::SortPairs(t, bytes, kin, kout, vin, vout, m, 0, end_bit, st));
    return MTS_OK;
}

template <class T>
mts_status to_host(T *h, const T *d, size_t count, cudaStream_t st) {
    MTS_CUDA(cudaMemcpyAsync(h, d, count * sizeof(T), cudaMemcpyDeviceToHost, st));
    MTS_CUDA(cudaStreamSynchronize(st));
    return MTS_OK;
}

mts_status build_tiles(mts_body *b, Tmp &tmp, cudaStream_t st, int T) {
    if (T < 64 || T > 512) {   // the force partials buffer holds one slot per 64 particles
        set_error("tile size %d outside [64, 512]", T);
        return MTS_ERR_STATE;
    }
    mts_ctx *ctx = b->ctx;
    const long long n = b->n;
    const long long ntiles = (n + T - 1) / T;
    const long long m = b->nnz + n;
    int32_t *vals = tmp.get<int32_t>(m), *vs = tmp.get<int32_t>(m);
    long long *seg = tmp.get<long long>(ntiles + 1);
    long long *flag = tmp.get<long long>(m), *scan = tmp.get<long long>(m);
    NEED(vals); NEED(vs); NEED(seg); NEED(flag); NEED(scan);
    k_tile_entries<<<grid_for(n), TPB, 0, st>>>(b->nb_off, b->nb_idx, n, vals);
    k_tile_seg<<<grid_for(ntiles + 1), TPB, 0, st>>>(b->nb_off, n, T, ntiles, seg);
    {
        size_t bytes = 0;
        MTS_CUDA(cub::DeviceSegmentedSort::SortKeys(nullptr, bytes, vals, vs, m, ntiles, seg, seg + 1, st));
        void *t = tmp.get<char>(bytes);
        NEED(t);
        MTS_CUDA(cub::DeviceSegmentedSort::SortKeys(t, bytes, vals, vs, m, ntiles, seg, seg + 1, st));
    }
    k_uniq_flags<<<grid_for(m), TPB, 0, st>>>(vs, m, flag);
    k_seg_start_flags<<<grid_for(ntiles), TPB, 0, st>>>(seg, ntiles, flag);
    MTS_TRY(cub_incl_sum(tmp, flag, scan, m, st));
    long long total = 0;
    MTS_TRY(to_host(&total, scan + m - 1, 1, st));
    MTS_TRY(dalloc_t(ctx, &b->halo_idx, total));
    MTS_TRY(dalloc_t(ctx, &b->halo_off, ntiles + 1));
    k_halo_compact<<<grid_for(m), TPB, 0, st>>>(vs, flag, scan, m, b->halo_idx);
    unsigned int *hmax = tmp.get<unsigned int>(1);
    NEED(hmax);
    MTS_CUDA(cudaMemsetAsync(hmax, 0, sizeof(unsigned), st));
    k_halo_off<<<grid_for(ntiles + 1), TPB, 0, st>>>(seg, scan, ntiles, total, b->halo_off, hmax);
    unsigned int hm = 0;
    MTS_TRY(to_host(&hm, hmax, 1, st));
    if (hm > 65535) {
        set_error("tile halo of %u particles exceeds the 16-bit local index", hm);
        return MTS_ERR_INVALID_ARG;
    }
    b->max_halo = (int)hm;
    {
        const int P = b->dim == 2 ? 2 : 4;
        MTS_TRY(dalloc_into(ctx, &b->halo_x, (size_t)total * P * b->rsize + 16));
        if (b->rsize == 8) {
            if (P == 2)
                k_halo_x<double, 2><<<grid_for(total), TPB, 0, st>>>(b->halo_off, b->halo_idx, ntiles, T, total, b->X64, (double *)b->halo_x);
            else
                k_halo_x<double, 4><<<grid_for(total), TPB, 0, st>>>(b->halo_off, b->halo_idx, ntiles, T, total, b->X64, (double *)b->halo_x);
        } else {
            if (P == 2)
                k_halo_x<float, 2><<<grid_for(total), TPB, 0, st>>>(b->halo_off, b->halo_idx, ntiles, T, total, b->X64, (float *)b->halo_x);
            else
                k_halo_x<float, 4><<<grid_for(total), TPB, 0, st>>>(b->halo_off, b->halo_idx, ntiles, T, total, b->X64, (float *)b->halo_x);
        }
    }
    long long *w = tmp.get<long long>(ntiles + 1);
    NEED(w);
    MTS_TRY(dalloc_t(ctx, &b->lell_off, ntiles + 1));
    MTS_TRY(dalloc_t(ctx, &b->tile_w, ntiles + 1));
    unsigned int *wmx = tmp.get<unsigned int>(1);
    NEED(wmx);
    MTS_CUDA(cudaMemsetAsync(wmx, 0, sizeof(unsigned), st));
    k_tile_w<<<grid_for(ntiles), TPB, 0, st>>>(b->nb_off, n, T, ntiles, w, wmx);
    MTS_CUDA(cudaMemsetAsync(w + ntiles, 0, sizeof(long long), st));
    MTS_TRY(cub_excl_sum(tmp, w, b->lell_off, ntiles + 1, st));
    long long len = 0;
    MTS_TRY(to_host(&len, b->lell_off + ntiles, 1, st));
    MTS_TRY(dalloc_t(ctx, &b->lell, std::max(len, 1LL)));
    MTS_TRY(dalloc_t(ctx, &b->lself, n));
    k_local_ell<<<grid_for(ntiles * T), TPB, 0, st>>>(b->nb_off, b->nb_idx, n, T, ntiles,
                                                        b->halo_off, b->halo_idx, b->lell_off,
                                                        b->tile_w, b->lell, b->lself);
    unsigned int wmax = 0;
    MTS_TRY(to_host(&wmax, wmx, 1, st));
    if (wmax > 1) {
        const int G = b->dim == 2 ? 16 : 8;
        int lgH = 6;
        while ((1 << lgH) < 2 * G * (int)wmax) ++lgH;
        const size_t sm = EllSchedSmem::bytes(1 << lgH, G);
        const long long ngroups = ntiles * (T / G);
        const unsigned grid = (unsigned)std::min(ngroups, 1LL << 20);
        if (G == 16) {
            MTS_CUDA(cudaFuncSetAttribute(k_ell_schedule<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            k_ell_schedule<16><<<grid, 32, sm, st>>>(b->lell, b->lell_off, b->tile_w, T, n, ngroups, lgH);
        } else {
            MTS_CUDA(cudaFuncSetAttribute(k_ell_schedule<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            k_ell_schedule<8><<<grid, 32, sm, st>>>(b->lell, b->lell_off, b->tile_w, T, n, ngroups, lgH);
        }
        MTS_CUDA(cudaGetLastError());
    }
    b->T = T;
    b->ntiles = ntiles;
    return MTS_OK;
}

// release the damping-order arrays of a layout that did not fit
void free_damping(mts_body *b) {
    void **ptrs[] = {(void **)&b->pair_a, (void **)&b->pair_b, (void **)&b->pair_col,
                     (void **)&b->pair_sub, (void **)&b->pair_key, (void **)&b->pair_ab,
                     (void **)&b->pair_g, (void **)&b->lvl_pair, (void **)&b->grp_lvl,
                     (void **)&b->touch_start, (void **)&b->touch_cnt, (void **)&b->pair_slot,
                     (void **)&b->kpad_ab, (void **)&b->kpad_g, (void **)&b->bperm,
                     (void **)&b->bflags, (void **)&b->grp_cons};
    for (void **pp : ptrs) {
        dfree(b->ctx, *pp);
        *pp = nullptr;
    }
}

// The canonical damping order for the layout in b->ax_shift / b->level_cap.
// *no_fit is set (with MTS_ERR_INVALID_ARG) when the CTA-per-group kernel of
// the wide layout cannot stage an owner group.
template <class R, int D>
mts_status build_damping(mts_body *b, Tmp &tmp, cudaStream_t st, const int *cell, bool *no_fit) {
    mts_ctx *ctx = b->ctx;
    const long long n = b->n;
    const bool wide = b->damp_layout == MTS_DAMP_WIDE;
    const Shifts sh{{b->ax_shift[0], b->ax_shift[1], b->ax_shift[2]}};
    int nblocked = 0;
    for (int k = 0; k < D; ++k) nblocked += b->ax_shift[k] < kWholeAxis;
    const int nbk = 1 << D, nbw = 1 << nblocked;
    *no_fit = false;

    // owned pairs, keyed by (colour, owner block)
    long long *pcnt = tmp.get<long long>(n + 1), *poff = tmp.get<long long>(n + 1);
    NEED(pcnt); NEED(poff);
    k_count_pairs<<<grid_for(n), TPB, 0, st>>>(b->nb_off, b->nb_idx, n, pcnt);
    MTS_CUDA(cudaMemsetAsync(pcnt + n, 0, sizeof(long long), st));
    MTS_TRY(cub_excl_sum(tmp, pcnt, poff, n + 1, st));
    long long m = 0;
    MTS_TRY(to_host(&m, poff + n, 1, st));
    b->npairs = m;
    if (m * 2 != b->nnz) {
        set_error("neighbour lists are not symmetric (%lld pairs, %lld entries)", m, b->nnz);
        return MTS_ERR_STATE;
    }
    const long long mm = std::max(m, 1LL);
    int32_t *pa0 = tmp.get<int32_t>(mm), *pb0 = tmp.get<int32_t>(mm);
    unsigned long long *pk0 = tmp.get<unsigned long long>(mm), *pk1 = tmp.get<unsigned long long>(mm);
    long long *ord = tmp.get<long long>(mm), *ord1 = tmp.get<long long>(mm);
    NEED(pa0); NEED(pb0); NEED(pk0); NEED(pk1); NEED(ord); NEED(ord1);
    k_fill_pairs<<<grid_for(n), TPB, 0, st>>>(b->nb_off, b->nb_idx, cell, n, D, sh, poff, pa0, pb0,
                                              pk0);
    k_iota<<<grid_for(m), TPB, 0, st>>>(ord, m);
    MTS_TRY(cub_sort_pairs(tmp, pk0, pk1, ord, ord1, m, 63, st));
    int32_t *pa1 = tmp.get<int32_t>(mm), *pb1 = tmp.get<int32_t>(mm);
    NEED(pa1); NEED(pb1);
    k_gather<<<grid_for(m), TPB, 0, st>>>(pa0, ord1, m, pa1);
    k_gather<<<grid_for(m), TPB, 0, st>>>(pb0, ord1, m, pb1);

    // owner groups
    long long *flag = tmp.get<long long>(mm), *gscan = tmp.get<long long>(mm);
    NEED(flag); NEED(gscan);
    k_run_flags<<<grid_for(m), TPB, 0, st>>>(pk1, m, flag);
    MTS_TRY(cub_incl_sum(tmp, flag, gscan, m, st));
    long long ng = 0;
    if (m > 0) MTS_TRY(to_host(&ng, gscan + m - 1, 1, st));
    b->n_groups = ng;
    const long long ngg = std::max(ng, 1LL);
    long long *gstart = tmp.get<long long>(ngg + 1);
    NEED(gstart);
    k_run_starts<<<grid_for(m), TPB, 0, st>>>(gscan, m, gstart);

    // block table over the block-sorted order (stable by block key; with the
    // same shift on every axis the Morton order is already block-sorted, so
    // the permutation is the identity there)
    unsigned long long *bkp = tmp.get<unsigned long long>(n), *bks = tmp.get<unsigned long long>(n);
    long long *io = tmp.get<long long>(n), *bp64 = tmp.get<long long>(n);
    long long *bflag = tmp.get<long long>(n), *bscan = tmp.get<long long>(n);
    int32_t *binv = tmp.get<int32_t>(n);
    NEED(bkp); NEED(bks); NEED(io); NEED(bp64); NEED(bflag); NEED(bscan); NEED(binv);
    k_block_keys<<<grid_for(n), TPB, 0, st>>>(cell, n, D, sh, bkp);
    k_iota<<<grid_for(n), TPB, 0, st>>>(io, n);
    MTS_TRY(cub_sort_pairs(tmp, bkp, bks, io, bp64, n, 64, st));
    MTS_TRY(dalloc_t(ctx, &b->bperm, n));
    k_to_i32<<<grid_for(n), TPB, 0, st>>>(bp64, n, b->bperm);
    k_inverse<int32_t><<<grid_for(n), TPB, 0, st>>>(bp64, n, binv);
    k_run_flags<<<grid_for(n), TPB, 0, st>>>(bks, n, bflag);
    MTS_TRY(cub_incl_sum(tmp, bflag, bscan, n, st));
    long long nblocks = 0;
    MTS_TRY(to_host(&nblocks, bscan + n - 1, 1, st));
    long long *bstart = tmp.get<long long>(nblocks + 1);
    unsigned long long *bkey = tmp.get<unsigned long long>(nblocks + 1);
    int *bcnt = tmp.get<int>(nblocks + 1);
    unsigned int *dmb = tmp.get<unsigned int>(1);
    NEED(bstart); NEED(bkey); NEED(bcnt); NEED(dmb);
    k_run_starts<<<grid_for(n), TPB, 0, st>>>(bscan, n, bstart);
    MTS_CUDA(cudaMemsetAsync(dmb, 0, sizeof(unsigned), st));
    k_block_table<<<grid_for(nblocks), TPB, 0, st>>>(bstart, nblocks, n, bks, bkey, bcnt, dmb);
    unsigned int hmb = 0;
    MTS_TRY(to_host(&hmb, dmb, 1, st));
    if (wide) {
        // 16-bit slot indices of the staged velocities, one dummy slot spare
        if ((long long)hmb * nbw + 1 > 65535) {
            set_error("wide damping block holds %u particles; at most %d fit the 16-bit slot index",
                      hmb, 65534 / nbw);
            *no_fit = true;
            return MTS_ERR_INVALID_ARG;
        }
    } else if ((long long)hmb * nbk > 32767) {
        set_error("damping block holds %u particles; at most %d fit the 15-bit local index",
                  hmb, 32767 / nbk);
        return MTS_ERR_INVALID_ARG;
    }
    b->mb = (int)hmb;
    b->nbw = nbw;

    int32_t *gcol = tmp.get<int32_t>(ngg);
    long long *gkey = tmp.get<long long>(ngg);
    NEED(gcol); NEED(gkey);
    MTS_TRY(dalloc_t(ctx, &b->touch_start, ngg * nbk));
    MTS_TRY(dalloc_t(ctx, &b->touch_cnt, ngg * nbk));
    k_touch<<<grid_for(ng), TPB, 0, st>>>(gstart, ng, pa1, pb1, cell, D, sh, bkey, bstart, bcnt,
                                           nblocks, b->touch_start, b->touch_cnt, gcol, gkey);

    // visit order of the greedy: owner group, offset class, then (a, b)
    const int Rr = (int)std::floor(2.0 * b->h / b->dx) + 1;
    if (std::pow(2.0 * Rr + 1.0, (double)D) > 65536.0) {
        set_error("smoothing length of %.3g cells: offset classes exceed 16 bits", b->h / b->dx);
        return MTS_ERR_INVALID_ARG;
    }
    int32_t *pa2 = tmp.get<int32_t>(mm), *pb2 = tmp.get<int32_t>(mm);
    long long *ord3 = tmp.get<long long>(mm);
    NEED(pa2); NEED(pb2); NEED(ord3);
    {
        unsigned long long *k3 = tmp.get<unsigned long long>(mm), *k3s = tmp.get<unsigned long long>(mm);
        long long *io3 = tmp.get<long long>(mm);
        NEED(k3); NEED(k3s); NEED(io3);
        k_pair_class<<<grid_for(m), TPB, 0, st>>>(pa1, pb1, gscan, m, cell, D, Rr, k3);
        k_iota<<<grid_for(m), TPB, 0, st>>>(io3, m);
        int gb3 = 1;
        while ((1LL << gb3) <= ng) ++gb3;
        MTS_TRY(cub_sort_pairs(tmp, k3, k3s, io3, ord3, m, std::min(64, gb3 + 16), st));
        k_gather<<<grid_for(m), TPB, 0, st>>>(pa1, ord3, m, pa2);
        k_gather<<<grid_for(m), TPB, 0, st>>>(pb1, ord3, m, pb2);
    }

    // greedy sub-colours, in batches of groups to bound the bitmask scratch
    int32_t *sub0 = tmp.get<int32_t>(mm), *nsub = tmp.get<int32_t>(ngg + 1);
    uint32_t *ab0 = tmp.get<uint32_t>(mm);
    int32_t *subc = tmp.get<int32_t>(mm);
    uint32_t *abc = tmp.get<uint32_t>(mm);
    NEED(sub0); NEED(nsub); NEED(ab0); NEED(subc); NEED(abc);
    long long per_group = (long long)nbw * b->mb * 4;   // 64-bit words
    long long batch = std::max(1LL, std::min(ng, (1LL << 25) / std::max(per_group, 1LL)));
    unsigned long long *used = tmp.get<unsigned long long>(batch * per_group + 1);
    NEED(used);
    for (long long gs = 0; gs < ng; gs += batch) {
        long long ge = std::min(ng, gs + batch);
        MTS_CUDA(cudaMemsetAsync(used, 0, (ge - gs) * per_group * sizeof(unsigned long long), st));
        k_greedy<<<grid_for(ge - gs, 64), 64, 0, st>>>(gstart, gs, ge, ng, m, pa2, pb2, cell, D, sh,
                                                         b->touch_start, binv, b->mb, nbw,
                                                         b->level_cap, used, subc, abc, nsub,
                                                         b->ctrl);
    }
    // back to (group, a, b) order, so that the final stable sort by
    // (group, sub-colour) lists each level in ascending (a, b)
    k_scatter<<<grid_for(m), TPB, 0, st>>>(subc, ord3, m, sub0);
    k_scatter<<<grid_for(m), TPB, 0, st>>>(abc, ord3, m, ab0);

    // final canonical order: (group, sub-colour), stable
    unsigned long long *k2 = tmp.get<unsigned long long>(mm), *k2s = tmp.get<unsigned long long>(mm);
    NEED(k2); NEED(k2s);
    k_group_of_pair<<<grid_for(m), TPB, 0, st>>>(gscan, m, sub0, k2);
    k_iota<<<grid_for(m), TPB, 0, st>>>(ord, m);
    int gbits = 1;
    while ((1LL << gbits) <= ng) ++gbits;
    MTS_TRY(cub_sort_pairs(tmp, k2, k2s, ord, ord1, m, std::min(64, gbits + 8), st));
    MTS_TRY(dalloc_t(ctx, &b->pair_a, mm));
    MTS_TRY(dalloc_t(ctx, &b->pair_b, mm));
    MTS_TRY(dalloc_t(ctx, &b->pair_sub, mm));
    MTS_TRY(dalloc_t(ctx, &b->pair_col, mm));
    MTS_TRY(dalloc_t(ctx, &b->pair_key, mm));
    MTS_TRY(dalloc_t(ctx, &b->pair_ab, mm));
    MTS_TRY(dalloc_into(ctx, &b->pair_g, mm * sizeof(R) + 16));
    k_gather<<<grid_for(m), TPB, 0, st>>>(pa1, ord1, m, b->pair_a);
    k_gather<<<grid_for(m), TPB, 0, st>>>(pb1, ord1, m, b->pair_b);
    k_gather<<<grid_for(m), TPB, 0, st>>>(sub0, ord1, m, b->pair_sub);
    k_gather<<<grid_for(m), TPB, 0, st>>>(ab0, ord1, m, b->pair_ab);
    // per-pair colour and owner key from the group of each final pair
    {
        long long *gid = tmp.get<long long>(mm), *g0i = tmp.get<long long>(mm);
        NEED(gid); NEED(g0i);
        k_gather<<<grid_for(m), TPB, 0, st>>>(gscan, ord1, m, gid);   // 1-based group ids
        k_minus_one<<<grid_for(m), TPB, 0, st>>>(gid, m, g0i);
        k_gather<<<grid_for(m), TPB, 0, st>>>(gcol, g0i, m, b->pair_col);
        k_gather<<<grid_for(m), TPB, 0, st>>>(gkey, g0i, m, b->pair_key);
    }

    // levels
    MTS_TRY(dalloc_t(ctx, &b->grp_lvl, ngg + 1));
    MTS_CUDA(cudaMemsetAsync(nsub + ng, 0, sizeof(int32_t), st));
    MTS_TRY(cub_excl_sum(tmp, nsub, b->grp_lvl, ng + 1, st));
    int nlev = 0;
    MTS_TRY(to_host(&nlev, b->grp_lvl + ng, 1, st));
    b->n_levels = nlev;
    MTS_TRY(dalloc_t(ctx, &b->lvl_pair, (long long)nlev + 1));
    k_levels<<<grid_for(m + 1), TPB, 0, st>>>(k2s, m, b->grp_lvl, b->lvl_pair, nlev);
    k_pair_coef<R, D><<<grid_for(m), TPB, 0, st>>>(b->pair_a, b->pair_b, m, b->X64, b->h,
                                                    kernel_alpha(D, b->h), b->V, (R *)b->pair_g);
    {
        unsigned int *mx = tmp.get<unsigned int>(3);
        NEED(mx);
        MTS_CUDA(cudaMemsetAsync(mx, 0, 3 * sizeof(unsigned), st));
        k_group_max<<<grid_for(ng), TPB, 0, st>>>(b->lvl_pair, b->grp_lvl, ng, mx);
        k_level_max<<<grid_for(nlev), TPB, 0, st>>>(b->lvl_pair, nlev, mx + 2);
        unsigned int hm[3];
        MTS_TRY(to_host(hm, mx, 3, st));
        b->max_group_pairs = (int)hm[0];
        b->max_group_levels = (int)hm[1];
        b->max_level_pairs = (int)hm[2];
    }
    if (wide) {
        const size_t need = damp_wide_smem(b);
        if (need > 227 * 1024) {
            set_error("wide damping needs %zu bytes of shared memory per owner group "
                      "(block %d particles, %d levels of up to %d pairs)", need, b->mb,
                      b->max_group_levels, b->max_level_pairs);
            *no_fit = true;
            return MTS_ERR_INVALID_ARG;
        }
        // the kernel streams the canonical order: pair words hold slot
        // indices, coefficients carry the constrained-pair sign
        MTS_TRY(dalloc_t(ctx, &b->pair_slot, mm));
        MTS_TRY(dalloc_t(ctx, &b->kpad_ab, mm));
        MTS_TRY(dalloc_into(ctx, &b->kpad_g, mm * sizeof(R) + 16));
        k_iota<<<grid_for(m), TPB, 0, st>>>(b->pair_slot, m);
        MTS_TRY(dalloc_t(ctx, &b->bflags, n));
        MTS_CUDA(cudaMemsetAsync(b->bflags, 0, n, st));   // flags start at zero
        MTS_CUDA(cudaMemcpyAsync(b->kpad_ab, b->pair_ab, m * sizeof(uint32_t),
                                 cudaMemcpyDeviceToDevice, st));
        MTS_CUDA(cudaMemcpyAsync(b->kpad_g, b->pair_g, m * sizeof(R), cudaMemcpyDeviceToDevice, st));
    } else {
        // padded per-level layout for the warp-per-group kernel (32 slots per level)
        const long long ns = 32LL * nlev;
        MTS_TRY(dalloc_t(ctx, &b->pair_slot, mm));
        MTS_TRY(dalloc_t(ctx, &b->kpad_ab, std::max(ns, 4LL)));
        MTS_TRY(dalloc_into(ctx, &b->kpad_g, std::max(ns, 4LL) * sizeof(R) + 16));
        const int bps = Pad<D>::v * (int)sizeof(R);
        // byte offset of the dummy slot; every slot position fits 16 bits
        const long long dummy = (long long)damp_slot_pos(nbk * b->mb, bps) * bps;
        if ((long long)(damp_slot_count(nbk * b->mb) - 1) * bps > 65535) {
            set_error("damping blocks too large for 16-bit byte offsets (%d particles)", b->mb);
            return MTS_ERR_INVALID_ARG;
        }
        k_fill_dummy<<<grid_for(std::max(ns, 4LL)), TPB, 0, st>>>(b->kpad_ab, std::max(ns, 4LL),
                                                                 (uint32_t)dummy);
        MTS_CUDA(cudaMemsetAsync(b->kpad_g, 0, std::max(ns, 4LL) * sizeof(R), st));
        int8_t *lane = tmp.get<int8_t>(mm);
        NEED(lane);
        k_level_lanes<<<grid_for(nlev), TPB, 0, st>>>(b->lvl_pair, nlev, b->pair_ab, bps, lane);
        k_fill_slots<<<grid_for(m), TPB, 0, st>>>(k2s, m, b->grp_lvl, b->lvl_pair, b->pair_ab,
                                                  lane, b->pair_slot, b->kpad_ab, bps);
        k_fill_slot_g<R><<<grid_for(m), TPB, 0, st>>>((const R *)b->pair_g, b->pair_slot, m,
                                                       (R *)b->kpad_g);
        if (bps == 16)
            k_fill_empty<<<grid_for(nlev), TPB, 0, st>>>(b->kpad_ab, nlev,
                                                         (uint32_t)dummy | ((uint32_t)dummy << 16));
        MTS_TRY(dalloc_t(ctx, &b->grp_cons, ngg));
        MTS_CUDA(cudaMemsetAsync(b->grp_cons, 0, ngg, st));   // flags start at zero
    }
    int *dcol = tmp.get<int>(16);
    NEED(dcol);
    k_col_off<<<grid_for(ng + 1), TPB, 0, st>>>(gcol, ng, nbk, dcol);
    MTS_TRY(to_host(b->col_off, dcol, nbk + 1, st));
    return MTS_OK;
}

// layout of the damping order: every axis blocked (cap 32 pairs per level),
// or axis k_whole unblocked (no cap)
void set_layout(mts_body *b, int layout, int k_whole) {
    b->damp_layout = layout;
    for (int k = 0; k < 3; ++k)
        b->ax_shift[k] = (layout == MTS_DAMP_WIDE && k == k_whole) ? kWholeAxis : b->blk_shift;
    b->level_cap = layout == MTS_DAMP_WIDE ? 0 : kLevelCap;
}

template <class R, int D>
mts_status build_typed(mts_body *b, const double *hX) {
    mts_ctx *ctx = b->ctx;
    cudaStream_t st = ctx->stream;
    const long long n = b->n;
    constexpr int P = Pad<D>::v;
    Tmp tmp{ctx, {}};

    // -- reference positions to the device, extent and finiteness
    double *Xo = tmp.get<double>(n * D);
    NEED(Xo);
    MTS_CUDA(cudaMemcpyAsync(Xo, hX, n * D * sizeof(double), cudaMemcpyHostToDevice, st));
    int nb = (int)std::min<long long>(grid_for(n), 1024);
    double *part = tmp.get<double>(nb * 4 + 4);
    NEED(part);
    k_extent_partial<<<nb, TPB, 0, st>>>(Xo, n, D, part);
    k_extent_final<<<1, 32, 0, st>>>(part, nb, part + nb * 4);
    double ext[4];
    MTS_TRY(to_host(ext, part + nb * 4, 4, st));
    if (ext[3] != 0.0) {
        set_error("reference positions contain NaN or Inf");
        return MTS_ERR_INVALID_ARG;
    }
    for (int k = 0; k < 3; ++k) b->Xmin[k] = k < D ? ext[k] : 0.0;

    // -- Morton keys and stable sort
    unsigned long long *keys = tmp.get<unsigned long long>(n), *keys_s = tmp.get<unsigned long long>(n);
    long long *vals = tmp.get<long long>(n);
    unsigned long long *cmax = tmp.get<unsigned long long>(4);
    NEED(keys); NEED(keys_s); NEED(vals); NEED(cmax);
    MTS_CUDA(cudaMemsetAsync(cmax, 0, 4 * sizeof(unsigned long long), st));
    k_keys<<<grid_for(n), TPB, 0, st>>>(Xo, n, D, b->Xmin[0], b->Xmin[1], b->Xmin[2], b->dx, keys,
                                          vals, cmax);
    unsigned long long hcmax[4];
    MTS_TRY(to_host(hcmax, cmax, 4, st));
    long long g0 = (long long)hcmax[0] + 1, g1 = (long long)hcmax[1] + 1,
              g2 = D == 3 ? (long long)hcmax[2] + 1 : 1;
    long long bits = D == 2 ? 31 : 21;
    if (g0 >= (1LL << bits) || g1 >= (1LL << bits) || g2 >= (1LL << bits)) {
        set_error("body extent too large for the Morton key (%lld x %lld x %lld cells)", g0, g1, g2);
        return MTS_ERR_INVALID_ARG;
    }
    long long ncell = g0 * g1 * g2;
    if (ncell > std::max<long long>(64 * n, 1LL << 22)) {
        set_error("body too sparse for the dense cell grid (%lld cells for %lld particles)", ncell, n);
        return MTS_ERR_INVALID_ARG;
    }
    MTS_TRY(cub_sort_pairs(tmp, keys, keys_s, vals, b->perm, n, D * (int)bits + 1 > 64 ? 64 : D * (int)bits, st));

    int *cell = tmp.get<int>(n * 3);
    NEED(cell);
    k_apply_perm<R, D><<<grid_for(n), TPB, 0, st>>>(Xo, b->perm, n, b->Xmin[0], b->Xmin[1],
                                                    b->Xmin[2], b->dx, b->X64, (R *)b->X,
                                                    b->rank, cell);

    // -- neighbours
    int *cstart = tmp.get<int>(ncell), *cend = tmp.get<int>(ncell);
    NEED(cstart); NEED(cend);
    MTS_CUDA(cudaMemsetAsync(cstart, 0xff, ncell * sizeof(int), st));
    MTS_CUDA(cudaMemsetAsync(cend, 0xff, ncell * sizeof(int), st));
    k_cell_ranges<<<grid_for(n), TPB, 0, st>>>(keys_s, cell, n, g0, g1, cstart, cend);
    int reach = (int)std::floor(2.0 * b->h / b->dx) + 1;
    long long *deg = tmp.get<long long>(n + 1);
    NEED(deg);
    k_neigh<D, false><<<grid_for(n), TPB, 0, st>>>(b->X64, cell, n, g0, g1, g2, reach, b->cut2,
                                                     cstart, cend, deg, nullptr, nullptr);
    MTS_CUDA(cudaMemsetAsync(deg + n, 0, sizeof(long long), st));
    MTS_TRY(dalloc_t(ctx, &b->nb_off, n + 1));
    MTS_TRY(cub_excl_sum(tmp, deg, b->nb_off, n + 1, st));
    MTS_TRY(to_host(&b->nnz, b->nb_off + n, 1, st));
    if (b->nnz == 0) {
        set_error("no particle has a neighbour within 2h: every correction matrix is singular");
        return MTS_ERR_SINGULAR_B;
    }
    int32_t *idx_u = tmp.get<int32_t>(std::max(b->nnz, 1LL));
    NEED(idx_u);
    MTS_TRY(dalloc_t(ctx, &b->nb_idx, std::max(b->nnz, 1LL)));
    k_neigh<D, true><<<grid_for(n), TPB, 0, st>>>(b->X64, cell, n, g0, g1, g2, reach, b->cut2,
                                                    cstart, cend, nullptr, b->nb_off, idx_u);
    if (b->nnz > 0) {
        size_t bytes = 0;
        MTS_CUDA(cub::DeviceSegmentedSort::SortKeys(nullptr, bytes, idx_u, b->nb_idx, b->nnz, n,
                                                    b->nb_off, b->nb_off + 1, st));
        void *t = tmp.get<char>(bytes);
        NEED(t);
        MTS_CUDA(cub::DeviceSegmentedSort::SortKeys(t, bytes, idx_u, b->nb_idx, b->nnz, n,
                                                    b->nb_off, b->nb_off + 1, st));
    }

    // -- B0
    double alpha = kernel_alpha(D, b->h);
    MTS_CUDA(cudaMemsetAsync(&b->ctrl->err, 0, sizeof(unsigned), st));
    k_b0<R, D><<<grid_for(n), TPB, 0, st>>>(b->X64, b->nb_off, b->nb_idx, n, b->h, alpha, b->V,
                                             (R *)b->B0, b->ctrl);

    // -- damping order.  AUTO and BLOCKS take blocks on every axis (the faster
    // warp-per-group kernel on the workloads measured); WIDE unblocks the
    // shortest axis (ties to the higher axis) when an owner group fits one CTA.
    {
        const long long cells[3] = {g0, g1, g2};
        int kmin = 0;
        for (int k = 1; k < D; ++k)
            if (cells[k] <= cells[kmin]) kmin = k;
        const bool try_wide = b->damp_req == MTS_DAMP_WIDE;
        bool built = false;
        if (try_wide) {
            set_layout(b, MTS_DAMP_WIDE, kmin);
            bool no_fit = false;
            const mts_status s = build_damping<R, D>(b, tmp, st, cell, &no_fit);
            if (s == MTS_OK) {
                built = true;
            } else if (!(no_fit && b->damp_req == MTS_DAMP_AUTO)) {
                return s;
            } else {
                MTS_CUDA(cudaStreamSynchronize(st));
                free_damping(b);
            }
        }
        if (!built) {
            set_layout(b, MTS_DAMP_BLOCKS, 0);
            bool no_fit = false;
            MTS_TRY((build_damping<R, D>(b, tmp, st, cell, &no_fit)));
        }
    }
    // -- Morton tiles and their halos (particles + neighbours), local ELL
    MTS_TRY(build_tiles(b, tmp, st, b->tile_req > 0 ? b->tile_req : tile_particles<R>()));

    // -- setup errors
    unsigned err = 0;
    MTS_TRY(to_host(&err, &b->ctrl->err, 1, st));
    if (err & kErrSingular) {
        set_error("singular correction-matrix sum (a particle without enough neighbours)");
        return MTS_ERR_SINGULAR_B;
    }
    if (err & kErrTooMany) {
        set_error("damping sub-colouring needs more than 256 colours");
        return MTS_ERR_STATE;
    }
    MTS_CUDA(cudaStreamSynchronize(st));
    return MTS_OK;
}

}  // namespace

// Rebuild the Morton tiles with T particles per tile (the block size of the
// gather kernels); the previous tile arrays are released first.
mts_status retile(mts_body *b, int T) {
    cudaStream_t st = b->ctx->stream;
    MTS_CUDA(cudaStreamSynchronize(st));
    void **ptrs[] = {(void **)&b->halo_off, (void **)&b->halo_idx, (void **)&b->halo_x,
                     (void **)&b->lell_off, (void **)&b->tile_w, (void **)&b->lell,
                     (void **)&b->lself};
    for (void **pp : ptrs) {
        dfree(b->ctx, *pp);
        *pp = nullptr;
    }
    Tmp tmp{b->ctx, {}};
    MTS_TRY(build_tiles(b, tmp, st, T));
    MTS_CUDA(cudaStreamSynchronize(st));
    return MTS_OK;
}

double kernel_alpha(int dim, double h) {
    if (dim == 2) return 7.0 / (4.0 * M_PI * h * h);
    return 21.0 / (16.0 * M_PI * h * h * h);
}

mts_status build_body(mts_body *b, const double *hX) {
    if (b->precision == MTS_FP64)
        return b->dim == 2 ? build_typed<double, 2>(b, hX) : build_typed<double, 3>(b, hX);
    return b->dim == 2 ? build_typed<float, 2>(b, hX) : build_typed<float, 3>(b, hX);
}

}  // namespace mts
