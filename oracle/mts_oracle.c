/*
 * mts_oracle.c -- plain, serial, FP64 CPU oracle for the multi-time-step SPH
 * solid relaxation of Tang et al., "An explicit multi-time stepping algorithm
 * for multi-time scale coupling problems in SPH" (arXiv 2309.04010).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * benchmark's CPU-baseline leg may load this library.  The CUDA library never
 * calls it, shares no code, header, table or constant generator with it, and
 * this file includes nothing from the CUDA side.
 *
 * Everything is FP64, evaluated in plain loops in the order the paper states
 * the steps, compiled with -ffp-contract=off (no fused multiply-add) so that
 * the neighbour test is bit-reproducible.  No blocking, fusion or reordering
 * beyond what the definitions state.
 *
 * Readings of the paper where it is silent or garbled (the same readings are
 * implemented by the CUDA library):
 *   - kernel: Wendland C2 with h = h_over_dx * dx and support 2h (the paper
 *     only says "kernel function", Sec. 3.1);
 *   - grad_a W_ab = W'(r) (X_a - X_b) / r  (derivative with respect to X_a);
 *   - F is evaluated in displacement form F = I + (sum V (u_b-u_a) x gradW) B0,
 *     which is the time integral of the rate form of Sec. 3.1 under the
 *     kick-then-drift order used here;
 *   - 2D is plane strain: F embedded in 3x3 with F_zz = 1;
 *   - elastic configs use St Venant-Kirchhoff, S = lambda tr(E) I + 2 mu E,
 *     E = (F^T F - I)/2 (App. B.2 writes a garbled Almansi strain);
 *   - swelling: Cauchy pressure p = 3 K beta (c - c0) added as -p J F^-T
 *     (App. B.2's p = C (a - a0) with C = 3 K beta, a = c);
 *   - Alg. 1 stores C_p^-1 (called C_p there), initialised to I; Newton for
 *     the plastic multiplier starts at 0;
 *   - damping (Sec. 4.3): each neighbour pair gets backward-Euler updates of
 *     the pair ODE  m_a dv_a/dt = -B_ab (v_a - v_b),  B_ab = -2 eta V^2 W'/r,
 *     in a symmetric sweep (canonical colour order with dt/2, then the
 *     reverse order with dt/2); a constrained axis has 1/m = 0;
 *   - substep order: stress -> kick -> pairwise damping -> BC -> drift ->
 *     kinetic-energy reduction (symplectic Euler with damping split);
 *   - diffusion (Sec. 3.2 reduced to a scalar): one-pass pairwise Laplacian
 *     dc_i/dt = 2 D sum_j V (c_i - c_j) W'(r_ij)/r_ij in the reference
 *     configuration, Jacobi update;
 *   - time step Sec. 4.1 with |v|max, |dv/dt|max from the previous substep;
 *   - kinetic-energy stop (Sec. 4.2): tested once E_k has passed its peak
 *     after the slow step's load or diffusion event (Sec. 5.1, 5.3).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OB_OK 0
#define OB_ERR_ARG 1
#define OB_ERR_OOM 2
#define OB_ERR_SINGULAR 4
#define OB_ERR_NONFINITE 5
#define OB_ERR_UNSTABLE_DT 7
#define OB_ERR_STATE 8

#define OB_SVK 0
#define OB_J2 1

/* field ids (same meaning as the public API's field enum, defined here
 * independently) */
#define OB_F_U 0
#define OB_F_X 1
#define OB_F_V 2
#define OB_F_DEFGRAD 3
#define OB_F_PB 4
#define OB_F_C 5
#define OB_F_ALPHA 6
#define OB_F_CPINV 7
#define OB_F_ACC 8

typedef struct {
    double dt_slow;         /* diffusion step (0 = no diffusion this slow step) */
    double ramp_value;      /* load scale: u_presc = ramp * u_unit            */
    double dt_sub_override; /* > 0: fixed substep size                        */
    double ke_tol;          /* < 0 disables the kinetic-energy stop           */
    double ke_ref;
    int64_t max_substeps;
    int32_t ke_mode;        /* 0 total E_k, 1 E_k per unit volume             */
    int32_t check_every;    /* ignored by the oracle (checks every substep)   */
    int32_t force_dt;       /* accept an unstable dt_slow                     */
    int32_t reserved;
} ob_step_params;

typedef struct {
    int64_t substeps;
    int32_t converged;
    int32_t status;
    double ke_final;
    double max_v;
    double max_a;
    double dt_last;
    double end_force[3];
    double tip_deflection[3];
} ob_report;

typedef struct {
    int dim;
    int64_t n;
    double dx, h, V, cut2;
    /* anisotropic kernel (N4, the paper's thin-body kernel): spacing dxk per
     * axis, h = h_over_dx * min dxk, s_k = h / (h_over_dx dxk) <= 1; the kernel
     * is W(x) = detS W_iso(|s (.) x|) with W_iso of smoothing length h */
    int aniso;
    double dxk[3], sk[3], detS;
    int blk_shift;           /* smallest damping block width (2^blk_shift cells) */
    int ax_shift[3];         /* damping block width per axis: 2^ax_shift cells;  */
                             /* OB_WHOLE_AXIS = one block spans the whole axis   */
    int level_cap;           /* max pairs per sub-colour of a block (0 = none)   */
    double Xmin[3];
    double *X;               /* sorted order, n x 3 (z = 0 in 2D)          */
    int64_t *perm;           /* sorted position -> original index          */
    int64_t *rank;           /* original index -> sorted position          */
    int64_t *cell;           /* n x 3 cell coordinates                     */
    int64_t *off;            /* CSR offsets, n + 1                         */
    int32_t *nbr;            /* CSR indices, ascending                     */
    int64_t nnz;
    double *B0;              /* n x 9                                      */
    /* canonical damping order */
    int64_t npairs;
    int32_t *pa, *pb, *pcol, *psub;
    int64_t *pkey;
    /* material */
    int model;
    double rho0, E, nu, K, mu, lambda, s0, sinf, delta, Hlin, eta;
    int has_diff;
    double D, beta, c0;
    int diff_mode;           /* 0: one-pass pairwise Laplacian, 1: two-stage flux */
    /* state, sorted order */
    double *u, *v, *acc, *PB, *cpinv, *alpha, *c, *u_unit, *cheld_val;
    unsigned char *fix, *fgrp, *tgrp, *cheld;
    double last_amax;
} ob_body;

/* ------------------------------------------------------------------ */
/* Kernel (Sec. 3.1): Wendland C2, q = r/h, support q < 2.             */
/*   W(q)  = a_d (1 - q/2)^4 (1 + 2q)                                  */
/*   W'(r) = -5 a_d q (1 - q/2)^3 / h                                  */
/*   a_2 = 7/(4 pi h^2), a_3 = 21/(16 pi h^3)                          */
/* ------------------------------------------------------------------ */
static double kernel_alpha(int dim, double h) {
    if (dim == 2) return 7.0 / (4.0 * M_PI * h * h);
    return 21.0 / (16.0 * M_PI * h * h * h);
}

double ob_kernel_w(int dim, double h, double r) {
    double q = r / h;
    if (q >= 2.0) return 0.0;
    double t = 1.0 - 0.5 * q;
    return kernel_alpha(dim, h) * t * t * t * t * (1.0 + 2.0 * q);
}

double ob_kernel_dwdr(int dim, double h, double r) {
    double q = r / h;
    if (q >= 2.0) return 0.0;
    double t = 1.0 - 0.5 * q;
    return -5.0 * kernel_alpha(dim, h) * q * t * t * t / h;
}

/* gradient with respect to X_a of W(|X_a - X_b|) (Sec. 3.1, kernel gradient) */
static void grad_w(const ob_body *b, int64_t a, int64_t j, double g[3]) {
    double d[3], r2 = 0.0;
    if (b->aniso) {
        /* grad of detS W_iso(|s (.) d|): detS W_iso'(r~) s_k^2 d_k / r~ */
        for (int k = 0; k < 3; k++) {
            d[k] = b->X[3 * a + k] - b->X[3 * j + k];
            double e = d[k] * b->sk[k];
            r2 += e * e;
        }
        double r = sqrt(r2);
        double dw = ob_kernel_dwdr(b->dim, b->h, r);
        for (int k = 0; k < 3; k++) g[k] = b->detS * (dw / r) * b->sk[k] * b->sk[k] * d[k];
        return;
    }
    for (int k = 0; k < 3; k++) {
        d[k] = b->X[3 * a + k] - b->X[3 * j + k];
        r2 += d[k] * d[k];
    }
    double r = sqrt(r2);
    double dw = ob_kernel_dwdr(b->dim, b->h, r);
    for (int k = 0; k < 3; k++) g[k] = dw * d[k] / r;
}

/* ------------------------------------------------------------------ */
/* small 3x3 helpers (row-major)                                        */
/* ------------------------------------------------------------------ */
static void m3_mul(const double A[9], const double B[9], double C[9]) {
    double T[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += A[3 * i + k] * B[3 * k + j];
            T[3 * i + j] = s;
        }
    memcpy(C, T, sizeof(T));
}
static void m3_transpose(const double A[9], double B[9]) {
    double T[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) T[3 * i + j] = A[3 * j + i];
    memcpy(B, T, sizeof(T));
}
static double m3_det(const double A[9]) {
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}
static double m3_inv(const double A[9], double B[9]) {
    double det = m3_det(A);
    double T[9];
    T[0] = (A[4] * A[8] - A[5] * A[7]) / det;
    T[1] = (A[2] * A[7] - A[1] * A[8]) / det;
    T[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    T[3] = (A[5] * A[6] - A[3] * A[8]) / det;
    T[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    T[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    T[6] = (A[3] * A[7] - A[4] * A[6]) / det;
    T[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    T[8] = (A[0] * A[4] - A[1] * A[3]) / det;
    memcpy(B, T, sizeof(T));
    return det;
}
static double m3_trace(const double A[9]) { return A[0] + A[4] + A[8]; }

/* symmetric 6-vector (xx, yy, zz, xy, yz, xz) <-> 3x3 */
static void sym_to_m3(const double s[6], double A[9]) {
    A[0] = s[0]; A[4] = s[1]; A[8] = s[2];
    A[1] = A[3] = s[3];
    A[5] = A[7] = s[4];
    A[2] = A[6] = s[5];
}
static void m3_to_sym(const double A[9], double s[6]) {
    s[0] = A[0]; s[1] = A[4]; s[2] = A[8];
    s[3] = 0.5 * (A[1] + A[3]);
    s[4] = 0.5 * (A[5] + A[7]);
    s[5] = 0.5 * (A[2] + A[6]);
}

/* ------------------------------------------------------------------ */
/* Morton order (setup): cell = floor((X - Xmin)/dx) per axis, key =   */
/* bit interleave with the x bit lowest, ties by original index.       */
/* ------------------------------------------------------------------ */
static uint64_t morton_key(int dim, const int64_t c[3]) {
    uint64_t key = 0;
    int bits = dim == 2 ? 32 : 21;
    for (int bit = 0; bit < bits; bit++)
        for (int k = 0; k < dim; k++)
            key |= (uint64_t)((c[k] >> bit) & 1) << (bit * dim + k);
    return key;
}

typedef struct { uint64_t key; int64_t orig; } key_idx;
static int cmp_key_idx(const void *pa, const void *pb) {
    const key_idx *a = pa, *b = pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->orig < b->orig ? -1 : (a->orig > b->orig);
}

/* ------------------------------------------------------------------ */
/* Neighbour lists: all j != i with |X_i - X_j|^2 < (2h)^2, ascending.  */
/* The neighbourhood is fixed in the reference configuration (Sec.     */
/* 3.1, total Lagrangian formulation).                                  */
/* ------------------------------------------------------------------ */
static int is_neighbour(const ob_body *b, int64_t i, int64_t j) {
    /* |s (.) (X_i - X_j)|^2 < (2h)^2: the kernel's support (an ellipsoid for
     * an anisotropic kernel, s = 1 otherwise) */
    double r2 = 0.0;
    for (int k = 0; k < 3; k++) {
        double d = (b->X[3 * i + k] - b->X[3 * j + k]) * b->sk[k];
        r2 += d * d;
    }
    return r2 < b->cut2;
}

static int build_neighbours_brute(ob_body *b) {
    int64_t n = b->n;
    b->off = calloc((size_t)n + 1, sizeof(int64_t));
    if (!b->off) return OB_ERR_OOM;
    for (int64_t i = 0; i < n; i++) {
        int64_t cnt = 0;
        for (int64_t j = 0; j < n; j++)
            if (j != i && is_neighbour(b, i, j)) cnt++;
        b->off[i + 1] = b->off[i] + cnt;
    }
    b->nnz = b->off[n];
    b->nbr = malloc((size_t)(b->nnz > 0 ? b->nnz : 1) * sizeof(int32_t));
    if (!b->nbr) return OB_ERR_OOM;
    for (int64_t i = 0; i < n; i++) {
        int64_t p = b->off[i];
        for (int64_t j = 0; j < n; j++)
            if (j != i && is_neighbour(b, i, j)) b->nbr[p++] = (int32_t)j;
    }
    return OB_OK;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* cell-list variant: bins of width 2h, a 3^d stencil, then the exact test */
static int build_neighbours_cells(ob_body *b) {
    int64_t n = b->n;
    double w = 2.0 * b->h;
    int64_t nb[3] = {1, 1, 1};
    double ext[3] = {0, 0, 0};
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < b->dim; k++) {
            double e = b->X[3 * i + k] - b->Xmin[k];
            if (e > ext[k]) ext[k] = e;
        }
    double wk[3];
    for (int k = 0; k < 3; k++) wk[k] = w / b->sk[k];   /* support extent per axis */
    for (int k = 0; k < b->dim; k++) nb[k] = (int64_t)floor(ext[k] / wk[k]) + 1;
    int64_t nbins = nb[0] * nb[1] * nb[2];
    int64_t *bin_of = malloc((size_t)n * sizeof(int64_t));
    int64_t *head = calloc((size_t)nbins + 1, sizeof(int64_t));
    int64_t *items = malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t *fill = calloc((size_t)nbins, sizeof(int64_t));
    b->off = calloc((size_t)n + 1, sizeof(int64_t));
    if (!bin_of || !head || !items || !fill || !b->off) return OB_ERR_OOM;
    for (int64_t i = 0; i < n; i++) {
        int64_t c[3] = {0, 0, 0};
        for (int k = 0; k < b->dim; k++) c[k] = (int64_t)floor((b->X[3 * i + k] - b->Xmin[k]) / wk[k]);
        bin_of[i] = (c[2] * nb[1] + c[1]) * nb[0] + c[0];
        head[bin_of[i] + 1]++;
    }
    for (int64_t q = 0; q < nbins; q++) head[q + 1] += head[q];
    for (int64_t i = 0; i < n; i++) items[head[bin_of[i]] + fill[bin_of[i]]++] = i;

    int32_t *tmp = malloc(4096 * sizeof(int32_t));
    int64_t cap = 1 << 20;
    int32_t *out = malloc((size_t)cap * sizeof(int32_t));
    if (!tmp || !out) return OB_ERR_OOM;
    int64_t nnz = 0;
    int zr = b->dim == 3 ? 1 : 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t bi = bin_of[i];
        int64_t c0 = bi % nb[0], c1 = (bi / nb[0]) % nb[1], c2 = bi / (nb[0] * nb[1]);
        int cnt = 0;
        for (int64_t z = c2 - zr; z <= c2 + zr; z++)
            for (int64_t y = c1 - 1; y <= c1 + 1; y++)
                for (int64_t x = c0 - 1; x <= c0 + 1; x++) {
                    if (x < 0 || y < 0 || z < 0 || x >= nb[0] || y >= nb[1] || z >= nb[2]) continue;
                    int64_t q = (z * nb[1] + y) * nb[0] + x;
                    for (int64_t t = head[q]; t < head[q + 1]; t++) {
                        int64_t j = items[t];
                        if (j != i && is_neighbour(b, i, j)) {
                            if (cnt >= 4096) return OB_ERR_ARG;
                            tmp[cnt++] = (int32_t)j;
                        }
                    }
                }
        qsort(tmp, (size_t)cnt, sizeof(int32_t), cmp_i32);
        if (nnz + cnt > cap) {
            while (nnz + cnt > cap) cap *= 2;
            out = realloc(out, (size_t)cap * sizeof(int32_t));
            if (!out) return OB_ERR_OOM;
        }
        memcpy(out + nnz, tmp, (size_t)cnt * sizeof(int32_t));
        nnz += cnt;
        b->off[i + 1] = nnz;
    }
    b->nnz = nnz;
    b->nbr = out;
    free(tmp); free(bin_of); free(head); free(items); free(fill);
    return OB_OK;
}

/* ------------------------------------------------------------------ */
/* Correction matrix (Sec. 3.1):                                        */
/*   B0_a = ( sum_b V_b (X_b - X_a) (x) grad_a W_ab )^-1, computed once */
/* ------------------------------------------------------------------ */
static int build_b0(ob_body *b) {
    int d = b->dim;
    b->B0 = calloc((size_t)b->n * 9, sizeof(double));
    if (!b->B0) return OB_ERR_OOM;
    for (int64_t a = 0; a < b->n; a++) {
        double S[9] = {0};
        for (int64_t p = b->off[a]; p < b->off[a + 1]; p++) {
            int64_t j = b->nbr[p];
            double g[3];
            grad_w(b, a, j, g);
            for (int r = 0; r < d; r++)
                for (int s = 0; s < d; s++)
                    S[3 * r + s] += b->V * (b->X[3 * j + r] - b->X[3 * a + r]) * g[s];
        }
        double norm = 0.0;
        for (int k = 0; k < 9; k++) norm += S[k] * S[k];
        norm = sqrt(norm);
        double *B = b->B0 + 9 * a;
        if (d == 2) {
            double det = S[0] * S[4] - S[1] * S[3];
            if (!(fabs(det) >= 1e-12 * norm * norm) || norm == 0.0) return OB_ERR_SINGULAR;
            B[0] = S[4] / det; B[1] = -S[1] / det;
            B[3] = -S[3] / det; B[4] = S[0] / det;
            B[8] = 1.0;
        } else {
            double det = m3_det(S);
            if (!(fabs(det) >= 1e-12 * norm * norm * norm) || norm == 0.0) return OB_ERR_SINGULAR;
            m3_inv(S, B);
        }
    }
    return OB_OK;
}

/* ------------------------------------------------------------------ */
/* Canonical order of the pairwise damping sweep (Sec. 4.3 leaves the   */
/* order to the cited splitting scheme; this is the order chosen):      */
/*   block = cell >> ax_shift[k] on axis k (2^shift cells, 2^shift * dx */
/*   > 2h; OB_WHOLE_AXIS = the axis is not blocked); pair (a<b) is owned */
/*   by the componentwise-min block of its two particles; block colour  */
/*   = parity bits of the owner block; inside an owner block its pairs, */
/*   visited by descending offset class (the sign-folded cell offset),  */
/*   then ascending (a,b), take the smallest sub-colour unused at a and */
/*   at b that holds fewer than level_cap pairs so far (greedy;         */
/*   level_cap 0 = no cap).  Sequential order: colour, owner block      */
/*   Morton key, sub-colour, a, b.  Pairs of one (colour, sub-colour)   */
/*   touch disjoint particles.  (Descending classes visit the longest   */
/*   offsets first, which keeps the largest groups near the degree      */
/*   bound on levels.)                                                  */
/* ------------------------------------------------------------------ */
typedef struct { int32_t col; int32_t sub; uint64_t key; int32_t cls; int32_t a, b; } pair_rec;

/* owner block, then offset class (descending), then (a, b): the order the
 * greedy visits */
static int cmp_pair_owner(const void *x, const void *y) {
    const pair_rec *p = x, *q = y;
    if (p->col != q->col) return p->col < q->col ? -1 : 1;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    if (p->cls != q->cls) return p->cls > q->cls ? -1 : 1;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    return (p->b > q->b) - (p->b < q->b);
}

/* offset class of a pair: the cell offset o = cell(b) - cell(a), sign-folded so
 * that o and -o fall in one class (first nonzero component positive), encoded
 * as a base-(2R+1) number with R = floor(2h/dx) + 1 */
static int32_t offset_class(const ob_body *b, int64_t a, int64_t j) {
    int64_t o[3] = {0, 0, 0};
    for (int k = 0; k < b->dim; k++) o[k] = b->cell[3 * j + k] - b->cell[3 * a + k];
    int sgn = 0;
    for (int k = b->dim - 1; k >= 0 && sgn == 0; k--)
        if (o[k] != 0) sgn = o[k] > 0 ? 1 : -1;
    int64_t R = (int64_t)floor(2.0 * b->h / b->dx) + 1, base = 2 * R + 1;
    int64_t c = 0;
    for (int k = b->dim - 1; k >= 0; k--) c = c * base + (sgn * o[k] + R);
    return (int32_t)c;
}
static int cmp_pair_final(const void *x, const void *y) {
    const pair_rec *p = x, *q = y;
    if (p->col != q->col) return p->col < q->col ? -1 : 1;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    if (p->sub != q->sub) return p->sub < q->sub ? -1 : 1;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    return (p->b > q->b) - (p->b < q->b);
}

#define OB_MAXSUB 256
#define OB_WHOLE_AXIS 62
static int build_colouring(ob_body *b) {
    int d = b->dim;
    int64_t np = b->nnz / 2;
    pair_rec *pr = malloc((size_t)(np > 0 ? np : 1) * sizeof(pair_rec));
    if (!pr) return OB_ERR_OOM;
    int64_t m = 0;
    for (int64_t a = 0; a < b->n; a++)
        for (int64_t p = b->off[a]; p < b->off[a + 1]; p++) {
            int64_t j = b->nbr[p];
            if (j <= a) continue;
            int64_t ob[3] = {0, 0, 0};
            int col = 0;
            for (int k = 0; k < d; k++) {
                int64_t ba = b->cell[3 * a + k] >> b->ax_shift[k];
                int64_t bb = b->cell[3 * j + k] >> b->ax_shift[k];
                ob[k] = ba < bb ? ba : bb;
                col |= (int)(ob[k] & 1) << k;
            }
            pr[m].col = col;
            pr[m].key = morton_key(d, ob);
            pr[m].cls = offset_class(b, a, j);
            pr[m].a = (int32_t)a;
            pr[m].b = (int32_t)j;
            pr[m].sub = 0;
            m++;
        }
    if (m != np) { free(pr); return OB_ERR_STATE; }
    qsort(pr, (size_t)m, sizeof(pair_rec), cmp_pair_owner);
    /* greedy sub-colouring per owner block */
    uint64_t *used = calloc((size_t)b->n * (OB_MAXSUB / 64), sizeof(uint64_t));
    if (!used) { free(pr); return OB_ERR_OOM; }
    int64_t s = 0;
    while (s < m) {
        int64_t e = s;
        while (e < m && pr[e].col == pr[s].col && pr[e].key == pr[s].key) e++;
        int count[OB_MAXSUB];
        memset(count, 0, sizeof(count));
        for (int64_t t = s; t < e; t++) {
            uint64_t *ua = used + (size_t)pr[t].a * (OB_MAXSUB / 64);
            uint64_t *ub = used + (size_t)pr[t].b * (OB_MAXSUB / 64);
            int c = 0;
            while (c < OB_MAXSUB &&
                   ((((ua[c >> 6] | ub[c >> 6]) >> (c & 63)) & 1) ||
                    (b->level_cap > 0 && count[c] >= b->level_cap)))
                c++;
            if (c >= OB_MAXSUB) { free(used); free(pr); return OB_ERR_STATE; }
            count[c]++;
            pr[t].sub = c;
            ua[c >> 6] |= 1ull << (c & 63);
            ub[c >> 6] |= 1ull << (c & 63);
        }
        for (int64_t t = s; t < e; t++) {
            memset(used + (size_t)pr[t].a * (OB_MAXSUB / 64), 0, OB_MAXSUB / 8);
            memset(used + (size_t)pr[t].b * (OB_MAXSUB / 64), 0, OB_MAXSUB / 8);
        }
        s = e;
    }
    free(used);
    qsort(pr, (size_t)m, sizeof(pair_rec), cmp_pair_final);
    b->npairs = m;
    b->pa = malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    b->pb = malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    b->pcol = malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    b->psub = malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    b->pkey = malloc((size_t)(m > 0 ? m : 1) * sizeof(int64_t));
    if (!b->pa || !b->pb || !b->pcol || !b->psub || !b->pkey) { free(pr); return OB_ERR_OOM; }
    for (int64_t t = 0; t < m; t++) {
        b->pa[t] = pr[t].a; b->pb[t] = pr[t].b;
        b->pcol[t] = pr[t].col; b->psub[t] = pr[t].sub;
        b->pkey[t] = (int64_t)pr[t].key;
    }
    free(pr);
    return OB_OK;
}

/* ------------------------------------------------------------------ */
/* body lifetime                                                        */
/* ------------------------------------------------------------------ */
void ob_destroy(ob_body *b) {
    if (!b) return;
    void *ptrs[] = {b->X, b->perm, b->rank, b->cell, b->off, b->nbr, b->B0, b->pa, b->pb,
                    b->pcol, b->psub, b->pkey, b->u, b->v, b->acc, b->PB, b->cpinv,
                    b->alpha, b->c, b->u_unit, b->cheld_val, b->fix, b->fgrp, b->tgrp,
                    b->cheld};
    for (size_t i = 0; i < sizeof(ptrs) / sizeof(ptrs[0]); i++) free(ptrs[i]);
    free(b);
}

/* layout of the damping order: block width per axis as a shift (cells =
 * 2^shift; OB_WHOLE_AXIS for an unblocked axis; negative = the smallest
 * power of two >= floor(2h/dx) + 1) and the cap on pairs per sub-colour */
int ob_create_layout(int dim, int64_t n, const double *Xorig, double dx, double h_over_dx,
                     int brute, const int32_t ax_shift[3], int32_t level_cap, ob_body **out);

int ob_create(int dim, int64_t n, const double *Xorig, double dx, double h_over_dx,
              int brute, ob_body **out) {
    const int32_t def[3] = {-1, -1, -1};
    return ob_create_layout(dim, n, Xorig, dx, h_over_dx, brute, def, 32, out);
}

int ob_create_aniso(int dim, int64_t n, const double *Xorig, const double dxk[3],
                    double h_over_dx, int brute, const int32_t ax_shift[3], int32_t level_cap,
                    ob_body **out);

int ob_create_layout(int dim, int64_t n, const double *Xorig, double dx, double h_over_dx,
                     int brute, const int32_t ax_shift[3], int32_t level_cap, ob_body **out) {
    const double dxk[3] = {dx, dx, dx};
    return ob_create_aniso(dim, n, Xorig, dxk, h_over_dx, brute, ax_shift, level_cap, out);
}

/* spacing dxk per axis; equal spacings give the isotropic kernel exactly */
int ob_create_aniso(int dim, int64_t n, const double *Xorig, const double dxk[3],
                    double h_over_dx, int brute, const int32_t ax_shift[3], int32_t level_cap,
                    ob_body **out) {
    *out = NULL;
    if (level_cap < 0) return OB_ERR_ARG;
    if ((dim != 2 && dim != 3) || n < 2 || !(h_over_dx > 0.0) || n > 2000000000LL)
        return OB_ERR_ARG;
    double dx = dxk[0];
    for (int k = 0; k < dim; k++) {
        if (!(dxk[k] > 0.0)) return OB_ERR_ARG;
        if (dxk[k] < dx) dx = dxk[k];
    }
    ob_body *b = calloc(1, sizeof(ob_body));
    if (!b) return OB_ERR_OOM;
    b->dim = dim; b->n = n; b->dx = dx;
    b->h = h_over_dx * dx;
    double w = 2.0 * b->h;
    b->cut2 = w * w;
    b->detS = 1.0;
    b->V = 1.0;
    for (int k = 0; k < 3; k++) {
        b->dxk[k] = k < dim ? dxk[k] : dx;
        b->sk[k] = dx / b->dxk[k];
        if (k < dim) {
            b->V *= b->dxk[k];
            b->detS *= b->sk[k];
            if (b->dxk[k] != dx) b->aniso = 1;
        }
    }
    /* block width: smallest power of two >= floor(2h/dx) + 1 cells */
    int64_t need = (int64_t)floor(w / dx) + 1;
    b->blk_shift = 0;
    while ((1LL << b->blk_shift) < need) b->blk_shift++;
    for (int k = 0; k < 3; k++) {
        int sh = ax_shift[k] < 0 ? b->blk_shift : ax_shift[k];
        if (sh < b->blk_shift || sh > OB_WHOLE_AXIS) { free(b); return OB_ERR_ARG; }
        b->ax_shift[k] = sh;
    }
    b->level_cap = level_cap;
    for (int k = 0; k < 3; k++) b->Xmin[k] = 0.0;
    for (int k = 0; k < dim; k++) {
        double mn = Xorig[k];
        for (int64_t i = 1; i < n; i++)
            if (Xorig[(size_t)i * dim + k] < mn) mn = Xorig[(size_t)i * dim + k];
        b->Xmin[k] = mn;
    }
    for (int64_t i = 0; i < n * dim; i++)
        if (!isfinite(Xorig[i])) { ob_destroy(b); return OB_ERR_ARG; }
    key_idx *ki = malloc((size_t)n * sizeof(key_idx));
    b->perm = malloc((size_t)n * sizeof(int64_t));
    b->rank = malloc((size_t)n * sizeof(int64_t));
    b->cell = calloc((size_t)n * 3, sizeof(int64_t));
    b->X = calloc((size_t)n * 3, sizeof(double));
    if (!ki || !b->perm || !b->rank || !b->cell || !b->X) { free(ki); ob_destroy(b); return OB_ERR_OOM; }
    for (int64_t i = 0; i < n; i++) {
        int64_t c[3] = {0, 0, 0};
        for (int k = 0; k < dim; k++) c[k] = (int64_t)floor((Xorig[(size_t)i * dim + k] - b->Xmin[k]) / b->dxk[k]);
        ki[i].key = morton_key(dim, c);
        ki[i].orig = i;
    }
    qsort(ki, (size_t)n, sizeof(key_idx), cmp_key_idx);
    for (int64_t s = 0; s < n; s++) {
        int64_t i = ki[s].orig;
        b->perm[s] = i;
        b->rank[i] = s;
        for (int k = 0; k < dim; k++) {
            b->X[3 * s + k] = Xorig[(size_t)i * dim + k];
            b->cell[3 * s + k] = (int64_t)floor((b->X[3 * s + k] - b->Xmin[k]) / b->dxk[k]);
        }
    }
    free(ki);
    int st = brute ? build_neighbours_brute(b) : build_neighbours_cells(b);
    if (st == OB_OK) st = build_b0(b);
    if (st == OB_OK) st = build_colouring(b);
    if (st != OB_OK) { ob_destroy(b); return st; }
    b->u = calloc((size_t)n * 3, sizeof(double));
    b->v = calloc((size_t)n * 3, sizeof(double));
    b->acc = calloc((size_t)n * 3, sizeof(double));
    b->PB = calloc((size_t)n * 9, sizeof(double));
    b->cpinv = calloc((size_t)n * 6, sizeof(double));
    b->alpha = calloc((size_t)n, sizeof(double));
    b->c = calloc((size_t)n, sizeof(double));
    b->u_unit = calloc((size_t)n * 3, sizeof(double));
    b->cheld_val = calloc((size_t)n, sizeof(double));
    b->fix = calloc((size_t)n, 1);
    b->fgrp = calloc((size_t)n, 1);
    b->tgrp = calloc((size_t)n, 1);
    b->cheld = calloc((size_t)n, 1);
    if (!b->u || !b->v || !b->acc || !b->PB || !b->cpinv || !b->alpha || !b->c || !b->u_unit ||
        !b->cheld_val || !b->fix || !b->fgrp || !b->tgrp || !b->cheld) {
        ob_destroy(b);
        return OB_ERR_OOM;
    }
    for (int64_t i = 0; i < n; i++) {
        b->cpinv[6 * i + 0] = b->cpinv[6 * i + 1] = b->cpinv[6 * i + 2] = 1.0;
    }
    b->model = OB_SVK;
    b->rho0 = 1.0;
    *out = b;
    return OB_OK;
}

int64_t ob_nnz(const ob_body *b) { return b->nnz; }
int64_t ob_npairs(const ob_body *b) { return b->npairs; }
int ob_blk_shift(const ob_body *b) { return b->blk_shift; }

int ob_neighbors(const ob_body *b, int64_t *off, int32_t *idx) {
    if (off) memcpy(off, b->off, (size_t)(b->n + 1) * sizeof(int64_t));
    if (idx) memcpy(idx, b->nbr, (size_t)b->nnz * sizeof(int32_t));
    return OB_OK;
}

int ob_perm(const ob_body *b, int64_t *perm) {
    memcpy(perm, b->perm, (size_t)b->n * sizeof(int64_t));
    return OB_OK;
}

int ob_colouring(const ob_body *b, int32_t *pa, int32_t *pb, int32_t *col, int64_t *key,
                 int32_t *sub) {
    size_t m = (size_t)b->npairs;
    if (pa) memcpy(pa, b->pa, m * sizeof(int32_t));
    if (pb) memcpy(pb, b->pb, m * sizeof(int32_t));
    if (col) memcpy(col, b->pcol, m * sizeof(int32_t));
    if (key) memcpy(key, b->pkey, m * sizeof(int64_t));
    if (sub) memcpy(sub, b->psub, m * sizeof(int32_t));
    return OB_OK;
}

/* ------------------------------------------------------------------ */
/* material and boundary conditions                                     */
/* ------------------------------------------------------------------ */
int ob_set_material(ob_body *b, int model, double rho0, double E, double nu, double s0,
                    double sinf, double delta, double H) {
    if ((model != OB_SVK && model != OB_J2) || !(rho0 > 0) || !(E > 0) || !(nu > -1.0) ||
        !(nu < 0.5))
        return OB_ERR_ARG;
    b->model = model;
    b->rho0 = rho0; b->E = E; b->nu = nu;
    /* App. A.2: E = 2 mu (1 + nu) = 3 K (1 - 2 nu); App. B.2: lambda = K - 2 mu / 3 */
    b->mu = E / (2.0 * (1.0 + nu));
    b->K = E / (3.0 * (1.0 - 2.0 * nu));
    b->lambda = b->K - 2.0 * b->mu / 3.0;
    b->s0 = s0; b->sinf = sinf; b->delta = delta; b->Hlin = H;
    return OB_OK;
}

int ob_set_damping(ob_body *b, double eta) {
    if (!(eta >= 0.0)) return OB_ERR_ARG;
    b->eta = eta;
    return OB_OK;
}

int ob_set_diffusion(ob_body *b, double D, double beta, double c0) {
    if (!(D >= 0.0) || !isfinite(beta) || !isfinite(c0)) return OB_ERR_ARG;
    b->has_diff = 1;
    b->D = D; b->beta = beta; b->c0 = c0;
    for (int64_t i = 0; i < b->n; i++)
        if (!b->cheld[i]) b->c[i] = c0;
    return OB_OK;
}

int ob_set_bc_displacement(ob_body *b, int64_t count, const int64_t *ids, unsigned mask,
                           const double *u_unit, int report_force) {
    for (int64_t t = 0; t < count; t++) {
        if (ids[t] < 0 || ids[t] >= b->n) return OB_ERR_ARG;
        int64_t s = b->rank[ids[t]];
        b->fix[s] |= (unsigned char)(mask & ((1u << b->dim) - 1));
        for (int k = 0; k < b->dim; k++)
            if (mask & (1u << k)) b->u_unit[3 * s + k] = u_unit ? u_unit[t * b->dim + k] : 0.0;
        if (report_force) b->fgrp[s] = 1;
    }
    return OB_OK;
}

int ob_set_bc_concentration(ob_body *b, int64_t count, const int64_t *ids, double value) {
    for (int64_t t = 0; t < count; t++) {
        if (ids[t] < 0 || ids[t] >= b->n) return OB_ERR_ARG;
        int64_t s = b->rank[ids[t]];
        b->cheld[s] = 1;
        b->cheld_val[s] = value;
        b->c[s] = value;
    }
    return OB_OK;
}

/* end of a time-limited contact (Sec. 5.3-5.4): the particles keep their c
 * and take part in the diffusion step again */
int ob_release_bc_concentration(ob_body *b, int64_t count, const int64_t *ids) {
    for (int64_t t = 0; t < count; t++) {
        if (ids[t] < 0 || ids[t] >= b->n) return OB_ERR_ARG;
        b->cheld[b->rank[ids[t]]] = 0;
    }
    return OB_OK;
}

int ob_set_tip(ob_body *b, int64_t count, const int64_t *ids) {
    memset(b->tgrp, 0, (size_t)b->n);
    for (int64_t t = 0; t < count; t++) {
        if (ids[t] < 0 || ids[t] >= b->n) return OB_ERR_ARG;
        b->tgrp[b->rank[ids[t]]] = 1;
    }
    return OB_OK;
}

/* ------------------------------------------------------------------ */
/* Stress at one particle (App. A, App. B.2).  F, P row-major 3x3.      */
/* ------------------------------------------------------------------ */
static double hardening_k(const ob_body *b, double al) {
    /* App. A.3: k = s0 + (sinf - s0)(1 - exp(-delta al)) + H al */
    return b->s0 + (b->sinf - b->s0) * (1.0 - exp(-b->delta * al)) + b->Hlin * al;
}
static double hardening_dk(const ob_body *b, double al) {
    return (b->sinf - b->s0) * b->delta * exp(-b->delta * al) + b->Hlin;
}

/* returns 1 if a plastic return was taken */
static int stress_point(const ob_body *b, const double F[9], double cpinv[6], double *alpha,
                        double c, double P[9], double *newton_res) {
    int plastic = 0;
    if (newton_res) *newton_res = 0.0;
    if (b->model == OB_SVK) {
        /* St Venant-Kirchhoff: E = (F^T F - I)/2, S = lambda tr(E) I + 2 mu E, P = F S */
        double Ft[9], C[9], Eg[9], S[9];
        m3_transpose(F, Ft);
        m3_mul(Ft, F, C);
        for (int k = 0; k < 9; k++) Eg[k] = 0.5 * C[k];
        Eg[0] -= 0.5; Eg[4] -= 0.5; Eg[8] -= 0.5;
        double tr = m3_trace(Eg);
        for (int k = 0; k < 9; k++) S[k] = 2.0 * b->mu * Eg[k];
        S[0] += b->lambda * tr; S[4] += b->lambda * tr; S[8] += b->lambda * tr;
        m3_mul(F, S, P);
    } else {
        /* Algorithm 1 (App. A.4): J2 return mapping, nonlinear hardening */
        double J = m3_det(F);
        double Fb[9], Fbt[9], Cp[9], tmp[9], bpre[9];
        double sc = 1.0 / cbrt(J);
        for (int k = 0; k < 9; k++) Fb[k] = sc * F[k];
        sym_to_m3(cpinv, Cp);
        m3_transpose(Fb, Fbt);
        m3_mul(Fb, Cp, tmp);
        m3_mul(tmp, Fbt, bpre);
        double trb = m3_trace(bpre);
        double spre[9];
        for (int k = 0; k < 9; k++) spre[k] = b->mu * bpre[k];
        spre[0] -= b->mu * trb / 3.0; spre[4] -= b->mu * trb / 3.0; spre[8] -= b->mu * trb / 3.0;
        double s = 0.0;
        for (int k = 0; k < 9; k++) s += spre[k] * spre[k];
        s = sqrt(s);
        const double r23 = sqrt(2.0 / 3.0);
        double kal = hardening_k(b, *alpha);
        double f = s - r23 * kal;
        double snew[9];
        memcpy(snew, spre, sizeof(snew));
        if (f > 0.0) {
            plastic = 1;
            double mubar = b->mu * trb / 3.0;
            double dg = 0.0, g = f;
            for (int it = 0; it < 30; it++) {
                g = s - r23 * hardening_k(b, *alpha + r23 * dg) - 2.0 * mubar * dg;
                if (fabs(g) <= 1e-13 * r23 * kal) break;
                double dgd = -(2.0 / 3.0) * hardening_dk(b, *alpha + r23 * dg) - 2.0 * mubar;
                dg -= g / dgd;
            }
            if (newton_res) *newton_res = g;
            for (int k = 0; k < 9; k++) snew[k] = spre[k] - 2.0 * mubar * dg * spre[k] / s;
            *alpha += r23 * dg;
            /* b_e = s/mu + tr(b_pre)/3 I;  C_p^-1 = Fb^-1 b_e Fb^-T */
            double be[9], Fbi[9], Fbit[9];
            for (int k = 0; k < 9; k++) be[k] = snew[k] / b->mu;
            be[0] += trb / 3.0; be[4] += trb / 3.0; be[8] += trb / 3.0;
            m3_inv(Fb, Fbi);
            m3_transpose(Fbi, Fbit);
            m3_mul(Fbi, be, tmp);
            m3_mul(tmp, Fbit, Cp);
            m3_to_sym(Cp, cpinv);
        }
        /* tau = K/2 (J^2 - 1) I + s;  P = tau F^-T */
        double tau[9], Fi[9], Fit[9];
        memcpy(tau, snew, sizeof(tau));
        double pv = 0.5 * b->K * (J * J - 1.0);
        tau[0] += pv; tau[4] += pv; tau[8] += pv;
        m3_inv(F, Fi);
        m3_transpose(Fi, Fit);
        m3_mul(tau, Fit, P);
    }
    if (b->has_diff && b->beta != 0.0) {
        /* App. B.2: sigma = sigma_s - p I with p = 3 K beta (c - c0):  P -= p J F^-T */
        double Fi[9], Fit[9];
        double J = m3_inv(F, Fi);
        m3_transpose(Fi, Fit);
        double p = 3.0 * b->K * b->beta * (c - b->c0);
        for (int k = 0; k < 9; k++) P[k] -= p * J * Fit[k];
    }
    return plastic;
}

/* public material-point driver (used by the return-mapping pins) */
int ob_stress_point(int model, double rho0, double E, double nu, double s0, double sinf,
                    double delta, double H, const double F[9], double cpinv[6], double *alpha,
                    double P[9], double *newton_res) {
    ob_body tmp;
    memset(&tmp, 0, sizeof(tmp));
    int st = ob_set_material(&tmp, model, rho0, E, nu, s0, sinf, delta, H);
    if (st != OB_OK) return -1;
    return stress_point(&tmp, F, cpinv, alpha, 0.0, P, newton_res);
}

/* ------------------------------------------------------------------ */
/* Substep pieces                                                       */
/* ------------------------------------------------------------------ */
/* F_a = I + (sum_b V (u_b - u_a) (x) grad_a W_ab) B0_a  (Sec. 2.1, Sec. 3.1) */
static void defgrad(const ob_body *b, int64_t a, double F[9]) {
    int d = b->dim;
    double G[9] = {0};
    for (int64_t p = b->off[a]; p < b->off[a + 1]; p++) {
        int64_t j = b->nbr[p];
        double g[3];
        grad_w(b, a, j, g);
        for (int r = 0; r < d; r++)
            for (int s = 0; s < d; s++)
                G[3 * r + s] += b->V * (b->u[3 * j + r] - b->u[3 * a + r]) * g[s];
    }
    m3_mul(G, b->B0 + 9 * a, F);
    F[0] += 1.0; F[4] += 1.0; F[8] += 1.0;
    if (d == 2) { F[2] = F[5] = F[6] = F[7] = 0.0; F[8] = 1.0; }
}

static int stage_stress(ob_body *b) {
    int d = b->dim;
    for (int64_t a = 0; a < b->n; a++) {
        double F[9], P[9];
        defgrad(b, a, F);
        stress_point(b, F, b->cpinv + 6 * a, b->alpha + a, b->c[a], P, NULL);
        /* store PB_a = P_a B0_a^T (d x d block): the force that is the
         * variation of sum V psi(F) for F = I + sum_b (u_b - u_a) (x) B0_a^T V grad W
         * (B0 is symmetric for an isotropic kernel) */
        double PBf[9], B0t[9];
        m3_transpose(b->B0 + 9 * a, B0t);
        m3_mul(P, B0t, PBf);
        for (int r = 0; r < d; r++)
            for (int s = 0; s < d; s++) b->PB[9 * a + 3 * r + s] = PBf[3 * r + s];
        for (int k = 0; k < 9; k++)
            if (!isfinite(PBf[k])) return OB_ERR_NONFINITE;
    }
    return OB_OK;
}

/* dv_a/dt = (1/rho0) sum_b V (PB_a + PB_b) grad_a W_ab  (Sec. 3.1, momentum
 * equation with the pair-averaged stress); kick the free axes. */
static double stage_force_kick(ob_body *b, double dt) {
    int d = b->dim;
    double amax = 0.0;
    for (int64_t a = 0; a < b->n; a++) {
        double acc[3] = {0, 0, 0};
        for (int64_t p = b->off[a]; p < b->off[a + 1]; p++) {
            int64_t j = b->nbr[p];
            double g[3];
            grad_w(b, a, j, g);
            for (int r = 0; r < d; r++)
                for (int s = 0; s < d; s++)
                    acc[r] += b->V * (b->PB[9 * a + 3 * r + s] + b->PB[9 * j + 3 * r + s]) * g[s];
        }
        double am2 = 0.0;
        for (int r = 0; r < d; r++) {
            acc[r] /= b->rho0;
            b->acc[3 * a + r] = acc[r];
            if (!(b->fix[a] & (1u << r))) {
                b->v[3 * a + r] += dt * acc[r];
                am2 += acc[r] * acc[r];
            }
        }
        double am = sqrt(am2);
        if (am > amax) amax = am;
    }
    return amax;
}

/* one backward-Euler update of one damping pair (Sec. 4.3) */
static void damp_pair(ob_body *b, int64_t a, int64_t j, double dt, double coef) {
    double m = b->rho0 * b->V;
    for (int k = 0; k < b->dim; k++) {
        double ima = (b->fix[a] & (1u << k)) ? 0.0 : 1.0 / m;
        double imb = (b->fix[j] & (1u << k)) ? 0.0 : 1.0 / m;
        double w = b->v[3 * a + k] - b->v[3 * j + k];
        double wn = w / (1.0 + dt * coef * (ima + imb));
        b->v[3 * a + k] -= dt * coef * wn * ima;
        b->v[3 * j + k] += dt * coef * wn * imb;
    }
}

/* B_ab = -2 eta V_a V_b W'(r0_ab)/r0_ab  (Sec. 4.3, viscous damping) */
static double damp_coef(const ob_body *b, int64_t a, int64_t j) {
    /* anisotropic kernel: the same formula on the scaled distance |s (.) d|
     * (the damping is a relaxation device; its form does not move the
     * equilibrium) */
    double r2 = 0.0;
    for (int k = 0; k < 3; k++) {
        double dd = (b->X[3 * a + k] - b->X[3 * j + k]) * b->sk[k];
        r2 += dd * dd;
    }
    double r = sqrt(r2);
    return -2.0 * b->eta * b->V * b->V * ob_kernel_dwdr(b->dim, b->h, r) / r;
}

/* Symmetric sweep: every pair once in canonical order with dt/2, then once
 * in the reverse order with dt/2.  A single one-directional sweep makes the
 * kick-damp-drift substep unstable for eta >= 1e4 (spectral radius of the
 * linearised substep above 1), the symmetric sweep keeps it at 1. */
static void stage_damping(ob_body *b, double dt) {
    if (b->eta == 0.0) return;
    double hdt = 0.5 * dt;
    for (int64_t t = 0; t < b->npairs; t++) {
        int64_t a = b->pa[t], j = b->pb[t];
        damp_pair(b, a, j, hdt, damp_coef(b, a, j));
    }
    for (int64_t t = b->npairs - 1; t >= 0; t--) {
        int64_t a = b->pa[t], j = b->pb[t];
        damp_pair(b, a, j, hdt, damp_coef(b, a, j));
    }
}

/* Constrained axes: v = 0, u = prescribed; free axes: u += dt v.  Then
 * E_k = sum 1/2 m |v|^2 and |v|max. */
static void stage_bc_drift(ob_body *b, double dt, double ramp, double *ke, double *vmax) {
    double m = b->rho0 * b->V;
    double e = 0.0, vm = 0.0;
    for (int64_t a = 0; a < b->n; a++) {
        double v2 = 0.0;
        for (int k = 0; k < b->dim; k++) {
            if (b->fix[a] & (1u << k)) {
                b->v[3 * a + k] = 0.0;
                b->u[3 * a + k] = ramp * b->u_unit[3 * a + k];
            } else {
                b->u[3 * a + k] += dt * b->v[3 * a + k];
            }
            v2 += b->v[3 * a + k] * b->v[3 * a + k];
        }
        e += 0.5 * m * v2;
        if (sqrt(v2) > vm) vm = sqrt(v2);
    }
    *ke = e;
    *vmax = vm;
}

int ob_substep(ob_body *b, double dt, double ramp, double *ke, double *vmax, double *amax) {
    int st = stage_stress(b);
    if (st != OB_OK) return st;
    double am = stage_force_kick(b, dt);
    stage_damping(b, dt);
    stage_bc_drift(b, dt, ramp, ke, vmax);
    *amax = am;
    b->last_amax = am;
    if (!isfinite(*ke)) return OB_ERR_NONFINITE;
    return OB_OK;
}

/* partial substep for stage-by-stage comparisons: 1 = F + stress + PB,
 * 2 = + force/kick, 3 = + damping, 4 = + BC/drift (full substep) */
int ob_substep_partial(ob_body *b, double dt, double ramp, int upto, double out[3]) {
    out[0] = out[1] = out[2] = 0.0;
    int st = stage_stress(b);
    if (st != OB_OK || upto <= 1) return st;
    out[2] = stage_force_kick(b, dt);
    if (upto <= 2) return OB_OK;
    stage_damping(b, dt);
    if (upto <= 3) return OB_OK;
    stage_bc_drift(b, dt, ramp, &out[0], &out[1]);
    return OB_OK;
}

/* ------------------------------------------------------------------ */
/* Slow process: diffusion (Sec. 2.2 Fick's law, Sec. 3.2, reduced to a */
/* scalar concentration; explicit Jacobi update).                       */
/* ------------------------------------------------------------------ */
static void defgrad(const ob_body *b, int64_t a, double F[9]);
static double two_stage_bound(const ob_body *b);

int ob_diffusion_dt(const ob_body *b, double *dt_paper, double *dt_stable) {
    /* Sec. 4.1: dt_d = 0.5 h^2 / D.  Max-principle bound: 1/max_i sum_j a_ij
     * with a_ij = 2 D V |W'_ij|/r_ij; the stable step is 0.9 of it.  For the
     * two-stage form: 0.9 * 2 / (a Gershgorin bound of its operator at the
     * current deformation). */
    *dt_paper = b->D > 0 ? 0.5 * b->h * b->h / b->D : INFINITY;
    if (b->diff_mode == 1) {
        double lam = two_stage_bound(b);
        *dt_stable = lam > 0 ? 1.8 / lam : INFINITY;
        return OB_OK;
    }
    double amax = 0.0;
    for (int64_t i = 0; i < b->n; i++) {
        double s = 0.0;
        for (int64_t p = b->off[i]; p < b->off[i + 1]; p++) {
            int64_t j = b->nbr[p];
            double r2 = 0.0;
            for (int k = 0; k < 3; k++) {
                double dd = b->X[3 * i + k] - b->X[3 * j + k];
                r2 += dd * dd;
            }
            double r = sqrt(r2);
            s += 2.0 * b->D * b->V * fabs(ob_kernel_dwdr(b->dim, b->h, r)) / r;
        }
        if (s > amax) amax = s;
    }
    *dt_stable = amax > 0 ? 0.9 / amax : INFINITY;
    return OB_OK;
}

/* Gershgorin bound of the two-stage operator c -> dc/dt: with s1_x =
 * sum_b V |grad0 W_xb|_1 and R_x = 2 D J_x |C_x^-1 B0_x^T|_inf s1_x (a bound
 * of the coefficient sum of each component of Q_x), every row of the
 * operator has absolute sum <= sum_b V |grad0 W_ab|_1 (R_a + R_b). */
static double two_stage_bound(const ob_body *b) {
    int d = b->dim;
    double *R = malloc((size_t)b->n * sizeof(double));
    if (!R) return INFINITY;
    for (int64_t a = 0; a < b->n; a++) {
        double s1 = 0.0;
        for (int64_t p = b->off[a]; p < b->off[a + 1]; p++) {
            double w[3];
            grad_w(b, a, b->nbr[p], w);
            for (int k = 0; k < d; k++) s1 += b->V * fabs(w[k]);
        }
        double F[9], Ft[9], Cm[9], Ci[9];
        defgrad(b, a, F);
        m3_transpose(F, Ft);
        m3_mul(Ft, F, Cm);
        m3_inv(Cm, Ci);
        double J = m3_det(F);
        double nrm = 0.0;   /* |C^-1 B0^T|_inf over the d x d block */
        for (int r = 0; r < d; r++) {
            double row = 0.0;
            for (int k = 0; k < d; k++) {
                double m = 0.0;
                for (int q = 0; q < d; q++) m += Ci[3 * r + q] * b->B0[9 * a + 3 * k + q];
                row += fabs(m);
            }
            if (row > nrm) nrm = row;
        }
        R[a] = 2.0 * b->D * fabs(J) * nrm * s1;
    }
    double lam = 0.0;
    for (int64_t a = 0; a < b->n; a++) {
        double row = 0.0;
        for (int64_t p = b->off[a]; p < b->off[a + 1]; p++) {
            int64_t j = b->nbr[p];
            double w[3], w1 = 0.0;
            grad_w(b, a, j, w);
            for (int k = 0; k < d; k++) w1 += fabs(w[k]);
            row += b->V * w1 * (R[a] + R[j]);
        }
        if (row > lam) lam = row;
    }
    free(R);
    return lam;
}

/* Two-stage diffusion in the deformed configuration (Sec. 3.2, flux then its
 * divergence, kernel gradients mapped by F).  Written in the reference
 * configuration through the Piola transform of the flux:
 *   stage 1: g_a = B0_a^T sum_b V (c_b - c_a) grad0_a W_ab   (corrected reference gradient)
 *            Q_a = -D J_a C_a^-1 g_a,  C = F^T F,  J = det F
 *   stage 2: c_a <- c_a - dt sum_b V (Q_a + Q_b) . grad0_a W_ab   (free-c particles)
 * The pair form of stage 2 is antisymmetric in a, b, so sum c is conserved
 * when nothing is held. */
static int diffusion_step_two_stage(ob_body *b, double dt) {
    int d = b->dim;
    double *Q = calloc((size_t)b->n * 3, sizeof(double));
    double *cn = malloc((size_t)b->n * sizeof(double));
    if (!Q || !cn) { free(Q); free(cn); return OB_ERR_OOM; }
    for (int64_t a = 0; a < b->n; a++) {
        double g[3] = {0, 0, 0};
        for (int64_t p = b->off[a]; p < b->off[a + 1]; p++) {
            int64_t j = b->nbr[p];
            double w[3];
            grad_w(b, a, j, w);
            for (int k = 0; k < d; k++) g[k] += b->V * (b->c[j] - b->c[a]) * w[k];
        }
        double g0[3] = {0, 0, 0};            /* B0^T g */
        for (int r = 0; r < d; r++)
            for (int k = 0; k < d; k++) g0[r] += b->B0[9 * a + 3 * k + r] * g[k];
        double F[9], Ft[9], Cm[9], Ci[9];
        defgrad(b, a, F);
        m3_transpose(F, Ft);
        m3_mul(Ft, F, Cm);
        m3_inv(Cm, Ci);
        double J = m3_det(F);
        for (int r = 0; r < d; r++) {
            double s = 0.0;
            for (int k = 0; k < d; k++) s += Ci[3 * r + k] * g0[k];
            Q[3 * a + r] = -b->D * J * s;
        }
    }
    for (int64_t a = 0; a < b->n; a++) {
        if (b->cheld[a]) { cn[a] = b->cheld_val[a]; continue; }
        double s = 0.0;
        for (int64_t p = b->off[a]; p < b->off[a + 1]; p++) {
            int64_t j = b->nbr[p];
            double w[3];
            grad_w(b, a, j, w);
            for (int k = 0; k < d; k++) s += b->V * (Q[3 * a + k] + Q[3 * j + k]) * w[k];
        }
        cn[a] = b->c[a] - dt * s;
    }
    memcpy(b->c, cn, (size_t)b->n * sizeof(double));
    free(Q);
    free(cn);
    return OB_OK;
}

int ob_set_diffusion_mode(ob_body *b, int mode) {
    if (mode != 0 && mode != 1) return OB_ERR_ARG;
    b->diff_mode = mode;
    return OB_OK;
}

int ob_diffusion_step(ob_body *b, double dt) {
    if (b->diff_mode == 1) return diffusion_step_two_stage(b, dt);
    /* the one-pass pairwise Laplacian is not consistent for an anisotropic
     * kernel (its second moment is not isotropic): two-stage form only */
    if (b->aniso) return OB_ERR_STATE;
    double *cn = malloc((size_t)b->n * sizeof(double));
    if (!cn) return OB_ERR_OOM;
    for (int64_t i = 0; i < b->n; i++) {
        if (b->cheld[i]) { cn[i] = b->cheld_val[i]; continue; }
        double s = 0.0;
        for (int64_t p = b->off[i]; p < b->off[i + 1]; p++) {
            int64_t j = b->nbr[p];
            double r2 = 0.0;
            for (int k = 0; k < 3; k++) {
                double dd = b->X[3 * i + k] - b->X[3 * j + k];
                r2 += dd * dd;
            }
            double r = sqrt(r2);
            s += 2.0 * b->D * b->V * (b->c[i] - b->c[j]) * ob_kernel_dwdr(b->dim, b->h, r) / r;
        }
        cn[i] = b->c[i] + dt * s;
    }
    memcpy(b->c, cn, (size_t)b->n * sizeof(double));
    free(cn);
    return OB_OK;
}

/* ------------------------------------------------------------------ */
/* Slow step (Sec. 4.2): outer increment, then damped substeps until the */
/* kinetic-energy criterion holds or max_substeps is reached.           */
/* After a load or diffusion event the kinetic energy first rises to a   */
/* peak and then decays under the damping to the criterion (Sec. 5.1 and */
/* Sec. 5.3, the kinetic-energy evolution after one stretching or one    */
/* diffusion step).  The criterion is therefore tested only once the     */
/* energy has stopped rising: from the first substep n with              */
/* E_k(n) <= E_k(n-1), where E_k(0) = 0 (the relaxation starts from the  */
/* event; a body that does not move at all is armed at once).  Once      */
/* armed it stays armed for the rest of the slow step.                   */
/* ------------------------------------------------------------------ */
int ob_advance_slow_step(ob_body *b, const ob_step_params *p, ob_report *rep) {
    memset(rep, 0, sizeof(*rep));
    if (p->max_substeps < 1 || !isfinite(p->ramp_value) || p->dt_slow < 0) return OB_ERR_ARG;
    /* load increment: jump the prescribed axes to ramp * u_unit (Sec. 4.1, dt_l) */
    for (int64_t a = 0; a < b->n; a++)
        for (int k = 0; k < b->dim; k++)
            if (b->fix[a] & (1u << k)) {
                b->u[3 * a + k] = p->ramp_value * b->u_unit[3 * a + k];
                b->v[3 * a + k] = 0.0;
            }
    if (p->dt_slow > 0.0) {
        if (!b->has_diff) return OB_ERR_STATE;
        double dtp, dts;
        ob_diffusion_dt(b, &dtp, &dts);
        if (p->dt_slow > dts * (1.0 + 1e-12) && !p->force_dt) return OB_ERR_UNSTABLE_DT;
        int st = ob_diffusion_step(b, p->dt_slow);
        if (st != OB_OK) return st;
    }
    /* Sec. 4.1: dt_s = 0.6 min(h/(c_s + |v|max), sqrt(h/|dv/dt|max)), c_s = sqrt(K/rho0) */
    double cs = sqrt(b->K / b->rho0);
    double dt = p->dt_sub_override > 0 ? p->dt_sub_override : 0.6 * b->h / cs;
    double volume = (double)b->n * b->V;
    int64_t nsub = 0;
    double ke = 0, vmax = 0, amax = 0;
    int converged = 0;
    double ke_prev = 0.0;   /* E_k(0) */
    int armed = 0;
    for (;;) {
        int st = ob_substep(b, dt, p->ramp_value, &ke, &vmax, &amax);
        if (st != OB_OK) { rep->status = st; rep->substeps = nsub + 1; return st; }
        nsub++;
        rep->dt_last = dt;
        if (ke <= ke_prev) armed = 1;       /* past the peak of E_k */
        ke_prev = ke;
        double crit = p->ke_mode == 1 ? ke / volume : ke;
        if (p->ke_tol >= 0.0 && armed && crit <= p->ke_tol * p->ke_ref) { converged = 1; break; }
        if (nsub >= p->max_substeps) break;
        if (p->dt_sub_override > 0) dt = p->dt_sub_override;
        else {
            double t1 = b->h / (cs + vmax);
            double t2 = sqrt(b->h / amax);
            dt = 0.6 * (t1 < t2 ? t1 : t2);
        }
    }
    rep->substeps = nsub;
    rep->converged = converged;
    rep->ke_final = ke;
    rep->max_v = vmax;
    rep->max_a = amax;
    double m = b->rho0 * b->V;
    int64_t nt = 0;
    for (int64_t a = 0; a < b->n; a++) {
        if (b->fgrp[a])
            for (int k = 0; k < b->dim; k++) rep->end_force[k] -= m * b->acc[3 * a + k];
        if (b->tgrp[a]) {
            nt++;
            for (int k = 0; k < b->dim; k++) rep->tip_deflection[k] += b->u[3 * a + k];
        }
    }
    if (nt > 0)
        for (int k = 0; k < b->dim; k++) rep->tip_deflection[k] /= (double)nt;
    return OB_OK;
}

/* ------------------------------------------------------------------ */
/* field access, original particle order                                */
/* ------------------------------------------------------------------ */
int ob_read_field(const ob_body *b, int field, double *out) {
    int d = b->dim;
    for (int64_t s = 0; s < b->n; s++) {
        int64_t i = b->perm[s];
        switch (field) {
        case OB_F_U: for (int k = 0; k < d; k++) out[i * d + k] = b->u[3 * s + k]; break;
        case OB_F_X: for (int k = 0; k < d; k++) out[i * d + k] = b->X[3 * s + k]; break;
        case OB_F_V: for (int k = 0; k < d; k++) out[i * d + k] = b->v[3 * s + k]; break;
        case OB_F_ACC: for (int k = 0; k < d; k++) out[i * d + k] = b->acc[3 * s + k]; break;
        case OB_F_DEFGRAD: {
            double F[9];
            defgrad(b, s, F);
            memcpy(out + 9 * i, F, sizeof(F));
            break;
        }
        case OB_F_PB:
            for (int r = 0; r < d; r++)
                for (int c = 0; c < d; c++) out[i * d * d + r * d + c] = b->PB[9 * s + 3 * r + c];
            break;
        case OB_F_C: out[i] = b->c[s]; break;
        case OB_F_ALPHA: out[i] = b->alpha[s]; break;
        case OB_F_CPINV: memcpy(out + 6 * i, b->cpinv + 6 * s, 6 * sizeof(double)); break;
        default: return OB_ERR_ARG;
        }
    }
    return OB_OK;
}

int ob_write_field(ob_body *b, int field, const double *in) {
    int d = b->dim;
    for (int64_t s = 0; s < b->n; s++) {
        int64_t i = b->perm[s];
        switch (field) {
        case OB_F_U: for (int k = 0; k < d; k++) b->u[3 * s + k] = in[i * d + k]; break;
        case OB_F_V: for (int k = 0; k < d; k++) b->v[3 * s + k] = in[i * d + k]; break;
        case OB_F_C: b->c[s] = in[i]; break;
        case OB_F_ALPHA: b->alpha[s] = in[i]; break;
        case OB_F_CPINV: memcpy(b->cpinv + 6 * s, in + 6 * i, 6 * sizeof(double)); break;
        default: return OB_ERR_ARG;
        }
    }
    return OB_OK;
}

int ob_b0(const ob_body *b, double *out) {
    /* B0 in original order, d x d row-major */
    int d = b->dim;
    for (int64_t s = 0; s < b->n; s++) {
        int64_t i = b->perm[s];
        for (int r = 0; r < d; r++)
            for (int c = 0; c < d; c++) out[i * d * d + r * d + c] = b->B0[9 * s + 3 * r + c];
    }
    return OB_OK;
}

int ob_dim(const ob_body *b) { return b->dim; }
int64_t ob_n(const ob_body *b) { return b->n; }
double ob_h(const ob_body *b) { return b->h; }
