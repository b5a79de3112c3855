/*
 * mtssph.h -- C ABI of the GB300 (sm_103a) multi-time-step SPH solid library.
 *
 * The library advances an elastic or elasto-plastic particle body with the
 * explicit multi-time-step scheme of Tang, Wu, Wang, Haidn and Hu, "An
 * explicit multi-time stepping algorithm for multi-time scale coupling
 * problems in SPH" (arXiv 2309.04010): an outer slow step (a load increment,
 * Sec. 4.1 dt_l, or an explicit concentration-diffusion step, Sec. 4.1 dt_d)
 * followed by many damped total-Lagrangian solid substeps (Sec. 3.1, Sec. 4.3)
 * until the kinetic-energy criterion of Sec. 4.2 holds.
 *
 * Conventions for every call:
 *   - every function returns mts_status (MTS_OK = 0); no C++ exception or
 *     longjmp crosses the ABI; mts_last_error() gives a message for the last
 *     failing call on the calling thread;
 *   - host pointers are plain host memory owned by the caller; the library
 *     copies what it needs before returning and never keeps a host pointer;
 *   - particle arrays passed in or out use the caller's ORIGINAL particle
 *     order; vectors are n x dim row-major, FP64;
 *   - device memory belongs to the library (allocated through the context's
 *     allocator) and is released by the matching destroy call;
 *   - calls on one context (and its bodies) are not thread-safe; all GPU work
 *     of a context is ordered on the context's stream;
 *   - a call that fails leaves the body usable unless it returns MTS_ERR_CUDA.
 */
#ifndef MTSSPH_H
#define MTSSPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MTS_OK = 0,
    MTS_ERR_INVALID_ARG = 1, /* a pointer, size or parameter is out of range        */
    MTS_ERR_OOM = 2,         /* the allocator returned NULL                          */
    MTS_ERR_CUDA = 3,        /* a CUDA runtime call failed (message has the code)   */
    MTS_ERR_SINGULAR_B = 4,  /* a correction matrix sum (Sec. 3.1) is singular      */
    MTS_ERR_NONFINITE = 5,   /* NaN/Inf in an input or in the kinetic energy         */
    MTS_ERR_TIMEOUT = 6,     /* reserved: a device wait ran out of its limit         */
    MTS_ERR_UNSTABLE_DT = 7, /* diffusion step above the stable limit                */
    MTS_ERR_STATE = 8        /* call not valid in the current state                  */
} mts_status;

typedef enum { MTS_FP64 = 0, MTS_MIXED = 1 } mts_precision;
typedef enum { MTS_ELASTIC_SVK = 0, MTS_NEOHOOKE_J2 = 1 } mts_material_model;

typedef struct mts_ctx mts_ctx;
typedef struct mts_body mts_body;
typedef struct mts_batch mts_batch;

/* Device allocator hook.  alloc returns a device pointer (NULL on failure),
 * aligned to at least 16 bytes (the kernels move arrays with 16-byte vector
 * loads and asynchronous copies; cudaMalloc and PyTorch's caching allocator
 * align to 256 bytes or more); release frees it.  A misaligned pointer is
 * released again and the call fails with MTS_ERR_INVALID_ARG.  Pass NULL to
 * mts_ctx_create to use cudaMalloc/cudaFree.  The Python binding passes
 * PyTorch's caching allocator here. */
typedef struct {
    void *(*alloc)(size_t bytes, void *user);
    void (*release)(void *ptr, size_t bytes, void *user);
    void *user;
} mts_allocator;

/* Context: one CUDA device and one stream.  stream = NULL creates a private
 * non-blocking stream owned by the context; otherwise the caller's
 * cudaStream_t is used and stays owned by the caller.  The captured substep
 * graphs launch their kernels with programmatic dependent launch (each kernel
 * may start while the previous one drains); setting the environment variable
 * MTS_NO_CHAIN_LAUNCH before the context is created turns that off, and a
 * capture that fails with it enabled is retried once without it. */
mts_status mts_ctx_create(int device, void *cuda_stream, const mts_allocator *alloc,
                          mts_ctx **out);
/* Destroy every body of the context first: a body keeps a pointer to it. */
void mts_ctx_destroy(mts_ctx *ctx);
/* Message for the last failing call on this thread ("" if none). */
const char *mts_last_error(void);
/* Library version: major * 10000 + minor * 100 + patch. */
int mts_version(void);

/* ------------------------------------------------------------------ */
/* Body and its fixed neighbourhood (Sec. 3.1: total Lagrangian, the    */
/* neighbour set and the correction matrix B0 are built once in the     */
/* reference configuration).                                             */
/* ------------------------------------------------------------------ */
typedef enum {
    MTS_DAMP_AUTO = 0,       /* library's choice (reported by mts_body_damping_layout): */
                             /* currently BLOCKS, the faster kernel where measured      */
    MTS_DAMP_BLOCKS = 1,     /* blocks on every axis, one warp per owner block,       */
                             /* at most 32 pairs per sub-colour                       */
    MTS_DAMP_WIDE = 2        /* shortest axis unblocked, one CTA per owner block,     */
                             /* no cap on pairs per sub-colour (MTS_ERR_INVALID_ARG   */
                             /* when an owner group does not fit one CTA)             */
} mts_damp_layout;

typedef struct {
    int32_t dim;             /* 2 (plane strain) or 3                                 */
    int32_t precision;       /* mts_precision                                         */
    int64_t n;               /* particle count, 2 <= n < 2^31                         */
    const double *X;         /* host, n x dim reference positions, copied             */
    double dx;               /* lattice spacing: particle volume dx^dim               */
    double h_over_dx;        /* smoothing length h = h_over_dx * dx, support 2h       */
    int32_t damp_layout;     /* mts_damp_layout of the pairwise damping order         */
    int32_t tile;            /* particles per Morton tile of the gather kernels (their */
                             /* block size): 0 = default (512 mixed, 128 FP64), else  */
                             /* 64, 128, 256 or 512 (mixed) / 64 or 128 (FP64)        */
    double dx_axis[3];       /* lattice spacing per axis (the anisotropic kernel of   */
                             /* thin bodies); all 0 = dx on every axis.  Otherwise dx */
                             /* is ignored, h = h_over_dx * min spacing and the       */
                             /* kernel is detS W(|s (.) x|), s_k = min spacing / dx_k */
} mts_body_desc;

/* Builds, on the GPU: the Morton order of the particles (cell = floor((X -
 * Xmin)/dx), bit-interleaved key with x lowest, ties by original index), the
 * neighbour CSR (all j != i with |X_i - X_j|^2 < (2h)^2 evaluated in FP64
 * without fused multiply-add, ascending), B0 (Sec. 3.1, correction matrix),
 * and the canonical damping order: owner blocks (width 2^shift cells per
 * blocked axis, 2^shift * dx > 2h), pair owner = componentwise-min block of
 * its particles, colour = parity bits of the owner, and inside an owner block
 * a greedy sub-colouring that visits pairs by sign-folded cell-offset class
 * and then (a, b), taking the smallest sub-colour unused at a and b (with room
 * under the level cap).  Errors: MTS_ERR_INVALID_ARG (bad desc, non-finite
 * X), MTS_ERR_SINGULAR_B, MTS_ERR_OOM. */
mts_status mts_body_create(mts_ctx *ctx, const mts_body_desc *desc, mts_body **out);
void mts_body_destroy(mts_body *body);

/* The damping order's layout (part of its definition, Sec. 4.3 ordering
 * reading): shift[k] = log2 of the owner-block width in cells on axis k, or
 * MTS_WHOLE_AXIS when axis k is not blocked; *level_cap = the cap on pairs per
 * sub-colour of one owner block (0 = none). */
#define MTS_WHOLE_AXIS 62
mts_status mts_body_damping_layout(const mts_body *body, int32_t shift[3], int32_t *level_cap);

/* Launch shapes of the substep kernels.  tile: particles per Morton tile of
 * the gather kernels (= their threads per block; 0 keeps the current tiles,
 * otherwise as mts_body_desc.tile) — the tiles are rebuilt, which changes the
 * rounding of the tile-relative positions but not the method; damp_warps:
 * owner groups (warps) per CTA of the damping kernel, 0 = as many of 4, 2, 1
 * as fit the shared memory, else 1, 2 or 4 (reduced while it does not fit;
 * the results do not depend on it).  mts_body_shapes reports the shapes in
 * use.  Errors: MTS_ERR_INVALID_ARG for other values or a NULL body. */
mts_status mts_body_set_shapes(mts_body *body, int32_t tile, int32_t damp_warps);
mts_status mts_body_shapes(const mts_body *body, int32_t *tile, int32_t *damp_warps);

/* Autotuner of the launch shapes: for every candidate (tiles 256 and 512 in
 * mixed precision, 64 and 128 in FP64; 1, 2 and 4 damping warps per CTA) it
 * runs one slow step of `substeps` substeps (load scale `ramp`, no
 * kinetic-energy stop, the production device loop) twice from the body's
 * current state and times the second run with CUDA events on the context's
 * stream; the fastest candidate (the first on ties) is applied and the state
 * is restored (mts_save_state / mts_load_state), so the body continues as if
 * the tuner had not run.  tile, damp_warps, best_ms: the choice and its time
 * (may be NULL).  substeps in [1, 1000]. */
mts_status mts_body_autotune(mts_body *body, int32_t substeps, double ramp, int32_t *tile,
                             int32_t *damp_warps, double *best_ms);

/* Sorted position -> original index (n entries, host). */
mts_status mts_body_permutation(const mts_body *body, int64_t *perm);
/* Neighbour CSR in SORTED index space.  *nnz receives the entry count;
 * offsets (n + 1) and idx (nnz) are filled when non-NULL. */
mts_status mts_body_neighbors(const mts_body *body, int64_t *nnz, int64_t *offsets,
                              int32_t *idx);
/* Canonical pairwise-damping order (Sec. 4.3, pairwise splitting): one entry
 * per neighbour pair a < b (sorted indices), listed in the sequential order
 * colour, owner-block Morton key, sub-colour, a, b.  Pairs of one (colour,
 * sub-colour) touch disjoint particles.  Any output pointer may be NULL. */
mts_status mts_body_colouring(const mts_body *body, int64_t *npairs, int32_t *pair_a,
                              int32_t *pair_b, int32_t *colour, int64_t *block_key,
                              int32_t *sub_colour);

/* ------------------------------------------------------------------ */
/* Material, damping, diffusion and boundary conditions                  */
/* ------------------------------------------------------------------ */
/* App. A / App. B.2.  E, nu give mu = E/(2(1+nu)), K = E/(3(1-2nu)),
 * lambda = K - 2mu/3 (App. A.2 moduli relation).  MTS_ELASTIC_SVK: St
 * Venant-Kirchhoff; MTS_NEOHOOKE_J2: Alg. 1 with k(a) = sigma0 +
 * (sigma_inf - sigma0)(1 - exp(-delta a)) + H a.  Hardening arguments are
 * ignored for SVK. */
mts_status mts_set_material(mts_body *body, mts_material_model model, double rho0, double E,
                            double nu, double sigma0, double sigma_inf, double delta,
                            double H);
/* Sec. 4.3 viscous damping coefficient eta >= 0 (0 switches damping off). */
mts_status mts_set_damping(mts_body *body, double eta);
/* Slow process (Sec. 2.2 Fick's law reduced to a scalar concentration c):
 * dc_i/dt = 2 D sum_j V (c_i - c_j) W'(r_ij)/r_ij; swelling pressure
 * p = 3 K beta (c - c0) enters the stress as -p J F^-T (App. B.2).  Sets c = c0
 * on particles that are not held. */
mts_status mts_set_diffusion(mts_body *body, double D, double beta, double c0);
/* Prescribed displacement u = ramp * u_unit on the axes of axis_mask (bit k =
 * axis k) for `count` particles `ids` (original indices).  u_unit: host,
 * count x dim, NULL = zeros (clamp).  report_force marks the set whose internal
 * force is reported as the end force.  Calls accumulate. */
mts_status mts_set_bc_displacement(mts_body *body, int64_t count, const int64_t *ids,
                                   uint32_t axis_mask, const double *u_per_unit_ramp,
                                   int32_t report_force);
/* Hold c = c_value on `count` particles (Dirichlet layers of the slow step). */
mts_status mts_set_bc_concentration(mts_body *body, int64_t count, const int64_t *ids,
                                    double c_value);
/* Discretisation of the diffusion step: 0 (default) = the one-pass pairwise
 * Laplacian in the reference configuration; 1 = the two-stage form of
 * Sec. 3.2 in the deformed configuration (flux, then its divergence, kernel
 * gradients mapped by F), written through the Piola transform of the flux:
 * Q_a = -D J_a C_a^-1 B0_a^T sum_b V (c_b - c_a) grad0_a W_ab with C = F^T F,
 * then c_a -= dt sum_b V (Q_a + Q_b) . grad0_a W_ab (conservative pair form).
 * mts_diffusion_dt then reports as the stable step 1.8 / a Gershgorin bound
 * of that operator at the current deformation.  The reverse mode covers
 * mode 0 only. */
mts_status mts_set_diffusion_mode(mts_body *body, int32_t mode);
/* Stop holding c on `count` particles (the end of a time-limited contact,
 * Sec. 5.3-5.4 droplet schedule): their c keeps its value and evolves by
 * diffusion from the next slow step on. */
mts_status mts_release_bc_concentration(mts_body *body, int64_t count, const int64_t *ids);
/* Particles whose mean displacement is reported as the tip deflection. */
mts_status mts_set_tip(mts_body *body, int64_t count, const int64_t *ids);
/* Diffusion step limits: dt_paper = 0.5 h^2 / D (Sec. 4.1) and the stable
 * limit 0.9 / max_i sum_j 2 D V |W'_ij|/r_ij of the explicit update. */
mts_status mts_diffusion_dt(mts_body *body, double *dt_paper, double *dt_stable);

/* ------------------------------------------------------------------ */
/* Slow step with its damped substeps (Sec. 4.1, Sec. 4.2, Sec. 4.3)     */
/* ------------------------------------------------------------------ */
typedef struct {
    double dt_slow;          /* diffusion step; 0 = no diffusion this slow step         */
    double ramp_value;       /* load scale: prescribed u = ramp * u_unit (Sec. 4.1 dt_l) */
    double dt_sub_override;  /* > 0: fixed substep size instead of the Sec. 4.1 rule     */
    double ke_tol;           /* stop when E_k <= ke_tol * ke_ref once E_k has passed its */
                             /* peak (see mts_advance_slow_step); < 0 disables the stop */
    double ke_ref;           /* reference energy (mode 0) or energy density (mode 1)    */
    int64_t max_substeps;    /* cap on substeps (>= 1); reaching it is not an error     */
    int32_t ke_mode;         /* 0: total E_k; 1: E_k per unit volume                    */
    int32_t check_every;     /* 0: the loop runs on the device (CUDA graph WHILE node);  */
                             /* k >= 1: graph chunks of k substeps, stop flag read by   */
                             /* the host after each chunk                               */
    int32_t force_dt;        /* 1: accept dt_slow above the stable diffusion limit      */
    int32_t reserved;
} mts_step_params;

typedef struct {
    int64_t substeps;        /* substeps taken                                         */
    int32_t converged;       /* 1 if the kinetic-energy criterion stopped the loop      */
    int32_t status;          /* mts_status of the step                                 */
    double ke_final;         /* E_k after the last substep                             */
    double max_v;            /* max |v| after the last substep (free axes)             */
    double max_a;            /* max |dv/dt| of the last substep (free axes)            */
    double dt_last;          /* size of the last substep                               */
    double end_force[3];     /* -sum m a over the report_force set, last substep       */
    double tip_deflection[3];/* mean u over the tip set                                */
    int64_t kernel_launches; /* library kernels launched by this call (incl. no-ops)   */
    int64_t prof_count;      /* substeps whose profiled stage was timed (see below)    */
    double prof_ms;          /* summed CUDA-event time of the profiled stage           */
} mts_step_report;

/* One slow step: jump prescribed axes to ramp * u_unit (v = 0 there), run
 * the diffusion step if dt_slow > 0, then substeps (stress, force and kick,
 * symmetric pairwise damping, BC and drift, FP64 kinetic energy) until
 * E_k <= ke_tol * ke_ref or max_substeps.  After the load or diffusion event
 * the kinetic energy first rises, then decays under the damping to the
 * criterion (Sec. 5.1 and 5.3), so the criterion is only tested from the
 * first substep n whose E_k(n) <= E_k(n-1), with E_k(0) = 0 (a body that
 * does not move at all is armed at its first substep).  The substep size follows
 * Sec. 4.1: dt0 = 0.6 h / c_s, then 0.6 min(h / (c_s + |v|max),
 * sqrt(h / |dv/dt|max)) with c_s = sqrt(K / rho0).  The stop flag lives on the
 * device; with check_every = 0 a conditional WHILE graph node runs exactly the
 * substeps needed, otherwise the host checks the flag every check_every
 * substeps (kernels after the stop return at once, so the count is exact).  Errors: MTS_ERR_UNSTABLE_DT, MTS_ERR_NONFINITE (report.status
 * says so too), MTS_ERR_STATE (no material set). */
mts_status mts_advance_slow_step(mts_body *body, const mts_step_params *params,
                                 mts_step_report *report);

/* Batches: many independent bodies advanced by one graph launch per slow
 * step (the batched multi-instance mode of the method).  The graph holds one
 * conditional WHILE node per body with no dependencies between them, so the
 * bodies' substep loops run concurrently on the GPU and each stops on its own
 * kinetic-energy criterion; every body computes exactly what
 * mts_advance_slow_step would compute for it (same kernels, same order).
 * mts_batch_create: `count` >= 1 distinct bodies of one context, borrowed
 * (destroy the batch before any of its bodies).  mts_batch_advance: params
 * and reports are arrays of `count`, in body order; params[i].check_every is
 * ignored (the loops always run on the device); each body's load jump and
 * diffusion step run before the launch.  Errors as mts_advance_slow_step for
 * the first failing body (its index in the message); the reports of all
 * bodies are filled as far as they ran. */
mts_status mts_batch_create(mts_ctx *ctx, int32_t count, mts_body *const *bodies, mts_batch **out);
mts_status mts_batch_advance(mts_batch *batch, const mts_step_params *params,
                             mts_step_report *reports);
/* Autotuner of a batch: the bodies run concurrently in the batch graph, so
 * one launch shape at a time is applied to every body (tile 256 or 512, or
 * 64 or 128 for FP64 bodies; 1, 2 or 4 damping warps) and one batch slow step
 * of `substeps` substeps (load scale `ramp`, no stop) is timed from the
 * bodies' saved states; the fastest shape is applied and the states are
 * restored.  The batch graph is captured again at the next advance. */
mts_status mts_batch_autotune(mts_batch *batch, int32_t substeps, double ramp);
void mts_batch_destroy(mts_batch *batch);

/* Time one stage of every substep with CUDA events recorded inside the
 * captured graph, on the library stream: 0 = off, 1 = stress (deformation
 * gradient, stress, P B0), 2 = force and kick, 3 = the whole damping sweep
 * (all colour launches), 4 = BC, drift and reductions.  The next
 * mts_advance_slow_step reports the summed time in prof_ms over prof_count
 * substeps.  The events add a small cost to each substep. */
mts_status mts_set_profiling(mts_body *body, int32_t stage);

/* Stage-by-stage entry for tests: runs one substep of size dt with load scale
 * ramp up to stage `upto` (1 = deformation gradient + stress + P B0, 2 = +
 * force and kick, 3 = + damping sweep, 4 = + BC and drift, i.e. a full
 * substep) without the stop logic. */
mts_status mts_substep_partial(mts_body *body, double dt, double ramp, int32_t upto);

typedef enum {
    MTS_F_U = 0,       /* displacement, n x dim                              */
    MTS_F_X = 1,       /* reference position, n x dim (read only)            */
    MTS_F_V = 2,       /* velocity, n x dim                                  */
    MTS_F_DEFGRAD = 3, /* deformation gradient from the current u, n x 9     */
    MTS_F_PB = 4,      /* P B0 of the last stress stage, n x dim x dim       */
    MTS_F_C = 5,       /* concentration, n                                   */
    MTS_F_ALPHA = 6,   /* equivalent plastic strain, n                       */
    MTS_F_CPINV = 7,   /* inverse plastic right Cauchy-Green (xx,yy,zz,xy,yz,xz) */
    MTS_F_ACC = 8      /* internal acceleration of the last force stage       */
} mts_field;

/* Copy a field to/from a caller-owned host buffer of exactly `len` doubles
 * (n times the field width), original order.  Writes: U, V, C, ALPHA, CPINV. */
mts_status mts_read_field(mts_body *body, int32_t field, double *host_out, int64_t len);
mts_status mts_write_field(mts_body *body, int32_t field, const double *host_in, int64_t len);

/* Checkpoint / resume of the evolving state (u, its FP32 gather copy in mixed
 * precision, v, the last acceleration, the plastic state C-bar_p^-1 and alpha,
 * the concentration), in the library's own sorted order and storage precision,
 * so that a load followed by the same slow steps reproduces the saved run bit
 * for bit.  Configuration (material, damping, diffusion, BCs) is not part of
 * the state.  mts_save_state: with host_buf == NULL only *bytes is set (the
 * size needed); otherwise *bytes must be at least that size and receives the
 * bytes written.  mts_load_state: the buffer must come from mts_save_state of
 * a body with the same n, dim and precision (checked against the header:
 * MTS_ERR_INVALID_ARG otherwise).  Both synchronise the context stream. */
mts_status mts_save_state(const mts_body *body, void *host_buf, size_t *bytes);
mts_status mts_load_state(mts_body *body, const void *host_buf, size_t bytes);

/* ------------------------------------------------------------------ */
/* Reverse mode (derivatives of slow steps), FP64 arithmetic            */
/* ------------------------------------------------------------------ */
/* With the substep sizes and counts of a forward run held fixed (the size
 * rule of Sec. 4.1 and the kinetic-energy stop of Sec. 4.2 are not
 * differentiated), a slow step is a fixed composition of maps; these calls
 * apply its transpose to an adjoint state (u-bar, v-bar, C-bar_p^-1-bar,
 * alpha-bar, c-bar) and accumulate the derivatives with respect to the
 * parameters theta = (E at fixed nu, sigma_0, sigma_inf, delta, H of the
 * hardening law App. A.3, D of Sec. 2.2, beta of App. B.2).
 *
 * The adjoint arithmetic and its accumulators are FP64 for both precisions.
 * A mixed-precision body (FP32 per-particle arithmetic) is reversed about its
 * own forward states: the forward recomputation runs on the body and tapes
 * its states in FP64, and the transposed substeps run on an FP64 twin that
 * mts_adjoint_enable builds from the body's positions (same order, neighbour
 * lists and damping order; it takes the body's parameters and boundary
 * conditions at every reverse-mode call), so the gradient is that of the
 * FP32 trajectory up to the FP32 rounding of the linearisation point.
 *
 * mts_adjoint_enable: allocate the tape for up to max_substeps substeps of one
 *   slow step (n x 12 doubles per substep in 3D) and a zero adjoint state
 *   (for a mixed-precision body also its FP64 twin); MTS_ERR_STATE for an
 *   anisotropic-kernel body.
 * mts_adjoint_reset: zero the adjoint state and the pending seeds.
 * mts_adjoint_seed: add to the adjoint state the derivative of an objective
 *   with respect to the outputs of the step about to be reversed: u_bar
 *   (host, n x dim, original order, or NULL) with respect to u at the end of
 *   the step, tip_bar[dim] with respect to the reported tip deflection (or
 *   NULL), force_bar[dim] with respect to the reported end force (or NULL).
 * mts_adjoint_slow_step: precondition: the body's state is the one at the
 *   start of the slow step to reverse (mts_load_state of a checkpoint) and
 *   params / substeps are those of its forward run.  Recomputes the step with
 *   a tape (leaving the body at its end, as the forward run did), then applies
 *   the transpose; afterwards the adjoint state is that of the state at the
 *   start of the step, and theta_bar[0..6] (host) has the step's parameter
 *   derivatives ADDED.  MTS_ERR_STATE if the recomputed step does not run
 *   exactly `substeps` substeps.
 * mts_read_adjoint: the adjoint of a state field (U, V, C, ALPHA, CPINV), host,
 *   original order, as mts_read_field. */
mts_status mts_adjoint_enable(mts_body *body, int64_t max_substeps);
mts_status mts_adjoint_reset(mts_body *body);
mts_status mts_adjoint_seed(mts_body *body, const double *u_bar, const double *tip_bar,
                            const double *force_bar);
mts_status mts_adjoint_slow_step(mts_body *body, const mts_step_params *params, int64_t substeps,
                                 double *theta_bar);
mts_status mts_read_adjoint(mts_body *body, int32_t field, double *host_out, int64_t len);

/* Equilibrium (implicit-function) adjoint of the state the body holds, for a
 * slow step relaxed to equilibrium: with x* = G(x*, theta) the substep map's
 * fixed point, lambda = s + A^T lambda (A = dG/dx at x*, s the seeds) is
 * summed as a Neumann series by repeated transposed substeps linearised about
 * x* (substep size: the one the next substep would take), and theta_bar
 * receives sum_k B^T (A^T)^k s (B = dG/dtheta).  Only the mechanical
 * relaxation is reversed: u-bar and v-bar decay, while c-bar and the plastic
 * state's adjoint accumulate their sensitivities; the diffusion step before
 * the relaxation is not included (D gets no contribution).  Stops when
 * |(u-bar, v-bar)| <= tol |(u-bar, v-bar)| at the start (checked every 8
 * iterations); *iters (may be NULL) = transposed substeps run.  Errors:
 * MTS_ERR_TIMEOUT after max_iters without reaching tol, MTS_ERR_STATE (no
 * material / reverse mode not enabled; enable with max_substeps >= 1). */
mts_status mts_adjoint_equilibrium(mts_body *body, int64_t max_iters, double tol,
                                   double *theta_bar, int64_t *iters);

/* ------------------------------------------------------------------ */
/* Self-check                                                           */
/* ------------------------------------------------------------------ */
/* The paper has no counterpart to this call.  In mixed precision the drift
 * and force kernels convert between FP32 and FP64 with integer operations
 * (IEEE 754 binary32/binary64: the same bits as the hardware conversions,
 * round to nearest even, off the FP64 pipe).  This call checks those
 * conversions against the hardware's on n counter-hashed bit patterns
 * (seeded; steered into subnormals, zeros, infinities, NaNs, overflow and
 * exact rounding ties) on the context's device and stream, and waits.
 * mismatches[0]: FP32 -> FP64 results that differ, mismatches[1]: FP64 ->
 * FP32 (two NaNs count as equal).  Allocates 16 bytes of device memory
 * through the context for the counts.  Errors: MTS_ERR_INVALID_ARG (NULL, n < 0),
 * MTS_ERR_OOM, MTS_ERR_CUDA. */
mts_status mts_selftest_conversions(mts_ctx *ctx, int64_t n, uint64_t seed, int64_t *mismatches);

/* ------------------------------------------------------------------ */
/* Allocation-free reduction                                            */
/* ------------------------------------------------------------------ */
/* The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory where they need the result: code whose device
 * memory is entirely owned by another allocator (a framework's caching
 * allocator or a fixed arena), code on a latency-critical path that cannot
 * afford the device-wide synchronisation of cudaMalloc/cudaFree, and code that
 * must not be able to fail with out-of-memory after set-up.
 *
 * Computes E_k = sum_i 1/2 mass |v_i|^2 and max_i |v_i| (|v_i|^2 formed in the
 * velocities' precision, then FP64 accumulation: the reduction the slow-step
 * driver applies after every substep).
 *   v_dev   device, n x dim contiguous velocities: float for MTS_MIXED,
 *           double for MTS_FP64 (caller-owned, read only)
 *   out_dev device, 2 doubles (caller-owned): out_dev[0] = E_k, out_dev[1] = max |v|
 *   stream  cudaStream_t to order the work on (NULL: the default stream); the
 *           call returns without waiting for the result.
 * Allocates nothing: no cudaMalloc, cudaFree or allocator of any library.  Its
 * only working memory is a fixed 16 KiB array of 1,024 block partials in this
 * library's static device memory, present on every GPU that loads the library
 * until the process exits.  The first call on each device looks that array's
 * device address up (with the device current), so make the first call on a
 * device before any stream capture on it.  All calls share the array and every
 * call overwrites the partials it reads, so two calls that overlap on the GPU
 * (for example on two streams) race and give wrong results.
 * Errors: MTS_ERR_INVALID_ARG for NULL pointers, an unsupported precision or
 * dim, n outside [1, MTS_NOALLOC_MAX_N], or a negative/non-finite mass;
 * MTS_ERR_CUDA if a launch fails. */
#define MTS_NOALLOC_MAX_N 2147483647LL
mts_status mts_kinetic_energy_noalloc(const void *v_dev, int32_t precision, int32_t dim, int64_t n,
                                      double mass, double *out_dev, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* MTSSPH_H */
