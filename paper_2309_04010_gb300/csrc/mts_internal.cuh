// mts_internal.cuh -- shared declarations of the sm_103a library (not installed).
//
// Layout in HBM (all particle arrays in Morton-sorted order):
//   X    R[PAD]   reference position relative to Xmin (PAD = 2 in 2D, 4 in 3D)
//   X64  f64[PAD] reference position (setup, reads)
//   u    f64[PAD] displacement, FP64 accumulator (both precisions)
//   uf   R[PAD]   gather copy of u for the neighbour loops (aliases u in FP64)
//   v    R[PAD]   velocity
//   acc  R[PAD]   internal acceleration of the last force stage
//   PB   R[MS]    P B0, rows padded to PAD (MS = 4 in 2D, 12 in 3D)
//   B0   R[MS]    correction matrix, same layout
//   cp   R[8]     C_p^-1 (xx,yy,zz,xy,yz,xz), alpha, pad (J2 only)
//   c    R        concentration
//   flags u8      bits 0-2 fixed axes, 3 force set, 4 tip set, 5 c held
//   halo i32      per Morton tile of T particles: the sorted union of the tile
//                 and its neighbours, staged in shared memory by the kernels
//   lell u16      per tile, neighbour-major local slots into the tile's halo,
//                 padded with the particle's own slot
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/mtssph.h"

namespace mts {

constexpr int kFixMask = 7;
constexpr int kForceBit = 8;
constexpr int kTipBit = 16;
constexpr int kCHeldBit = 32;
constexpr int kBlock = 256;  // threads per block of the per-particle kernels
// threads per block (= particles per Morton tile) of the tile kernels: larger
// FP32 tiles cut the halo per particle (a 512-particle tile of the 3D lattice
// stages ~3.4 halo particles per tile particle, a 256-particle one ~5.7)
template <class R> struct TileThreads { static constexpr int v = sizeof(R) == 4 ? 512 : 256; };
template <class R> constexpr int tile_particles() { return sizeof(R) == 4 ? 512 : 128; }
// largest tile a body of this precision may use (the FP64 reverse-mode
// kernels are built for blocks of at most 128 threads)
inline int tile_max(int rsize) { return rsize == 4 ? 512 : 128; }
constexpr int kLevelCap = 32;  // pairs per damping level: one warp-wide pass

// Shared-memory position of velocity slot s in the warp-per-group damping
// kernel.  With 16-byte slots (FP32 3D), slots are permuted inside aligned
// groups of eight (one 128-byte row of the 32 banks) so that the lattice-
// regular slots of one level spread over the banks; other slot sizes keep
// their order.  The slot area is padded to whole groups of eight (the dummy
// slot of empty level entries is slot nb * mb).
__host__ __device__ __forceinline__ int damp_slot_pos(int s, int slot_bytes) {
    return slot_bytes == 16 ? (s ^ (((s >> 3) * 3) & 7)) : s;
}
__host__ __device__ __forceinline__ int damp_slot_count(int nb_mb) { return (nb_mb + 1 + 7) & ~7; }
// pair_slot of a canonical pair: its slot in the padded per-level layout; bit
// kSlotSwapBit set when the set-up stored the pair's two particles in the
// other order in the slot word (low half: pair_b).  A free pair's update is
// symmetric in its two particles bit for bit, so the order only moves the
// shared-memory accesses.
constexpr int kSlotSwapBit = 62;
constexpr long long kSlotMask = (1LL << kSlotSwapBit) - 1;
constexpr int kWholeAxis = 62; // owner-block shift of an unblocked axis
constexpr int kWideThreads = 256;   // threads of the CTA-per-group damping kernel
constexpr int kWideRing = 8;        // level buffers of its pair-data ring

// ------------------------------------------------------------------ errors
void set_error(const char *fmt, ...);
mts_status cuda_fail(cudaError_t e, const char *what);
#define MTS_CUDA(call)                                        \
    do {                                                      \
        cudaError_t _e = (call);                              \
        if (_e != cudaSuccess) return cuda_fail(_e, #call);   \
    } while (0)
#define MTS_TRY(call)                                         \
    do {                                                      \
        mts_status _s = (call);                               \
        if (_s != MTS_OK) return _s;                          \
    } while (0)

// ------------------------------------------------------------------ control
// Device-resident state of the substep loop.  Kernels read dt, ramp and done
// from here, so one captured graph serves every slow step.
struct Control {
    double dt, ramp, dt_fixed, ke_thr, volume;
    double ke, vmax, amax, dt_last;
    double end_force[3];
    long long nsub, max_sub;
    int done, converged, status, ke_mode;
    int use_tol;
    int armed;                // kinetic energy has stopped rising in this slow step
    unsigned int counter;     // last-block-done counter of the drift kernel
    unsigned int err;         // setup error bits
};

constexpr unsigned kErrSingular = 1u;
constexpr unsigned kErrNonfinite = 2u;
constexpr unsigned kErrTooMany = 4u;

// ------------------------------------------------------------------ args
template <class R>
struct Args {
    long long n;
    int dim;
    // geometry
    const R *X;
    const R *B0;
    // state
    double *u;
    R *uf;
    R *v;
    R *acc;
    R *PB;
    R *cp;
    R *c;
    R *c_tmp;
    const uint8_t *flags;
    const double *u_unit;
    const R *c_held;
    // constants
    R inv_h;       // 1/h
    R kcoef;       // V * (-5 alpha_d / h^2): grad_a W_ab * V = kcoef (1-q/2)^3 (X_a - X_b)
    R inv_rho0;
    R lambda, mu, K, s0, sinf, delta, Hlin;
    R swell;       // 3 K beta
    R c0;
    R dcoef;       // 2 D * kcoef (diffusion, includes V)
    R diffD;       // D (two-stage diffusion)
    int aniso;     // anisotropic kernel: positions scaled by sk
    R sk[3];       // per-axis scale of the positions (1 = isotropic)
    R detS;        // product of sk over the axes
    R *qflux;      // two-stage diffusion: Piola-mapped flux per particle (PAD)
    int swelling;
    double mass, h, cs;
    // damping
    R eta;
    const uint32_t *pair_ab;     // padded: level L in slots [32 L, 32 L + 32)
    const R *pair_g;
    const long long *lvl_pair;   // level -> first pair, total_levels + 1
    const int32_t *grp_lvl;      // group -> first level, n_groups + 1
    const int32_t *touch_start;  // group x NB: first block-sorted position of a touched block
    const int32_t *touch_cnt;
    const uint8_t *grp_cons;     // group -> 1 if a touched particle has a constrained axis
    const int32_t *bperm;        // block-sorted position -> particle
    const uint8_t *bflags;       // flags in block-sorted order (wide layout)
    int transpose;               // damping: apply the transposed pair updates (adjoint)
    int mb;                      // max particles per damping block (local stride)
    int nbw;                     // touched blocks per owner group (2^blocked axes)
    int max_group_pairs;         // largest pair list of one owner group
    int max_group_levels;
    int max_level_pairs;         // largest level (sub-colour of one group)
    // Morton tiles of T particles with their neighbour halo (shared-memory staging)
    int T;                       // particles per tile = threads per CTA
    long long ntiles;            // CTAs of the tiled kernels (= force partials)
    int max_halo;                // largest halo (tile + neighbours)
    const long long *halo_off;   // tile -> first halo entry, ntiles + 1
    const int32_t *halo_idx;     // halo particle indices, ascending per tile
    const R *halo_x;             // per halo entry: X relative to the tile's first particle
    const uint16_t *lself;       // particle -> its slot in its tile's halo
    const uint16_t *lell;        // local neighbour slots, neighbour-major per tile
    const long long *lell_off;   // tile -> first local ELL entry
    const int32_t *tile_w;       // tile -> ELL width
    // device loop control: inside a conditional WHILE graph node the drift
    // kernel sets the node's condition to "not done"
    cudaGraphConditionalHandle cond;
    int use_cond;
    // reductions
    Control *ctrl;
    double *part_force;          // grid x 4 (amax, m a_x, m a_y, m a_z)
    double *part_drift;          // grid x 2 (ke, vmax)
};

// ------------------------------------------------------------------ structs
struct Alloc {
    mts_allocator a;
    bool custom;
};

}  // namespace mts

struct mts_ctx {
    int device;
    cudaStream_t stream;
    bool own_stream;
    bool pdl;             // programmatic dependent launch in captured substep chains
    mts::Alloc alloc;
    std::vector<void *> live;
};

struct mts_body {
    mts_ctx *ctx;
    int dim;
    int precision;
    long long n;
    double dx, h, V, cut2;
    int blk_shift;
    int damp_req;         // requested mts_damp_layout
    int damp_warps_req;   // damping warps per CTA: 0 = as many of 4, 2, 1 as fit
    int tile_req;         // particles per Morton tile requested at creation (0 = default)
    bool pdl_now;         // capturing the substep chain with programmatic launches
    int damp_layout;      // resolved: MTS_DAMP_BLOCKS or MTS_DAMP_WIDE
    bool damp_ring;       // BLOCKS kernel streams the level slots through a ring (set by
                          // prepare_kernels from the groups per colour and the SM count)
    // one-launch damping sweep (BLOCKS layout): every (colour launch, group)
    // of the symmetric sweep is a task taken from a queue in sweep order; a
    // task waits until the earlier tasks that touch its blocks have finished
    int32_t *pd_blk;      // per group x 2^d touched blocks: block index (-1: none)
    uint8_t *pd_req;      // per task x 2^d: earlier tasks of the sweep touching that block
    unsigned *pd_done;    // per block: finished tasks touching it; [pd_nblocks]: the queue
    long long pd_ntasks, pd_nblocks;
    int pd_nph;                 // colour launches of the multi-launch form it replaces
    long long pd_off[17];       // first task of each of them
    long long pd_goff[16];      // first group of its colour
    int pd_mode[16];            // 1 forward, 2 reverse, 3 both
    int pd_grid;                // CTAs of the launch (resident capacity)
    bool pd_on;                 // tables built and the one-launch form in use
    int ax_shift[3];      // owner-block width per axis (kWholeAxis = unblocked)
    int level_cap;        // pairs per sub-colour of one group (0 = none)
    double Xmin[3];
    size_t rsize;  // sizeof(R)

    // setup products
    long long *perm;      // sorted -> original
    long long *rank;      // original -> sorted
    double *X64;          // sorted, PAD
    long long *nb_off;    // CSR
    int32_t *nb_idx;
    long long nnz;

    // canonical damping order
    long long npairs;
    long long *pair_slot;     // slot of each canonical pair in the padded layout
    uint32_t *kpad_ab;        // padded per-level pair words (32 slots per level)
    void *kpad_g;             // padded per-level pair coefficients
    int32_t *pair_a, *pair_b, *pair_col, *pair_sub;
    long long *pair_key;
    uint32_t *pair_ab;
    void *pair_g;
    long long *lvl_pair;
    int32_t *grp_lvl;
    int32_t *touch_start, *touch_cnt;
    uint8_t *grp_cons;           // blocks layout: group touches a constrained particle
    int32_t *bperm;           // block-sorted position -> particle (identity for BLOCKS)
    uint8_t *bflags;          // flags in block-sorted order (WIDE only)
    long long n_groups, n_levels;
    int col_off[9];
    int mb, nbw;
    int max_group_pairs, max_group_levels, max_level_pairs;

    // Morton tiles with neighbour halos
    int T;
    long long ntiles;
    int max_halo;
    long long *halo_off;
    int32_t *halo_idx;
    void *halo_x;             // per halo entry, storage precision: X - X(first particle of tile)
    uint16_t *lself;
    uint16_t *lell;
    long long *lell_off;
    int32_t *tile_w;

    // state
    void *X, *B0, *uf, *v, *acc, *PB, *cp, *c, *c_tmp, *c_held;
    double *u, *u_unit;
    uint8_t *flags;
    std::vector<uint8_t> h_flags;

    // material
    bool has_material;
    int model;
    double rho0, E, nu, K, mu, lambda, s0, sinf, delta, Hlin, eta;
    bool has_diff;
    double D, beta, c0;
    int diff_mode;            // 0: one-pass Laplacian, 1: two-stage flux (deformed configuration)
    // the one-pass operator's Gershgorin bound depends on the reference
    // configuration and D only: kept for the D it was computed with
    bool diff_amax_ok;
    double diff_amax, diff_amax_D;
    // anisotropic kernel: positions are stored scaled by sk (X~ = s (.) X, the
    // kernel isotropic with h in those coordinates); V is the real volume
    int aniso;
    double sk[3], detS;
    void *qflux;              // n x PAD, allocated with diff_mode 1

    // loop machinery
    mts::Control *ctrl;
    mts::Control *h_ctrl;   // pinned
    double *part_force, *part_drift;
    double *scratch;        // n x 9 doubles for field transfers
    unsigned long long *d_first;   // first non-finite index of a written field
    double *h_stage;        // pinned staging for field transfers (n x 9)
    cudaGraphExec_t graph;
    int graph_chunk;
    bool graph_dirty;
    int tip_count;
    int prof_stage;
    int graph_prof_stage;
    bool graph_is_loop;           // conditional WHILE graph (one substep per iteration)
    cudaGraphConditionalHandle cond;
    int use_cond;
    std::vector<cudaEvent_t> prof_ev;   // 2 per substep of a chunk
    long long launches_per_substep;
    long long graph_gen;          // bumped whenever captured kernel arguments go stale

    // reverse mode (FP64 bodies; mts_adjoint_enable)
    long long adj_cap;            // substeps the tape holds (0 = off)
    double *tape_u, *tape_cp, *tape_dt, *tape_c;   // per substep u (n x PAD), C_p^-1 and
                                                   // alpha (n x 8), dt; c before diffusion
    double *adj_u, *adj_v, *adj_cp, *adj_c;        // adjoint state (sorted order)
    double *adj_a, *adj_G;        // scratch: acceleration adjoint, per-particle d x d
    double *adj_theta, *adj_part; // 8 parameter accumulators, per-tile partials
    mts::Control *adj_ctrl;       // dt of the substep being reversed
    double adj_force_seed[3];     // pending end-force adjoint of the next reversed step
    // mixed-precision bodies: an FP64 twin (same positions, so the same order,
    // neighbours and damping order) that holds the tape and the adjoint state;
    // the forward recomputation runs on the body itself
    mts_body *shadow;
};

struct mts_batch {
    mts_ctx *ctx;
    std::vector<mts_body *> bodies;
    std::vector<long long> gens;  // graph_gen of each body at capture
    cudaGraphExec_t graph;
};

namespace mts {
// allocation through the context allocator
void *dalloc(mts_ctx *ctx, size_t bytes);
void dfree(mts_ctx *ctx, void *p);
mts_status dalloc_into(mts_ctx *ctx, void **p, size_t bytes);
template <class T>
inline mts_status dalloc_t(mts_ctx *ctx, T **p, size_t count) {
    return dalloc_into(ctx, reinterpret_cast<void **>(p), count * sizeof(T) + 16);
}

// setup (mts_setup.cu)
mts_status build_body(mts_body *b, const double *hX);

// substep machinery (mts_substep.cu)
mts_status launch_stress(mts_body *b);
mts_status launch_force(mts_body *b);
mts_status launch_damping(mts_body *b, long long *launches = nullptr);
// the damping sweep transposed, on an FP64 adjoint velocity array, dt from ctrl
mts_status launch_damping_adjoint(mts_body *b, double *vbar, Control *ctrl);
// kernel arguments of a body (mts_substep.cu)
template <class R> Args<R> make_args(mts_body *b);
// reverse mode (mts_adjoint.cu), FP64 bodies
mts_status adjoint_prepare(mts_body *b);
// tape entry k: u, C_p^-1 / alpha and dt of `src` (FP64 or mixed) into the tape of
// `dst` (the FP64 body that runs the transposed substeps: src itself, or its twin)
mts_status adjoint_tape(const mts_body *src, mts_body *dst, long long k);
// concentration of `src` (storage precision) into an FP64 device array
mts_status copy_c_to_double(const mts_body *src, double *dst);
mts_status adjoint_substep(mts_body *b, long long k, bool last);
mts_status adjoint_diffusion(mts_body *b, double dt);
mts_status adjoint_load(mts_body *b);
mts_status adjoint_seed(mts_body *b, const double *ubar_orig_dev, const double tip[3]);
mts_status adjoint_out(mts_body *b, int field, double *out_dev);
mts_status adjoint_norm2(mts_body *b, double *part_dev, double *out_dev);
mts_status launch_drift(mts_body *b);
mts_status prepare_kernels(mts_body *b);
mts_status retile(mts_body *b, int T);
int damp_warps_of(const mts_body *b);
// shared memory of the CTA-per-group damping kernel for this body's layout
size_t damp_wide_smem(const mts_body *b);
mts_status update_pair_fixbits(mts_body *b);
mts_status launch_slow_begin(mts_body *b);
mts_status launch_diffusion(mts_body *b, double dt);
mts_status diffusion_bound(mts_body *b, double *amax_sum);
// Gershgorin bound of the two-stage diffusion operator at the current deformation
mts_status diffusion_bound_two_stage(mts_body *b, double *lambda);
mts_status launch_defgrad(mts_body *b, double *out_sorted);
mts_status launch_tip(mts_body *b, double *out3);
mts_status launch_reset_ctrl(mts_body *b, double dt, double dt_fixed, double ramp,
                             long long max_sub, double ke_thr, int ke_mode, int use_tol);
// field transfers in sorted order (device scratch, double)
mts_status field_to_scratch(mts_body *b, int field);
mts_status scratch_to_field(mts_body *b, int field);
int field_width(const mts_body *b, int field);

// kernel-function constants
double kernel_alpha(int dim, double h);
}  // namespace mts
