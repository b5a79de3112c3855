// mts_api.cu -- the C ABI (include/mtssph.h): contexts, bodies, boundary
// conditions, the slow-step driver and field transfers.
//
// The slow-step driver (Sec. 4.2 two-loop scheme) keeps the inner loop on the
// device: a chunk of `check_every` substeps is captured once into a CUDA graph
// and replayed; every kernel reads dt, the load scale and the stop flag from a
// device control block, so the graph is valid for every slow step and the
// substeps after the stop inside a chunk are no-ops.  The host reads the
// control block back once per chunk.
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "mts_internal.cuh"
#include "mts_device.cuh"

namespace mts {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

mts_status cuda_fail(cudaError_t e, const char *what) {
    set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
    return MTS_ERR_CUDA;
}

void *dalloc(mts_ctx *ctx, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (ctx->alloc.custom) {
        p = ctx->alloc.a.alloc(bytes, ctx->alloc.a.user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

void dfree(mts_ctx *ctx, void *p) {
    if (!p) return;
    if (ctx->alloc.custom)
        ctx->alloc.a.release(p, 0, ctx->alloc.a.user);
    else
        cudaFree(p);
}

mts_status dalloc_into(mts_ctx *ctx, void **p, size_t bytes) {
    *p = dalloc(ctx, bytes);
    if (!*p) {
        set_error("device allocation of %zu bytes failed", bytes);
        return MTS_ERR_OOM;
    }
    if (reinterpret_cast<uintptr_t>(*p) & 15u) {
        dfree(ctx, *p);
        *p = nullptr;
        set_error("the allocator returned a pointer not aligned to 16 bytes");
        return MTS_ERR_INVALID_ARG;
    }
    return MTS_OK;
}

}  // namespace mts

using namespace mts;

namespace {

template <class T>
void free_dev(mts_body *b, T *&p) {
    dfree(b->ctx, (void *)p);
    p = nullptr;
}

void body_free(mts_body *b) {
    if (!b) return;
    if (b->shadow) {
        body_free(b->shadow);
        b->shadow = nullptr;
    }
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (cudaEvent_t e : b->prof_ev) cudaEventDestroy(e);
    void **ptrs[] = {(void **)&b->perm, (void **)&b->rank, (void **)&b->X64, (void **)&b->nb_off,
                     (void **)&b->nb_idx, (void **)&b->pair_a, (void **)&b->pair_b,
                     (void **)&b->pair_col, (void **)&b->pair_sub, (void **)&b->pair_key,
                     (void **)&b->pair_ab, (void **)&b->pair_g, (void **)&b->lvl_pair,
                     (void **)&b->grp_lvl, (void **)&b->touch_start, (void **)&b->touch_cnt,
                     (void **)&b->X, (void **)&b->B0, (void **)&b->uf, (void **)&b->v,
                     (void **)&b->acc, (void **)&b->PB, (void **)&b->cp, (void **)&b->c,
                     (void **)&b->c_tmp, (void **)&b->c_held, (void **)&b->u, (void **)&b->u_unit,
                     (void **)&b->flags, (void **)&b->ctrl, (void **)&b->part_force,
                     (void **)&b->part_drift, (void **)&b->scratch, (void **)&b->halo_off,
                     (void **)&b->halo_idx, (void **)&b->halo_x, (void **)&b->lself, (void **)&b->lell,
                     (void **)&b->lell_off, (void **)&b->tile_w, (void **)&b->pair_slot,
                     (void **)&b->kpad_ab, (void **)&b->kpad_g, (void **)&b->bperm,
                     (void **)&b->bflags, (void **)&b->grp_cons, (void **)&b->qflux, (void **)&b->tape_u, (void **)&b->tape_cp,
                     (void **)&b->tape_dt, (void **)&b->tape_c, (void **)&b->adj_u,
                     (void **)&b->adj_v, (void **)&b->adj_cp, (void **)&b->adj_c,
                     (void **)&b->adj_a, (void **)&b->adj_G, (void **)&b->adj_theta,
                     (void **)&b->adj_part, (void **)&b->adj_ctrl, (void **)&b->pd_blk,
                     (void **)&b->pd_req, (void **)&b->pd_done, (void **)&b->d_first};
    for (void **pp : ptrs) {
        dfree(b->ctx, *pp);
        *pp = nullptr;
    }
    if (b->h_ctrl) cudaFreeHost(b->h_ctrl);
    if (b->h_stage) cudaFreeHost(b->h_stage);
    delete b;
}

__global__ void k_init_state(double *u, void *uf, void *v, void *acc, void *cp, void *c,
                             void *c_held, uint8_t *flags, double *u_unit, long long n, int pad,
                             int rsize) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = 0; k < pad; ++k) {
        u[i * pad + k] = 0.0;
        u_unit[i * pad + k] = 0.0;
    }
    flags[i] = 0;
    if (rsize == 4) {
        float *f;
        if (uf) { f = (float *)uf; for (int k = 0; k < pad; ++k) f[i * pad + k] = 0.f; }
        f = (float *)v; for (int k = 0; k < pad; ++k) f[i * pad + k] = 0.f;
        f = (float *)acc; for (int k = 0; k < pad; ++k) f[i * pad + k] = 0.f;
        f = (float *)cp; for (int k = 0; k < 8; ++k) f[i * 8 + k] = k < 3 ? 1.f : 0.f;
        ((float *)c)[i] = 0.f;
        ((float *)c_held)[i] = 0.f;
    } else {
        double *f;
        f = (double *)v; for (int k = 0; k < pad; ++k) f[i * pad + k] = 0.0;
        f = (double *)acc; for (int k = 0; k < pad; ++k) f[i * pad + k] = 0.0;
        f = (double *)cp; for (int k = 0; k < 8; ++k) f[i * 8 + k] = k < 3 ? 1.0 : 0.0;
        ((double *)c)[i] = 0.0;
        ((double *)c_held)[i] = 0.0;
    }
}

// c <- c0 on particles that are not held, c <- c_held on held ones
__global__ void k_set_c(void *c, const void *c_held, const uint8_t *flags, long long n, double c0,
                        int rsize, int only_held) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool held = flags[i] & kCHeldBit;
    if (only_held && !held) return;
    if (rsize == 4)
        ((float *)c)[i] = held ? ((const float *)c_held)[i] : (float)c0;
    else
        ((double *)c)[i] = held ? ((const double *)c_held)[i] : c0;
}

mts_status upload_bc(mts_body *b, const std::vector<double> &u_unit_sorted) {
    cudaStream_t st = b->ctx->stream;
    MTS_CUDA(cudaMemcpyAsync(b->flags, b->h_flags.data(), b->n, cudaMemcpyHostToDevice, st));
    if (!u_unit_sorted.empty())
        MTS_CUDA(cudaMemcpyAsync(b->u_unit, u_unit_sorted.data(),
                                 u_unit_sorted.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    MTS_TRY(update_pair_fixbits(b));
    MTS_CUDA(cudaStreamSynchronize(st));
    return MTS_OK;
}

mts_status get_rank_host(mts_body *b, std::vector<long long> &rank) {
    rank.resize(b->n);
    MTS_CUDA(cudaMemcpyAsync(rank.data(), b->rank, b->n * sizeof(long long), cudaMemcpyDeviceToHost,
                             b->ctx->stream));
    MTS_CUDA(cudaStreamSynchronize(b->ctx->stream));
    return MTS_OK;
}

// The inner loop as a conditional WHILE node whose body is one substep; the
// drift kernel's last block sets the condition to "not done".  No host round
// trip and no work after the stop.  (Event-record nodes are not allowed in a
// conditional body, so profiled runs use capture_chunk instead.)
mts_status capture_loop_once(mts_body *b) {
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    MTS_TRY(prepare_kernels(b));
    cudaStream_t st = b->ctx->stream;
    cudaGraph_t g = nullptr;
    MTS_CUDA(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(e, "cudaGraphConditionalHandleCreate");
    }
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(e, "cudaGraphAddNode(conditional)");
    }
    cudaGraph_t body = np.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(e, "cudaStreamBeginCaptureToGraph");
    }
    b->cond = h;
    b->use_cond = 1;
    b->pdl_now = b->ctx->pdl;
    long long ndamp = 0;
    mts_status s = launch_stress(b);
    if (s == MTS_OK) s = launch_force(b);
    if (s == MTS_OK) s = launch_damping(b, &ndamp);
    if (s == MTS_OK) s = launch_drift(b);
    b->use_cond = 0;
    b->pdl_now = false;
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(st, &captured);
    if (s != MTS_OK || e != cudaSuccess) {
        cudaGraphDestroy(g);
        return s != MTS_OK ? s : cuda_fail(e, "cudaStreamEndCapture");
    }
    b->launches_per_substep = 3 + ndamp;
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate(loop)");
    b->graph_is_loop = true;
    b->graph_prof_stage = 0;
    b->graph_dirty = false;
    return MTS_OK;
}

// A capture that fails with programmatic dependent launch enabled is retried
// once without it (and the context keeps ordinary launches from then on).
template <class F>
mts_status with_chain_fallback(mts_ctx *ctx, F capture) {
    mts_status s = capture();
    if (s != MTS_OK && ctx->pdl) {
        ctx->pdl = false;
        s = capture();
    }
    return s;
}

mts_status capture_loop(mts_body *b) {
    if (b->graph && !b->graph_dirty && b->graph_is_loop) return MTS_OK;
    return with_chain_fallback(b->ctx, [&] { return capture_loop_once(b); });
}

mts_status capture_chunk_once(mts_body *b, int chunk) {
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    MTS_TRY(prepare_kernels(b));
    cudaStream_t st = b->ctx->stream;
    const int ps = b->prof_stage;
    if (ps > 0) {
        while ((int)b->prof_ev.size() < 2 * chunk) {
            cudaEvent_t e;
            MTS_CUDA(cudaEventCreate(&e));
            b->prof_ev.push_back(e);
        }
    }
    MTS_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    mts_status s = MTS_OK;
    long long ndamp = 0;
    auto mark = [&](int k, int stage, int end) {
        if (s == MTS_OK && ps == stage) {
            cudaError_t e = cudaEventRecordWithFlags(b->prof_ev[2 * k + end], st,
                                                     cudaEventRecordExternal);
            if (e != cudaSuccess) s = cuda_fail(e, "cudaEventRecordWithFlags");
        }
    };
    b->pdl_now = b->ctx->pdl && ps == 0;
    for (int k = 0; k < chunk && s == MTS_OK; ++k) {
        mark(k, 1, 0);
        s = launch_stress(b);
        mark(k, 1, 1);
        mark(k, 2, 0);
        if (s == MTS_OK) s = launch_force(b);
        mark(k, 2, 1);
        mark(k, 3, 0);
        if (s == MTS_OK) s = launch_damping(b, &ndamp);
        mark(k, 3, 1);
        mark(k, 4, 0);
        if (s == MTS_OK) s = launch_drift(b);
        mark(k, 4, 1);
    }
    b->pdl_now = false;
    b->launches_per_substep = 3 + ndamp;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (s != MTS_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    b->graph_chunk = chunk;
    b->graph_prof_stage = ps;
    b->graph_is_loop = false;
    b->graph_dirty = false;
    return MTS_OK;
}

mts_status capture_chunk(mts_body *b, int chunk) {
    if (b->graph && !b->graph_dirty && !b->graph_is_loop && b->graph_chunk == chunk &&
        b->graph_prof_stage == b->prof_stage)
        return MTS_OK;
    return with_chain_fallback(b->ctx, [&] { return capture_chunk_once(b, chunk); });
}

// Validation, load jump and diffusion step of one slow step (before its substeps).
mts_status slow_step_begin(mts_body *b, const mts_step_params *p, long long *launches,
                           double *c_tape = nullptr) {
    if (!b->has_material) {
        set_error("mts_advance_slow_step: no material set");
        return MTS_ERR_STATE;
    }
    if (p->max_substeps < 1 || !std::isfinite(p->ramp_value) || !(p->dt_slow >= 0) ||
        !std::isfinite(p->dt_slow) || !(p->dt_sub_override >= 0) || !std::isfinite(p->ke_ref) ||
        !std::isfinite(p->ke_tol) || (p->ke_mode != 0 && p->ke_mode != 1)) {
        set_error("mts_advance_slow_step: invalid step parameters");
        return MTS_ERR_INVALID_ARG;
    }
    MTS_CUDA(cudaSetDevice(b->ctx->device));
    if (p->dt_slow > 0) {
        if (!b->has_diff) {
            set_error("mts_advance_slow_step: dt_slow > 0 without diffusion");
            return MTS_ERR_STATE;
        }
        if (b->aniso && b->diff_mode == 0) {
            set_error("mts_advance_slow_step: an anisotropic kernel needs the two-stage diffusion "
                      "(mts_set_diffusion_mode 1)");
            return MTS_ERR_STATE;
        }
        double dtp, dts;
        MTS_TRY(mts_diffusion_dt(b, &dtp, &dts));
        if (p->dt_slow > dts * (1.0 + 1e-12) && !p->force_dt) {
            set_error("diffusion step %g above the stable limit %g (paper's 0.5 h^2/D = %g)",
                      p->dt_slow, dts, dtp);
            return MTS_ERR_UNSTABLE_DT;
        }
    }
    const double cs = std::sqrt(b->K / b->rho0);
    const double dt0 = p->dt_sub_override > 0 ? p->dt_sub_override : 0.6 * b->h / cs;
    const int use_tol = p->ke_tol >= 0 ? 1 : 0;
    MTS_TRY(launch_reset_ctrl(b, dt0, p->dt_sub_override, p->ramp_value, p->max_substeps,
                              p->ke_tol * p->ke_ref, p->ke_mode, use_tol));
    MTS_TRY(launch_slow_begin(b));
    *launches = 2;
    if (p->dt_slow > 0) {
        if (c_tape)   // concentration before the step, for the adjoint's D derivative
            MTS_CUDA(cudaMemcpyAsync(c_tape, b->c, b->n * sizeof(double), cudaMemcpyDeviceToDevice,
                                     b->ctx->stream));
        MTS_TRY(launch_diffusion(b, p->dt_slow));
        *launches += 2;
    }
    return MTS_OK;
}

// Report of a finished slow step from the host copy of the control block.
mts_status slow_step_report(mts_body *b, mts_step_report *rep, long long launches) {
    const Control &C = *b->h_ctrl;
    rep->substeps = C.nsub;
    rep->converged = C.converged;
    rep->status = C.status;
    rep->ke_final = C.ke;
    rep->max_v = C.vmax;
    rep->max_a = C.amax;
    rep->dt_last = C.dt_last;
    for (int k = 0; k < 3; ++k) rep->end_force[k] = k < b->dim ? C.end_force[k] : 0.0;
    double tip[3] = {0, 0, 0};
    if (b->tip_count > 0) {
        MTS_TRY(launch_tip(b, tip));
        launches += 2;
    }
    rep->kernel_launches = launches;
    for (int k = 0; k < 3; ++k) rep->tip_deflection[k] = tip[k];
    if (C.status != MTS_OK) {
        if (C.status == MTS_ERR_TIMEOUT)
            set_error("damping sweep: a wait for an earlier pair update ran out of time "
                      "(substep %lld)", (long long)C.nsub);
        else
            set_error("non-finite kinetic energy after substep %lld", (long long)C.nsub);
        return (mts_status)C.status;
    }
    return MTS_OK;
}

// One graph for a batch: a conditional WHILE node per body, no edges between
// them; each body graph is that body's substep, captured with the node's own
// conditional handle (the body's drift kernel ends only its own loop).
mts_status capture_batch_once(mts_batch *bt) {
    const int nb = (int)bt->bodies.size();
    if (bt->graph) {
        cudaGraphExecDestroy(bt->graph);
        bt->graph = nullptr;
    }
    cudaStream_t st = bt->ctx->stream;
    cudaGraph_t g = nullptr;
    MTS_CUDA(cudaGraphCreate(&g, 0));
    mts_status s = MTS_OK;
    for (int i = 0; i < nb && s == MTS_OK; ++i) {
        mts_body *b = bt->bodies[i];
        s = prepare_kernels(b);
        if (s != MTS_OK) break;
        cudaGraphConditionalHandle h;
        cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault);
        if (e != cudaSuccess) { s = cuda_fail(e, "cudaGraphConditionalHandleCreate"); break; }
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
        if (e != cudaSuccess) { s = cuda_fail(e, "cudaGraphAddNode(conditional)"); break; }
        e = cudaStreamBeginCaptureToGraph(st, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { s = cuda_fail(e, "cudaStreamBeginCaptureToGraph"); break; }
        const cudaGraphConditionalHandle own = b->cond;
        b->cond = h;
        b->use_cond = 1;
        b->pdl_now = b->ctx->pdl;
        long long ndamp = 0;
        s = launch_stress(b);
        if (s == MTS_OK) s = launch_force(b);
        if (s == MTS_OK) s = launch_damping(b, &ndamp);
        if (s == MTS_OK) s = launch_drift(b);
        b->use_cond = 0;
        b->pdl_now = false;
        b->cond = own;
        cudaGraph_t captured = nullptr;
        e = cudaStreamEndCapture(st, &captured);
        if (s == MTS_OK && e != cudaSuccess) s = cuda_fail(e, "cudaStreamEndCapture");
        b->launches_per_substep = 3 + ndamp;
    }
    if (s != MTS_OK) {
        cudaGraphDestroy(g);
        return s;
    }
    cudaError_t e = cudaGraphInstantiate(&bt->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate(batch)");
    bt->gens.resize(nb);
    for (int i = 0; i < nb; ++i) bt->gens[i] = bt->bodies[i]->graph_gen;
    return MTS_OK;
}

mts_status capture_batch(mts_batch *bt) {
    const int nb = (int)bt->bodies.size();
    bool fresh = bt->graph != nullptr && (int)bt->gens.size() == nb;
    for (int i = 0; fresh && i < nb; ++i) fresh = bt->gens[i] == bt->bodies[i]->graph_gen;
    if (fresh) return MTS_OK;
    return with_chain_fallback(bt->ctx, [&] { return capture_batch_once(bt); });
}

bool valid_field(int f) { return f >= MTS_F_U && f <= MTS_F_ACC; }

}  // namespace

extern "C" {

const char *mts_last_error(void) { return g_err; }
int mts_version(void) { return 100; }

mts_status mts_ctx_create(int device, void *cuda_stream, const mts_allocator *alloc, mts_ctx **out) {
    if (!out) {
        set_error("mts_ctx_create: out is NULL");
        return MTS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    int ndev = 0;
    MTS_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) {
        set_error("mts_ctx_create: device %d not present (%d devices)", device, ndev);
        return MTS_ERR_INVALID_ARG;
    }
    if (alloc && (!alloc->alloc || !alloc->release)) {
        set_error("mts_ctx_create: allocator needs both alloc and release");
        return MTS_ERR_INVALID_ARG;
    }
    MTS_CUDA(cudaSetDevice(device));
    mts_ctx *c = new (std::nothrow) mts_ctx();
    if (!c) return MTS_ERR_OOM;
    c->device = device;
    c->pdl = std::getenv("MTS_NO_CHAIN_LAUNCH") == nullptr;
    c->alloc.custom = alloc != nullptr;
    if (alloc) c->alloc.a = *alloc;
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
        c->own_stream = false;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return cuda_fail(e, "cudaStreamCreateWithFlags");
        }
        c->own_stream = true;
    }
    *out = c;
    return MTS_OK;
}

void mts_ctx_destroy(mts_ctx *ctx) {
    if (!ctx) return;
    if (ctx->own_stream) {
        cudaStreamSynchronize(ctx->stream);
        cudaStreamDestroy(ctx->stream);
    }
    delete ctx;
}

mts_status mts_body_create(mts_ctx *ctx, const mts_body_desc *desc, mts_body **out) {
    if (!ctx || !desc || !out || !desc->X) {
        set_error("mts_body_create: NULL argument");
        return MTS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if ((desc->dim != 2 && desc->dim != 3) || desc->n < 2 || desc->n >= (1LL << 31) ||
        !(desc->dx > 0) || !std::isfinite(desc->dx) || !(desc->h_over_dx > 0) ||
        !(desc->h_over_dx < 8) || (desc->precision != MTS_FP64 && desc->precision != MTS_MIXED) ||
        desc->damp_layout < MTS_DAMP_AUTO || desc->damp_layout > MTS_DAMP_WIDE) {
        set_error("mts_body_create: invalid descriptor (dim %d, n %lld, dx %g, h/dx %g, precision %d, "
                  "damping layout %d)", desc->dim, (long long)desc->n, desc->dx, desc->h_over_dx,
                  desc->precision, desc->damp_layout);
        return MTS_ERR_INVALID_ARG;
    }
    {
        const int tmax = tile_max(desc->precision == MTS_FP64 ? 8 : 4);
        const int T = desc->tile;
        if (T != 0 && (T < 64 || T > tmax || (T & (T - 1)) != 0)) {
            set_error("mts_body_create: tile %d (0, or a power of two in [64, %d])", T, tmax);
            return MTS_ERR_INVALID_ARG;
        }
    }
    // per-axis spacing (anisotropic kernel): all zero = isotropic
    double dxk[3] = {desc->dx, desc->dx, desc->dx};
    bool any_axis = false;
    for (int k = 0; k < desc->dim; ++k) any_axis |= desc->dx_axis[k] != 0.0;
    if (any_axis)
        for (int k = 0; k < desc->dim; ++k) {
            if (!(desc->dx_axis[k] > 0) || !std::isfinite(desc->dx_axis[k])) {
                set_error("mts_body_create: dx_axis[%d] = %g", k, desc->dx_axis[k]);
                return MTS_ERR_INVALID_ARG;
            }
            dxk[k] = desc->dx_axis[k];
        }
    double dref = dxk[0];
    for (int k = 1; k < desc->dim; ++k) dref = std::min(dref, dxk[k]);
    MTS_CUDA(cudaSetDevice(ctx->device));
    mts_body *b = new (std::nothrow) mts_body();
    if (!b) return MTS_ERR_OOM;
    b->ctx = ctx;
    b->dim = desc->dim;
    b->precision = desc->precision;
    b->n = desc->n;
    b->dx = dref;
    b->h = desc->h_over_dx * dref;
    const double w = 2.0 * b->h;
    b->cut2 = w * w;
    b->V = 1.0;
    b->detS = 1.0;
    for (int k = 0; k < 3; ++k) {
        b->sk[k] = k < b->dim ? dref / dxk[k] : 1.0;
        if (k < b->dim) {
            b->V *= dxk[k];
            b->detS *= b->sk[k];
            b->aniso |= dxk[k] != dref;
        }
    }
    long long need = (long long)std::floor(w / b->dx) + 1;
    b->blk_shift = 0;
    while ((1LL << b->blk_shift) < need) ++b->blk_shift;
    b->damp_req = desc->damp_layout;
    b->tile_req = desc->tile;
    b->damp_warps_req = 0;
    b->rsize = b->precision == MTS_FP64 ? 8 : 4;
    b->graph_dirty = true;
    ++b->graph_gen;
    const long long n = b->n;
    const int pad = b->dim == 2 ? 2 : 4;
    const int ms = b->dim == 2 ? 4 : 12;
    const size_t R = b->rsize;
    mts_status s = MTS_OK;
    auto A = [&](void **p, size_t bytes) {
        if (s == MTS_OK) s = dalloc_into(ctx, p, bytes + 16);
    };
    A((void **)&b->perm, n * 8);
    A((void **)&b->rank, n * 8);
    A((void **)&b->X64, n * pad * 8);
    A(&b->X, n * pad * R);
    A(&b->B0, n * ms * R);
    A((void **)&b->u, n * pad * 8);
    if (R == 4) A(&b->uf, n * pad * R);
    A(&b->v, n * pad * R);
    A(&b->acc, n * pad * R);
    A(&b->PB, n * ms * R);
    A(&b->cp, n * 8 * R);
    A(&b->c, n * R);
    A(&b->c_tmp, n * R);
    A(&b->c_held, n * R);
    A((void **)&b->u_unit, n * pad * 8);
    A((void **)&b->flags, n);
    A((void **)&b->ctrl, sizeof(Control));
    const long long grid = (n + kBlock - 1) / kBlock;
    // one force partial per tile: tiles hold at least 64 particles
    A((void **)&b->part_force, ((n + 63) / 64) * 4 * 8);
    A((void **)&b->part_drift, grid * 2 * 8);
    A((void **)&b->scratch, (size_t)n * 18 * 8);
    A((void **)&b->d_first, 8);
    if (s == MTS_OK && cudaMallocHost((void **)&b->h_ctrl, sizeof(Control)) != cudaSuccess) {
        set_error("pinned allocation failed");
        s = MTS_ERR_OOM;
    }
    if (s != MTS_OK) {
        body_free(b);
        return s;
    }
    cudaStream_t st = ctx->stream;
    cudaMemsetAsync(b->ctrl, 0, sizeof(Control), st);
    k_init_state<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(b->u, b->uf, b->v, b->acc, b->cp, b->c,
                                                               b->c_held, b->flags, b->u_unit, n, pad,
                                                               (int)R);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        body_free(b);
        return cuda_fail(e, "k_init_state");
    }
    if (b->aniso) {
        // the whole set-up runs on positions scaled to the isotropic kernel
        std::vector<double> Xs((size_t)n * b->dim);
        for (long long i = 0; i < n; ++i)
            for (int k = 0; k < b->dim; ++k) Xs[i * b->dim + k] = desc->X[i * b->dim + k] * b->sk[k];
        s = build_body(b, Xs.data());
    } else {
        s = build_body(b, desc->X);
    }
    if (s != MTS_OK) {
        cudaStreamSynchronize(st);
        body_free(b);
        return s;
    }
    b->h_flags.assign(n, 0);
    *out = b;
    return MTS_OK;
}

void mts_body_destroy(mts_body *body) {
    if (!body) return;
    cudaStreamSynchronize(body->ctx->stream);
    body_free(body);
}

mts_status mts_body_damping_layout(const mts_body *b, int32_t shift[3], int32_t *level_cap) {
    if (!b || !shift || !level_cap) {
        set_error("mts_body_damping_layout: NULL argument");
        return MTS_ERR_INVALID_ARG;
    }
    for (int k = 0; k < 3; ++k) shift[k] = b->ax_shift[k] >= kWholeAxis ? MTS_WHOLE_AXIS : b->ax_shift[k];
    *level_cap = b->level_cap;
    return MTS_OK;
}

mts_status mts_body_set_shapes(mts_body *b, int32_t tile, int32_t damp_warps) {
    if (!b) {
        set_error("mts_body_set_shapes: NULL body");
        return MTS_ERR_INVALID_ARG;
    }
    const int tmax = tile_max((int)b->rsize);
    if ((tile != 0 && (tile < 64 || tile > tmax || (tile & (tile - 1)) != 0)) ||
        (damp_warps != 0 && damp_warps != 1 && damp_warps != 2 && damp_warps != 4)) {
        set_error("mts_body_set_shapes: tile %d (0, or a power of two in [64, %d]), damp_warps %d "
                  "(0, 1, 2 or 4)", tile, tmax, damp_warps);
        return MTS_ERR_INVALID_ARG;
    }
    MTS_CUDA(cudaSetDevice(b->ctx->device));
    if (tile != 0 && tile != b->T) {
        MTS_TRY(retile(b, tile));
        if (b->adj_cap > 0) MTS_TRY(adjoint_prepare(b));
    }
    b->damp_warps_req = damp_warps;
    b->graph_dirty = true;
    ++b->graph_gen;
    return MTS_OK;
}

mts_status mts_body_shapes(const mts_body *b, int32_t *tile, int32_t *damp_warps) {
    if (!b || !tile || !damp_warps) {
        set_error("mts_body_shapes: NULL argument");
        return MTS_ERR_INVALID_ARG;
    }
    *tile = b->T;
    *damp_warps = damp_warps_of(b);
    return MTS_OK;
}

mts_status mts_body_autotune(mts_body *b, int32_t substeps, double ramp, int32_t *tile,
                             int32_t *damp_warps, double *best_ms) {
    if (!b || substeps < 1 || substeps > 1000 || !std::isfinite(ramp)) {
        set_error("mts_body_autotune: NULL body, substeps %d (1..1000) or ramp %g", substeps, ramp);
        return MTS_ERR_INVALID_ARG;
    }
    if (!b->has_material) {
        set_error("mts_body_autotune: no material set");
        return MTS_ERR_STATE;
    }
    MTS_CUDA(cudaSetDevice(b->ctx->device));
    size_t bytes = 0;
    MTS_TRY(mts_save_state(b, nullptr, &bytes));
    std::vector<unsigned char> saved(bytes);
    MTS_TRY(mts_save_state(b, saved.data(), &bytes));
    const int tiles32[2] = {256, 512}, tiles64[2] = {64, 128}, warps[3] = {1, 2, 4};
    const int *tiles = b->rsize == 4 ? tiles32 : tiles64;
    mts_step_params p{};
    p.ramp_value = ramp;
    p.ke_tol = -1.0;
    p.ke_ref = 1.0;
    p.max_substeps = substeps;
    mts_step_report rep{};
    cudaEvent_t e0, e1;
    MTS_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(cudaGetLastError(), "cudaEventCreate");
    }
    mts_status s = MTS_OK;
    int best_t = b->T, best_w = damp_warps_of(b);
    double best = 1e300;
    for (int ti = 0; ti < 2 && s == MTS_OK; ++ti)
        for (int wi = 0; wi < 3 && s == MTS_OK; ++wi) {
            s = mts_body_set_shapes(b, tiles[ti], warps[wi]);
            if (s == MTS_OK && damp_warps_of(b) != warps[wi]) continue;   // does not fit
            for (int rep_i = 0; rep_i < 2 && s == MTS_OK; ++rep_i) {   // capture, then time
                s = mts_load_state(b, saved.data(), bytes);
                if (s != MTS_OK) break;
                if (rep_i == 1 && cudaEventRecord(e0, b->ctx->stream) != cudaSuccess) {
                    s = cuda_fail(cudaGetLastError(), "cudaEventRecord");
                    break;
                }
                s = mts_advance_slow_step(b, &p, &rep);
                if (s == MTS_OK && rep_i == 1) {
                    cudaError_t e = cudaEventRecord(e1, b->ctx->stream);
                    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                    float ms = 0.0f;
                    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                    if (e != cudaSuccess) {
                        s = cuda_fail(e, "autotune timing");
                    } else if (ms < best) {
                        best = ms;
                        best_t = tiles[ti];
                        best_w = warps[wi];
                    }
                }
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s == MTS_OK) s = mts_body_set_shapes(b, best_t, best_w);
    if (s == MTS_OK) s = mts_load_state(b, saved.data(), bytes);
    if (s != MTS_OK) return s;
    if (tile) *tile = best_t;
    if (damp_warps) *damp_warps = best_w;
    if (best_ms) *best_ms = best;
    return MTS_OK;
}

mts_status mts_body_permutation(const mts_body *b, int64_t *perm) {
    if (!b || !perm) {
        set_error("mts_body_permutation: NULL argument");
        return MTS_ERR_INVALID_ARG;
    }
    MTS_CUDA(cudaMemcpyAsync(perm, b->perm, b->n * 8, cudaMemcpyDeviceToHost, b->ctx->stream));
    MTS_CUDA(cudaStreamSynchronize(b->ctx->stream));
    return MTS_OK;
}

mts_status mts_body_neighbors(const mts_body *b, int64_t *nnz, int64_t *offsets, int32_t *idx) {
    if (!b || !nnz) {
        set_error("mts_body_neighbors: NULL argument");
        return MTS_ERR_INVALID_ARG;
    }
    *nnz = b->nnz;
    cudaStream_t st = b->ctx->stream;
    if (offsets) MTS_CUDA(cudaMemcpyAsync(offsets, b->nb_off, (b->n + 1) * 8, cudaMemcpyDeviceToHost, st));
    if (idx) MTS_CUDA(cudaMemcpyAsync(idx, b->nb_idx, b->nnz * 4, cudaMemcpyDeviceToHost, st));
    MTS_CUDA(cudaStreamSynchronize(st));
    return MTS_OK;
}

mts_status mts_body_colouring(const mts_body *b, int64_t *npairs, int32_t *pa, int32_t *pb,
                              int32_t *colour, int64_t *block_key, int32_t *sub) {
    if (!b || !npairs) {
        set_error("mts_body_colouring: NULL argument");
        return MTS_ERR_INVALID_ARG;
    }
    *npairs = b->npairs;
    cudaStream_t st = b->ctx->stream;
    const size_t m = (size_t)b->npairs;
    if (pa) MTS_CUDA(cudaMemcpyAsync(pa, b->pair_a, m * 4, cudaMemcpyDeviceToHost, st));
    if (pb) MTS_CUDA(cudaMemcpyAsync(pb, b->pair_b, m * 4, cudaMemcpyDeviceToHost, st));
    if (colour) MTS_CUDA(cudaMemcpyAsync(colour, b->pair_col, m * 4, cudaMemcpyDeviceToHost, st));
    if (block_key) MTS_CUDA(cudaMemcpyAsync(block_key, b->pair_key, m * 8, cudaMemcpyDeviceToHost, st));
    if (sub) MTS_CUDA(cudaMemcpyAsync(sub, b->pair_sub, m * 4, cudaMemcpyDeviceToHost, st));
    MTS_CUDA(cudaStreamSynchronize(st));
    return MTS_OK;
}

mts_status mts_set_material(mts_body *b, mts_material_model model, double rho0, double E, double nu,
                            double sigma0, double sigma_inf, double delta, double H) {
    if (!b || (model != MTS_ELASTIC_SVK && model != MTS_NEOHOOKE_J2) || !(rho0 > 0) || !(E > 0) ||
        !(nu > -1.0) || !(nu < 0.5) || !std::isfinite(rho0) || !std::isfinite(E)) {
        set_error("mts_set_material: invalid parameters");
        return MTS_ERR_INVALID_ARG;
    }
    if (model == MTS_NEOHOOKE_J2 && (!(sigma0 > 0) || !std::isfinite(sigma_inf) ||
                                     !(delta >= 0) || !std::isfinite(H))) {
        set_error("mts_set_material: invalid hardening parameters");
        return MTS_ERR_INVALID_ARG;
    }
    b->has_material = true;
    b->model = model;
    b->rho0 = rho0;
    b->E = E;
    b->nu = nu;
    b->mu = E / (2.0 * (1.0 + nu));
    b->K = E / (3.0 * (1.0 - 2.0 * nu));
    b->lambda = b->K - 2.0 * b->mu / 3.0;
    b->s0 = sigma0;
    b->sinf = sigma_inf;
    b->delta = delta;
    b->Hlin = H;
    b->graph_dirty = true;
    ++b->graph_gen;
    return MTS_OK;
}

mts_status mts_set_damping(mts_body *b, double eta) {
    if (!b || !(eta >= 0) || !std::isfinite(eta)) {
        set_error("mts_set_damping: eta must be finite and >= 0");
        return MTS_ERR_INVALID_ARG;
    }
    b->eta = eta;
    b->graph_dirty = true;
    ++b->graph_gen;
    return MTS_OK;
}

mts_status mts_set_diffusion(mts_body *b, double D, double beta, double c0) {
    if (!b || !(D >= 0) || !std::isfinite(D) || !std::isfinite(beta) || !std::isfinite(c0)) {
        set_error("mts_set_diffusion: invalid parameters");
        return MTS_ERR_INVALID_ARG;
    }
    b->has_diff = true;
    b->D = D;
    b->beta = beta;
    b->c0 = c0;
    b->graph_dirty = true;
    ++b->graph_gen;
    k_set_c<<<(unsigned)((b->n + 255) / 256), 256, 0, b->ctx->stream>>>(b->c, b->c_held, b->flags, b->n,
                                                                        c0, (int)b->rsize, 0);
    MTS_CUDA(cudaGetLastError());
    MTS_CUDA(cudaStreamSynchronize(b->ctx->stream));
    return MTS_OK;
}

mts_status mts_set_bc_displacement(mts_body *b, int64_t count, const int64_t *ids, uint32_t mask,
                                   const double *u_unit, int32_t report_force) {
    if (!b || count < 0 || (count > 0 && !ids)) {
        set_error("mts_set_bc_displacement: invalid arguments");
        return MTS_ERR_INVALID_ARG;
    }
    std::vector<long long> rank;
    MTS_TRY(get_rank_host(b, rank));
    const int pad = b->dim == 2 ? 2 : 4;
    std::vector<double> uu((size_t)b->n * pad);
    MTS_CUDA(cudaMemcpyAsync(uu.data(), b->u_unit, uu.size() * 8, cudaMemcpyDeviceToHost, b->ctx->stream));
    MTS_CUDA(cudaStreamSynchronize(b->ctx->stream));
    const uint32_t m = mask & ((1u << b->dim) - 1);
    for (int64_t t = 0; t < count; ++t) {
        if (ids[t] < 0 || ids[t] >= b->n) {
            set_error("mts_set_bc_displacement: id %lld out of range", (long long)ids[t]);
            return MTS_ERR_INVALID_ARG;
        }
        const long long s = rank[ids[t]];
        b->h_flags[s] |= (uint8_t)m;
        for (int k = 0; k < b->dim; ++k)
            if (m & (1u << k)) {
                double val = u_unit ? u_unit[t * b->dim + k] : 0.0;
                if (!std::isfinite(val)) {
                    set_error("mts_set_bc_displacement: non-finite u_unit");
                    return MTS_ERR_INVALID_ARG;
                }
                uu[s * pad + k] = val;
            }
        if (report_force) b->h_flags[s] |= kForceBit;
    }
    b->graph_dirty = true;
    ++b->graph_gen;
    return upload_bc(b, uu);
}

mts_status mts_release_bc_concentration(mts_body *b, int64_t count, const int64_t *ids) {
    if (!b || count < 0 || (count > 0 && !ids)) {
        set_error("mts_release_bc_concentration: invalid arguments");
        return MTS_ERR_INVALID_ARG;
    }
    std::vector<long long> rank;
    MTS_TRY(get_rank_host(b, rank));
    for (int64_t t = 0; t < count; ++t) {
        if (ids[t] < 0 || ids[t] >= b->n) {
            set_error("mts_release_bc_concentration: id %lld out of range", (long long)ids[t]);
            return MTS_ERR_INVALID_ARG;
        }
        b->h_flags[rank[ids[t]]] &= (uint8_t)~kCHeldBit;
    }
    MTS_TRY(upload_bc(b, {}));
    return MTS_OK;
}

mts_status mts_set_bc_concentration(mts_body *b, int64_t count, const int64_t *ids, double value) {
    if (!b || count < 0 || (count > 0 && !ids) || !std::isfinite(value)) {
        set_error("mts_set_bc_concentration: invalid arguments");
        return MTS_ERR_INVALID_ARG;
    }
    std::vector<long long> rank;
    MTS_TRY(get_rank_host(b, rank));
    std::vector<char> held((size_t)b->n * b->rsize);
    MTS_CUDA(cudaMemcpyAsync(held.data(), b->c_held, held.size(), cudaMemcpyDeviceToHost, b->ctx->stream));
    MTS_CUDA(cudaStreamSynchronize(b->ctx->stream));
    for (int64_t t = 0; t < count; ++t) {
        if (ids[t] < 0 || ids[t] >= b->n) {
            set_error("mts_set_bc_concentration: id %lld out of range", (long long)ids[t]);
            return MTS_ERR_INVALID_ARG;
        }
        const long long s = rank[ids[t]];
        b->h_flags[s] |= kCHeldBit;
        if (b->rsize == 4)
            reinterpret_cast<float *>(held.data())[s] = (float)value;
        else
            reinterpret_cast<double *>(held.data())[s] = value;
    }
    cudaStream_t st = b->ctx->stream;
    MTS_CUDA(cudaMemcpyAsync(b->c_held, held.data(), held.size(), cudaMemcpyHostToDevice, st));
    MTS_TRY(upload_bc(b, {}));
    k_set_c<<<(unsigned)((b->n + 255) / 256), 256, 0, st>>>(b->c, b->c_held, b->flags, b->n, 0.0,
                                                            (int)b->rsize, 1);
    MTS_CUDA(cudaGetLastError());
    MTS_CUDA(cudaStreamSynchronize(st));
    return MTS_OK;
}

mts_status mts_set_tip(mts_body *b, int64_t count, const int64_t *ids) {
    if (!b || count < 0 || (count > 0 && !ids)) {
        set_error("mts_set_tip: invalid arguments");
        return MTS_ERR_INVALID_ARG;
    }
    std::vector<long long> rank;
    MTS_TRY(get_rank_host(b, rank));
    for (auto &f : b->h_flags) f &= (uint8_t)~kTipBit;
    for (int64_t t = 0; t < count; ++t) {
        if (ids[t] < 0 || ids[t] >= b->n) {
            set_error("mts_set_tip: id %lld out of range", (long long)ids[t]);
            return MTS_ERR_INVALID_ARG;
        }
        b->h_flags[rank[ids[t]]] |= kTipBit;
    }
    b->tip_count = (int)count;
    return upload_bc(b, {});
}

mts_status mts_diffusion_dt(mts_body *b, double *dt_paper, double *dt_stable) {
    if (!b || !dt_paper || !dt_stable) {
        set_error("mts_diffusion_dt: NULL argument");
        return MTS_ERR_INVALID_ARG;
    }
    if (!b->has_diff) {
        set_error("mts_diffusion_dt: no diffusion set");
        return MTS_ERR_STATE;
    }
    *dt_paper = b->D > 0 ? 0.5 * b->h * b->h / b->D : INFINITY;
    if (b->diff_mode == 1) {
        double lam = 0;
        MTS_TRY(diffusion_bound_two_stage(b, &lam));
        *dt_stable = lam > 0 ? 1.8 / lam : INFINITY;
        return MTS_OK;
    }
    if (!b->diff_amax_ok || b->diff_amax_D != b->D) {
        MTS_TRY(diffusion_bound(b, &b->diff_amax));
        b->diff_amax_D = b->D;
        b->diff_amax_ok = true;
    }
    const double amax = b->diff_amax;
    *dt_stable = amax > 0 ? 0.9 / amax : INFINITY;
    return MTS_OK;
}

mts_status mts_set_diffusion_mode(mts_body *b, int32_t mode) {
    if (!b || (mode != 0 && mode != 1)) {
        set_error("mts_set_diffusion_mode: mode must be 0 or 1");
        return MTS_ERR_INVALID_ARG;
    }
    if (mode == 1 && !b->qflux) {
        const size_t pad = b->dim == 2 ? 2 : 4;
        MTS_TRY(dalloc_into(b->ctx, &b->qflux, (size_t)b->n * pad * b->rsize + 16));
        MTS_CUDA(cudaMemsetAsync(b->qflux, 0, (size_t)b->n * pad * b->rsize, b->ctx->stream));
    }
    b->diff_mode = mode;
    return MTS_OK;
}

mts_status mts_advance_slow_step(mts_body *b, const mts_step_params *p, mts_step_report *rep) {
    if (!b || !p || !rep) {
        set_error("mts_advance_slow_step: NULL argument");
        return MTS_ERR_INVALID_ARG;
    }
    memset(rep, 0, sizeof(*rep));
    long long launches = 0;
    MTS_TRY(slow_step_begin(b, p, &launches));
    cudaStream_t st = b->ctx->stream;
    long long done_before = 0;
    double prof_ms = 0.0;
    long long prof_n = 0;
    if (b->prof_stage == 0 && p->check_every <= 0) {
        // device-side loop: one graph launch runs substeps until the stop flag
        MTS_TRY(capture_loop(b));
        MTS_CUDA(cudaGraphLaunch(b->graph, st));
        MTS_CUDA(cudaMemcpyAsync(b->h_ctrl, b->ctrl, sizeof(Control), cudaMemcpyDeviceToHost, st));
        MTS_CUDA(cudaStreamSynchronize(st));
        launches += b->h_ctrl->nsub * b->launches_per_substep;
    }
    const int chunk = std::max(1, std::min(p->check_every > 0 ? p->check_every : 32, 4096));
    if (b->prof_stage > 0 || p->check_every > 0) MTS_TRY(capture_chunk(b, chunk));
    for (; b->prof_stage > 0 || p->check_every > 0;) {
        MTS_CUDA(cudaGraphLaunch(b->graph, st));
        launches += chunk * b->launches_per_substep;
        MTS_CUDA(cudaMemcpyAsync(b->h_ctrl, b->ctrl, sizeof(Control), cudaMemcpyDeviceToHost, st));
        MTS_CUDA(cudaStreamSynchronize(st));
        if (b->graph_prof_stage > 0) {
            const long long ran = std::min<long long>(b->h_ctrl->nsub - done_before, chunk);
            for (long long k = 0; k < ran; ++k) {
                float ms = 0.f;
                MTS_CUDA(cudaEventElapsedTime(&ms, b->prof_ev[2 * k], b->prof_ev[2 * k + 1]));
                prof_ms += ms;
            }
            prof_n += ran;
        }
        done_before = b->h_ctrl->nsub;
        if (b->h_ctrl->done) break;
    }
    rep->prof_ms = prof_ms;
    rep->prof_count = prof_n;
    return slow_step_report(b, rep, launches);
}

mts_status mts_batch_create(mts_ctx *ctx, int32_t count, mts_body *const *bodies, mts_batch **out) {
    if (!ctx || !bodies || !out || count < 1) {
        set_error("mts_batch_create: NULL argument or count < 1");
        return MTS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    std::vector<mts_body *> v(bodies, bodies + count);
    for (int i = 0; i < count; ++i) {
        if (!v[i] || v[i]->ctx != ctx) {
            set_error("mts_batch_create: body %d is NULL or belongs to another context", i);
            return MTS_ERR_INVALID_ARG;
        }
        for (int j = 0; j < i; ++j)
            if (v[j] == v[i]) {
                set_error("mts_batch_create: body %d appears twice (%d)", i, j);
                return MTS_ERR_INVALID_ARG;
            }
    }
    mts_batch *bt = new (std::nothrow) mts_batch();
    if (!bt) return MTS_ERR_OOM;
    bt->ctx = ctx;
    bt->bodies = std::move(v);
    bt->graph = nullptr;
    *out = bt;
    return MTS_OK;
}

mts_status mts_batch_autotune(mts_batch *bt, int32_t substeps, double ramp) {
    if (!bt || substeps < 1 || substeps > 1000 || !std::isfinite(ramp)) {
        set_error("mts_batch_autotune: NULL batch, substeps %d (1..1000) or ramp %g", substeps, ramp);
        return MTS_ERR_INVALID_ARG;
    }
    const int nb = (int)bt->bodies.size();
    for (mts_body *b : bt->bodies)
        if (!b->has_material) {
            set_error("mts_batch_autotune: a body has no material");
            return MTS_ERR_STATE;
        }
    MTS_CUDA(cudaSetDevice(bt->ctx->device));
    // every body's state, restored before each trial and at the end
    std::vector<std::vector<unsigned char>> saved(nb);
    for (int i = 0; i < nb; ++i) {
        size_t bytes = 0;
        MTS_TRY(mts_save_state(bt->bodies[i], nullptr, &bytes));
        saved[i].resize(bytes);
        MTS_TRY(mts_save_state(bt->bodies[i], saved[i].data(), &bytes));
    }
    auto restore = [&]() -> mts_status {
        for (int i = 0; i < nb; ++i)
            MTS_TRY(mts_load_state(bt->bodies[i], saved[i].data(), saved[i].size()));
        return MTS_OK;
    };
    std::vector<mts_step_params> p(nb);
    for (auto &q : p) {
        q = mts_step_params{};
        q.ramp_value = ramp;
        q.ke_tol = -1.0;
        q.ke_ref = 1.0;
        q.max_substeps = substeps;
    }
    std::vector<mts_step_report> rep(nb);
    // one shape for the whole batch at a time (the bodies run concurrently,
    // so the batch is timed as a whole): tile index into each body's tile set
    const int tiles32[2] = {256, 512}, tiles64[2] = {64, 128}, warps[3] = {1, 2, 4};
    cudaEvent_t e0, e1;
    MTS_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(cudaGetLastError(), "cudaEventCreate");
    }
    mts_status s = MTS_OK;
    int best_ti = 1, best_w = 4;
    double best = 1e300;
    for (int ti = 0; ti < 2 && s == MTS_OK; ++ti)
        for (int wi = 0; wi < 3 && s == MTS_OK; ++wi) {
            for (mts_body *b : bt->bodies) {
                s = mts_body_set_shapes(b, b->rsize == 4 ? tiles32[ti] : tiles64[ti], warps[wi]);
                if (s != MTS_OK) break;
            }
            for (int r = 0; r < 2 && s == MTS_OK; ++r) {   // capture, then time
                s = restore();
                if (s != MTS_OK) break;
                if (r == 1 && cudaEventRecord(e0, bt->ctx->stream) != cudaSuccess) {
                    s = cuda_fail(cudaGetLastError(), "cudaEventRecord");
                    break;
                }
                s = mts_batch_advance(bt, p.data(), rep.data());
                if (s == MTS_OK && r == 1) {
                    cudaError_t e = cudaEventRecord(e1, bt->ctx->stream);
                    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                    float ms = 0.0f;
                    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                    if (e != cudaSuccess) {
                        s = cuda_fail(e, "batch autotune timing");
                    } else if (ms < best) {
                        best = ms;
                        best_ti = ti;
                        best_w = warps[wi];
                    }
                }
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (mts_body *b : bt->bodies) {
        if (s != MTS_OK) break;
        s = mts_body_set_shapes(b, b->rsize == 4 ? tiles32[best_ti] : tiles64[best_ti], best_w);
    }
    if (s == MTS_OK) s = restore();
    return s;
}

void mts_batch_destroy(mts_batch *bt) {
    if (!bt) return;
    if (bt->graph) {
        cudaStreamSynchronize(bt->ctx->stream);
        cudaGraphExecDestroy(bt->graph);
    }
    delete bt;
}

mts_status mts_batch_advance(mts_batch *bt, const mts_step_params *p, mts_step_report *rep) {
    if (!bt || !p || !rep) {
        set_error("mts_batch_advance: NULL argument");
        return MTS_ERR_INVALID_ARG;
    }
    const int nb = (int)bt->bodies.size();
    for (int i = 0; i < nb; ++i) memset(rep + i, 0, sizeof(*rep));
    std::vector<long long> launches(nb, 0);
    for (int i = 0; i < nb; ++i) {
        const mts_status s = slow_step_begin(bt->bodies[i], p + i, &launches[i]);
        if (s != MTS_OK) {
            char msg[512];
            snprintf(msg, sizeof msg, "batch body %d: %s", i, mts_last_error());
            set_error("%s", msg);
            return s;
        }
    }
    MTS_TRY(capture_batch(bt));
    cudaStream_t st = bt->ctx->stream;
    MTS_CUDA(cudaGraphLaunch(bt->graph, st));
    for (mts_body *b : bt->bodies)
        MTS_CUDA(cudaMemcpyAsync(b->h_ctrl, b->ctrl, sizeof(Control), cudaMemcpyDeviceToHost, st));
    MTS_CUDA(cudaStreamSynchronize(st));
    mts_status first = MTS_OK;
    for (int i = 0; i < nb; ++i) {
        mts_body *b = bt->bodies[i];
        const mts_status s =
            slow_step_report(b, rep + i, launches[i] + b->h_ctrl->nsub * b->launches_per_substep);
        if (s != MTS_OK && first == MTS_OK) {
            char msg[512];
            snprintf(msg, sizeof msg, "batch body %d: %s", i, mts_last_error());
            set_error("%s", msg);
            first = s;
        }
    }
    return first;
}

mts_status mts_set_profiling(mts_body *b, int32_t stage) {
    if (!b || stage < 0 || stage > 4) {
        set_error("mts_set_profiling: stage must be 0..4");
        return MTS_ERR_INVALID_ARG;
    }
    b->prof_stage = stage;
    return MTS_OK;
}

mts_status mts_substep_partial(mts_body *b, double dt, double ramp, int32_t upto) {
    if (!b || !(dt > 0) || !std::isfinite(dt) || !std::isfinite(ramp) || upto < 1 || upto > 4) {
        set_error("mts_substep_partial: invalid arguments");
        return MTS_ERR_INVALID_ARG;
    }
    if (!b->has_material) {
        set_error("mts_substep_partial: no material set");
        return MTS_ERR_STATE;
    }
    MTS_CUDA(cudaSetDevice(b->ctx->device));
    MTS_TRY(prepare_kernels(b));
    MTS_TRY(launch_reset_ctrl(b, dt, dt, ramp, 1LL << 62, 0.0, 0, 0));
    MTS_TRY(launch_stress(b));
    if (upto >= 2) MTS_TRY(launch_force(b));
    if (upto >= 3) MTS_TRY(launch_damping(b));
    if (upto >= 4) MTS_TRY(launch_drift(b));
    MTS_CUDA(cudaStreamSynchronize(b->ctx->stream));
    return MTS_OK;
}

}  // extern "C"

namespace {
// smallest index of a non-finite value of x[0, n) (a double is not finite
// exactly when its eleven exponent bits are all ones); *first starts at ~0
// self-check of the integer-pipe conversions (f2d_bits, d2f_bits) against
// the hardware's, on counter-hashed bit patterns steered into the edge cases:
// binary32 subnormals, zeros, infinities and NaNs; binary64 values whose
// binary32 result is normal, subnormal, zero or overflows, exact rounding
// ties, binary64 subnormals and non-finite values
__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {   // splitmix64 finaliser
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

__global__ void k_selftest_conv(long long n, unsigned long long seed, unsigned long long *mis) {
    unsigned long long bad_f2d = 0, bad_d2f = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long x = mix64(seed + (unsigned long long)i), y = mix64(x);
        uint32_t fb = (uint32_t)x;
        switch ((x >> 32) & 7u) {
            case 0: fb &= 0x807fffffu; break;                 // subnormal (or zero)
            case 1: fb |= 0x7f800000u; break;                 // infinity or NaN
            case 2: fb &= 0x80000000u; break;                 // signed zero
            default: break;
        }
        const float f = __uint_as_float(fb);
        const double h1 = (double)f, h2 = f2d_bits(f);
        if (!(isnan(h1) && isnan(h2)) && __double_as_longlong(h1) != __double_as_longlong(h2)) ++bad_f2d;
        unsigned long long db = y;
        const unsigned c = (unsigned)((x >> 40) & 7u);
        if (c <= 4) {   // exponent field around the binary32 range (normal, subnormal, overflow)
            const unsigned long long E = 850ull + (x >> 48) % 320ull;
            db = (db & ~(0x7ffull << 52)) | (E << 52);
            if (c == 4) db = (db & ~0x1fffffffull) | 0x10000000ull;   // exact tie at the last bit
        } else if (c == 5) {
            db &= ~(0x7ffull << 52);                               // binary64 subnormal
        } else if (c == 6) {
            db |= 0x7ffull << 52;                                  // infinity or NaN
        }
        const double d = __longlong_as_double((long long)db);
        const float g1 = (float)d, g2 = d2f_bits(d);
        if (!(isnan(g1) && isnan(g2)) && __float_as_uint(g1) != __float_as_uint(g2)) ++bad_d2f;
    }
    if (bad_f2d) atomicAdd(mis, bad_f2d);
    if (bad_d2f) atomicAdd(mis + 1, bad_d2f);
}

__global__ void k_first_nonfinite(const double *x, long long n, unsigned long long *first) {
    constexpr unsigned long long kExp = 0x7ff0000000000000ull;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long v = (unsigned long long)__double_as_longlong(x[i]);
        if ((v & kExp) == kExp) atomicMin(first, (unsigned long long)i);
    }
}
}  // namespace

extern "C" {

mts_status mts_selftest_conversions(mts_ctx *ctx, int64_t n, uint64_t seed, int64_t *mismatches) {
    if (!ctx || !mismatches || n < 0) {
        set_error("mts_selftest_conversions: invalid arguments");
        return MTS_ERR_INVALID_ARG;
    }
    MTS_CUDA(cudaSetDevice(ctx->device));
    unsigned long long *d = (unsigned long long *)dalloc(ctx, 2 * sizeof(unsigned long long));
    if (!d) {
        set_error("mts_selftest_conversions: device allocation failed");
        return MTS_ERR_OOM;
    }
    unsigned long long h[2] = {0, 0};
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof h, ctx->stream);
    if (e == cudaSuccess && n > 0) {
        k_selftest_conv<<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, ctx->stream>>>(n, seed, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, d);
    MTS_CUDA(e);
    mismatches[0] = (int64_t)h[0];
    mismatches[1] = (int64_t)h[1];
    return MTS_OK;
}

mts_status mts_read_field(mts_body *b, int32_t field, double *out, int64_t len) {
    if (!b || !out || !valid_field(field)) {
        set_error("mts_read_field: invalid arguments");
        return MTS_ERR_INVALID_ARG;
    }
    const int w = field_width(b, field);
    if (len != b->n * w) {
        set_error("mts_read_field: len %lld, expected %lld", (long long)len, (long long)(b->n * w));
        return MTS_ERR_INVALID_ARG;
    }
    MTS_CUDA(cudaSetDevice(b->ctx->device));
    MTS_TRY(field_to_scratch(b, field));
    MTS_CUDA(cudaMemcpyAsync(out, b->scratch, len * 8, cudaMemcpyDeviceToHost, b->ctx->stream));
    MTS_CUDA(cudaStreamSynchronize(b->ctx->stream));
    return MTS_OK;
}

mts_status mts_write_field(mts_body *b, int32_t field, const double *in, int64_t len) {
    if (!b || !in || !(field == MTS_F_U || field == MTS_F_V || field == MTS_F_C ||
                       field == MTS_F_ALPHA || field == MTS_F_CPINV)) {
        set_error("mts_write_field: invalid arguments (writable: U, V, C, ALPHA, CPINV)");
        return MTS_ERR_INVALID_ARG;
    }
    const int w = field_width(b, field);
    if (len != b->n * w) {
        set_error("mts_write_field: len %lld, expected %lld", (long long)len, (long long)(b->n * w));
        return MTS_ERR_INVALID_ARG;
    }
    // the values are checked on the device once in the scratch buffer; only
    // a clean field is moved from there into the body's state
    MTS_CUDA(cudaSetDevice(b->ctx->device));
    cudaStream_t st = b->ctx->stream;
    MTS_CUDA(cudaMemcpyAsync(b->scratch, in, len * 8, cudaMemcpyHostToDevice, st));
    MTS_CUDA(cudaMemsetAsync(b->d_first, 0xff, sizeof(unsigned long long), st));
    const long long blocks = std::min<long long>((len + 255) / 256, 4096);
    k_first_nonfinite<<<(unsigned)std::max<long long>(blocks, 1), 256, 0, st>>>(b->scratch, len, b->d_first);
    MTS_CUDA(cudaGetLastError());
    unsigned long long first = 0;
    MTS_CUDA(cudaMemcpyAsync(&first, b->d_first, sizeof first, cudaMemcpyDeviceToHost, st));
    MTS_CUDA(cudaStreamSynchronize(st));
    if (first != ~0ull) {
        set_error("mts_write_field: non-finite value at %lld", (long long)first);
        return MTS_ERR_NONFINITE;
    }
    MTS_TRY(scratch_to_field(b, field));
    MTS_CUDA(cudaStreamSynchronize(st));
    return MTS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- state
namespace {
constexpr uint32_t kStateMagic = 0x3153544du;   // "MTS1"

struct StateHeader {
    uint32_t magic;
    int32_t dim, precision, narrays;
    int64_t n;
};

// the state arrays of a body: device pointer and byte count
int state_arrays(const mts_body *b, void **ptr, size_t *len) {
    const size_t n = (size_t)b->n, R = b->rsize, pad = b->dim == 2 ? 2 : 4;
    int k = 0;
    ptr[k] = b->u;   len[k++] = n * pad * 8;
    if (R == 4) { ptr[k] = b->uf; len[k++] = n * pad * R; }
    ptr[k] = b->v;   len[k++] = n * pad * R;
    ptr[k] = b->acc; len[k++] = n * pad * R;
    ptr[k] = b->cp;  len[k++] = n * 8 * R;
    ptr[k] = b->c;   len[k++] = n * R;
    return k;
}
}  // namespace

extern "C" {

mts_status mts_save_state(const mts_body *b, void *buf, size_t *bytes) {
    if (!b || !bytes) {
        set_error("mts_save_state: NULL argument");
        return MTS_ERR_INVALID_ARG;
    }
    void *ptr[8];
    size_t len[8];
    const int na = state_arrays(b, ptr, len);
    size_t need = sizeof(StateHeader);
    for (int k = 0; k < na; ++k) need += len[k];
    if (!buf) {
        *bytes = need;
        return MTS_OK;
    }
    if (*bytes < need) {
        set_error("mts_save_state: buffer of %zu bytes, %zu needed", *bytes, need);
        return MTS_ERR_INVALID_ARG;
    }
    MTS_CUDA(cudaSetDevice(b->ctx->device));
    StateHeader h{kStateMagic, b->dim, b->precision, na, b->n};
    char *o = static_cast<char *>(buf);
    std::memcpy(o, &h, sizeof(h));
    o += sizeof(h);
    for (int k = 0; k < na; ++k) {
        MTS_CUDA(cudaMemcpyAsync(o, ptr[k], len[k], cudaMemcpyDeviceToHost, b->ctx->stream));
        o += len[k];
    }
    MTS_CUDA(cudaStreamSynchronize(b->ctx->stream));
    *bytes = need;
    return MTS_OK;
}

mts_status mts_load_state(mts_body *b, const void *buf, size_t bytes) {
    if (!b || !buf) {
        set_error("mts_load_state: NULL argument");
        return MTS_ERR_INVALID_ARG;
    }
    void *ptr[8];
    size_t len[8];
    const int na = state_arrays(b, ptr, len);
    size_t need = sizeof(StateHeader);
    for (int k = 0; k < na; ++k) need += len[k];
    StateHeader h{};
    if (bytes >= sizeof(h)) std::memcpy(&h, buf, sizeof(h));
    if (bytes != need || h.magic != kStateMagic || h.dim != b->dim || h.precision != b->precision ||
        h.n != b->n || h.narrays != na) {
        set_error("mts_load_state: buffer does not hold the state of a body like this one "
                  "(%zu bytes, %zu expected)", bytes, need);
        return MTS_ERR_INVALID_ARG;
    }
    MTS_CUDA(cudaSetDevice(b->ctx->device));
    const char *in = static_cast<const char *>(buf) + sizeof(h);
    for (int k = 0; k < na; ++k) {
        MTS_CUDA(cudaMemcpyAsync(ptr[k], in, len[k], cudaMemcpyHostToDevice, b->ctx->stream));
        in += len[k];
    }
    MTS_CUDA(cudaStreamSynchronize(b->ctx->stream));
    return MTS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- reverse mode
namespace {
void free_adjoint(mts_body *b) {
    void **ptrs[] = {(void **)&b->tape_u, (void **)&b->tape_cp, (void **)&b->tape_dt,
                     (void **)&b->tape_c, (void **)&b->adj_u, (void **)&b->adj_v,
                     (void **)&b->adj_cp, (void **)&b->adj_c, (void **)&b->adj_a,
                     (void **)&b->adj_G, (void **)&b->adj_theta, (void **)&b->adj_part,
                     (void **)&b->adj_ctrl};
    for (void **pp : ptrs) {
        dfree(b->ctx, *pp);
        *pp = nullptr;
    }
    b->adj_cap = 0;
}

mts_status zero_adjoint(mts_body *b) {
    cudaStream_t st = b->ctx->stream;
    const size_t n = (size_t)b->n, pad = b->dim == 2 ? 2 : 4;
    MTS_CUDA(cudaMemsetAsync(b->adj_u, 0, n * pad * 8, st));
    MTS_CUDA(cudaMemsetAsync(b->adj_v, 0, n * pad * 8, st));
    MTS_CUDA(cudaMemsetAsync(b->adj_cp, 0, n * 8 * 8, st));
    MTS_CUDA(cudaMemsetAsync(b->adj_c, 0, n * 8, st));
    MTS_CUDA(cudaMemsetAsync(b->adj_theta, 0, 8 * 8, st));
    MTS_CUDA(cudaMemsetAsync(b->adj_ctrl, 0, sizeof(Control), st));
    for (int k = 0; k < 3; ++k) b->adj_force_seed[k] = 0.0;
    return MTS_OK;
}

mts_status adjoint_ready(mts_body *b, const char *who) {
    if (!b) {
        set_error("%s: NULL body", who);
        return MTS_ERR_INVALID_ARG;
    }
    if ((b->shadow ? b->shadow : b)->adj_cap <= 0) {
        set_error("%s: reverse mode not enabled (mts_adjoint_enable)", who);
        return MTS_ERR_STATE;
    }
    MTS_CUDA(cudaSetDevice(b->ctx->device));
    return MTS_OK;
}

// The body that holds the tape and the adjoint state: the body itself (FP64),
// or the FP64 twin of a mixed-precision body.
mts_body *adj_of(mts_body *b) { return b->shadow ? b->shadow : b; }

// FP64 twin of a mixed-precision body for its reverse mode: created from the
// body's own FP64 positions with its damping-order layout, so its Morton
// order, neighbour lists and damping order are those of the body (checked).
mts_status make_shadow(mts_body *b) {
    if (b->shadow) return MTS_OK;
    std::vector<double> X((size_t)b->n * b->dim);
    MTS_TRY(mts_read_field(b, MTS_F_X, X.data(), (int64_t)X.size()));
    mts_body_desc d{};
    d.dim = b->dim;
    d.precision = MTS_FP64;
    d.n = b->n;
    d.X = X.data();
    d.dx = b->dx;
    d.h_over_dx = b->h / b->dx;
    d.damp_layout = b->damp_layout;
    d.tile = 0;
    mts_body *s = nullptr;
    MTS_TRY(mts_body_create(b->ctx, &d, &s));
    std::vector<long long> pa((size_t)b->n), pb((size_t)b->n);
    cudaStream_t st = b->ctx->stream;
    mts_status e = MTS_OK;
    if (cudaMemcpyAsync(pa.data(), b->perm, b->n * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(pb.data(), s->perm, b->n * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        e = cuda_fail(cudaGetLastError(), "make_shadow");
    } else if (pa != pb || s->npairs != b->npairs || s->nnz != b->nnz) {
        set_error("mts_adjoint_enable: the FP64 twin of the body has another set-up order");
        e = MTS_ERR_STATE;
    }
    if (e != MTS_OK) {
        mts_body_destroy(s);
        return e;
    }
    b->shadow = s;
    return MTS_OK;
}

// Bring the twin's parameters, boundary conditions and concentration to the
// body's (both hold the particles in the same order).
mts_status shadow_sync(mts_body *b) {
    mts_body *s = b->shadow;
    if (!s) return MTS_OK;
    s->has_material = b->has_material;
    s->model = b->model;
    s->rho0 = b->rho0; s->E = b->E; s->nu = b->nu; s->K = b->K; s->mu = b->mu;
    s->lambda = b->lambda; s->s0 = b->s0; s->sinf = b->sinf; s->delta = b->delta;
    s->Hlin = b->Hlin; s->eta = b->eta;
    s->has_diff = b->has_diff; s->D = b->D; s->beta = b->beta; s->c0 = b->c0;
    s->diff_mode = b->diff_mode;
    s->tip_count = b->tip_count;
    cudaStream_t st = b->ctx->stream;
    const size_t pad = b->dim == 2 ? 2 : 4;
    if (s->h_flags != b->h_flags) {
        s->h_flags = b->h_flags;
        MTS_CUDA(cudaMemcpyAsync(s->flags, b->flags, b->n, cudaMemcpyDeviceToDevice, st));
        MTS_TRY(update_pair_fixbits(s));
    }
    MTS_CUDA(cudaMemcpyAsync(s->u_unit, b->u_unit, b->n * pad * 8, cudaMemcpyDeviceToDevice, st));
    MTS_TRY(copy_c_to_double(b, (double *)s->c));
    ++s->graph_gen;
    return MTS_OK;
}
}  // namespace

extern "C" {

mts_status mts_adjoint_enable(mts_body *b, int64_t max_substeps) {
    if (!b || max_substeps < 1) {
        set_error("mts_adjoint_enable: NULL body or max_substeps < 1");
        return MTS_ERR_INVALID_ARG;
    }
    if (b->aniso) {
        set_error("mts_adjoint_enable: the reverse mode has no anisotropic-kernel form");
        return MTS_ERR_STATE;
    }
    MTS_CUDA(cudaSetDevice(b->ctx->device));
    MTS_CUDA(cudaStreamSynchronize(b->ctx->stream));
    if (b->precision != MTS_FP64) {
        // mixed precision: the tape and the adjoint state live on an FP64 twin
        MTS_TRY(make_shadow(b));
        MTS_TRY(shadow_sync(b));
        b = b->shadow;
        MTS_TRY(prepare_kernels(b));   // its transposed damping sweep runs the FP64 kernel
    }
    free_adjoint(b);
    const size_t n = (size_t)b->n, pad = b->dim == 2 ? 2 : 4, ms = b->dim == 2 ? 4 : 12;
    const size_t K = (size_t)max_substeps;
    mts_status s = MTS_OK;
    auto A = [&](void **p, size_t bytes) {
        if (s == MTS_OK) s = dalloc_into(b->ctx, p, bytes + 16);
    };
    A((void **)&b->tape_u, K * n * pad * 8);
    A((void **)&b->tape_cp, K * n * 8 * 8);
    A((void **)&b->tape_dt, K * 8);
    A((void **)&b->tape_c, n * 8);
    A((void **)&b->adj_u, n * pad * 8);
    A((void **)&b->adj_v, n * pad * 8);
    A((void **)&b->adj_cp, n * 8 * 8);
    A((void **)&b->adj_c, n * 8);
    A((void **)&b->adj_a, n * pad * 8);
    A((void **)&b->adj_G, n * ms * 8);
    A((void **)&b->adj_theta, 8 * 8);
    A((void **)&b->adj_part, (size_t)b->ntiles * 8 * 8);
    A((void **)&b->adj_ctrl, sizeof(Control));
    if (s != MTS_OK) {
        free_adjoint(b);
        return s;
    }
    b->adj_cap = max_substeps;
    MTS_TRY(zero_adjoint(b));
    MTS_TRY(adjoint_prepare(b));
    MTS_CUDA(cudaStreamSynchronize(b->ctx->stream));
    return MTS_OK;
}

mts_status mts_adjoint_reset(mts_body *b) {
    MTS_TRY(adjoint_ready(b, "mts_adjoint_reset"));
    MTS_TRY(zero_adjoint(adj_of(b)));
    MTS_CUDA(cudaStreamSynchronize(b->ctx->stream));
    return MTS_OK;
}

mts_status mts_adjoint_seed(mts_body *b, const double *u_bar, const double *tip_bar,
                            const double *force_bar) {
    MTS_TRY(adjoint_ready(b, "mts_adjoint_seed"));
    MTS_TRY(shadow_sync(b));
    b = adj_of(b);
    if (u_bar)
        MTS_CUDA(cudaMemcpyAsync(b->scratch, u_bar, (size_t)b->n * b->dim * 8,
                                 cudaMemcpyHostToDevice, b->ctx->stream));
    MTS_TRY(adjoint_seed(b, u_bar ? b->scratch : nullptr, tip_bar));
    if (force_bar)
        for (int k = 0; k < b->dim; ++k) b->adj_force_seed[k] += force_bar[k];
    MTS_CUDA(cudaStreamSynchronize(b->ctx->stream));
    return MTS_OK;
}

mts_status mts_adjoint_slow_step(mts_body *b, const mts_step_params *p, int64_t substeps,
                                 double *theta_bar) {
    MTS_TRY(adjoint_ready(b, "mts_adjoint_slow_step"));
    mts_body *a = adj_of(b);     // tape and adjoint state (b itself, or its FP64 twin)
    if (!p || !theta_bar || substeps < 1 || substeps > a->adj_cap) {
        set_error("mts_adjoint_slow_step: NULL argument or substeps %lld outside [1, %lld]",
                  (long long)substeps, (long long)a->adj_cap);
        return MTS_ERR_INVALID_ARG;
    }
    if (p->dt_slow > 0 && b->diff_mode != 0) {
        set_error("mts_adjoint_slow_step: the reverse mode covers the one-pass diffusion step only");
        return MTS_ERR_STATE;
    }
    cudaStream_t st = b->ctx->stream;
    // recompute the slow step from its start, taping every substep's input
    mts_step_params q = *p;
    q.max_substeps = substeps;
    q.ke_tol = -1.0;
    long long launches = 0;
    MTS_TRY(shadow_sync(b));
    if (a != b) MTS_TRY(copy_c_to_double(b, a->tape_c));   // c before the diffusion step
    MTS_TRY(slow_step_begin(b, &q, &launches, a == b ? b->tape_c : nullptr));
    MTS_TRY(prepare_kernels(b));
    b->use_cond = 0;
    for (long long k = 0; k < substeps; ++k) {
        MTS_TRY(adjoint_tape(b, a, k));
        MTS_TRY(launch_stress(b));
        MTS_TRY(launch_force(b));
        MTS_TRY(launch_damping(b));
        MTS_TRY(launch_drift(b));
    }
    MTS_CUDA(cudaMemcpyAsync(b->h_ctrl, b->ctrl, sizeof(Control), cudaMemcpyDeviceToHost, st));
    MTS_CUDA(cudaStreamSynchronize(st));
    if (b->h_ctrl->nsub != substeps || b->h_ctrl->status != MTS_OK) {
        set_error("mts_adjoint_slow_step: the recomputed step ran %lld substeps (status %d), "
                  "expected %lld", (long long)b->h_ctrl->nsub, b->h_ctrl->status,
                  (long long)substeps);
        return MTS_ERR_STATE;
    }
    // reverse (on the twin: the concentration of the substeps, after the
    // diffusion step, is the one the stress law's transpose reads)
    if (a != b) MTS_TRY(copy_c_to_double(b, (double *)a->c));
    for (long long k = substeps - 1; k >= 0; --k) MTS_TRY(adjoint_substep(a, k, k == substeps - 1));
    if (q.dt_slow > 0) MTS_TRY(adjoint_diffusion(a, q.dt_slow));
    MTS_TRY(adjoint_load(a));
    double th[8];
    MTS_CUDA(cudaMemcpyAsync(th, a->adj_theta, sizeof(th), cudaMemcpyDeviceToHost, st));
    MTS_CUDA(cudaMemsetAsync(a->adj_theta, 0, sizeof(th), st));
    MTS_CUDA(cudaStreamSynchronize(st));
    for (int k = 0; k < 7; ++k) theta_bar[k] += th[k];
    for (int k = 0; k < 3; ++k) a->adj_force_seed[k] = 0.0;
    return MTS_OK;
}

mts_status mts_read_adjoint(mts_body *b, int32_t field, double *out, int64_t len) {
    MTS_TRY(adjoint_ready(b, "mts_read_adjoint"));
    if (!out || !(field == MTS_F_U || field == MTS_F_V || field == MTS_F_C ||
                  field == MTS_F_ALPHA || field == MTS_F_CPINV)) {
        set_error("mts_read_adjoint: invalid arguments (fields U, V, C, ALPHA, CPINV)");
        return MTS_ERR_INVALID_ARG;
    }
    const int w = field_width(b, field);
    if (len != b->n * w) {
        set_error("mts_read_adjoint: len %lld, expected %lld", (long long)len, (long long)(b->n * w));
        return MTS_ERR_INVALID_ARG;
    }
    MTS_TRY(adjoint_out(adj_of(b), field, adj_of(b)->scratch));
    MTS_CUDA(cudaMemcpyAsync(out, adj_of(b)->scratch, len * 8, cudaMemcpyDeviceToHost,
                             b->ctx->stream));
    MTS_CUDA(cudaStreamSynchronize(b->ctx->stream));
    return MTS_OK;
}

}  // extern "C"

extern "C" mts_status mts_adjoint_equilibrium(mts_body *b, int64_t max_iters, double tol,
                                             double *theta_bar, int64_t *iters) {
    MTS_TRY(adjoint_ready(b, "mts_adjoint_equilibrium"));
    if (!theta_bar || max_iters < 1 || !(tol > 0.0) || !std::isfinite(tol)) {
        set_error("mts_adjoint_equilibrium: NULL theta_bar, max_iters < 1 or tol not > 0");
        return MTS_ERR_INVALID_ARG;
    }
    if (!b->has_material) {
        set_error("mts_adjoint_equilibrium: no material set");
        return MTS_ERR_STATE;
    }
    cudaStream_t st = b->ctx->stream;
    // the held state, with the size the next substep would take, is the one
    // taped entry every transposed substep linearises about (a mixed-precision
    // body's state, taped into its FP64 twin, which runs the iteration)
    MTS_TRY(shadow_sync(b));
    mts_body *const src = b;
    b = adj_of(b);
    MTS_TRY(adjoint_tape(src, b, 0));
    // norm scratch: one double per block of the drift grid (part_drift holds two)
    double *part = b->part_drift, *nrm = b->scratch;
    double h[2];
    MTS_TRY(adjoint_norm2(b, part, nrm));
    MTS_CUDA(cudaMemcpyAsync(h, nrm, 8, cudaMemcpyDeviceToHost, st));
    MTS_CUDA(cudaStreamSynchronize(st));
    double n0 = h[0];
    int64_t it = 0;
    const bool force_seed = b->adj_force_seed[0] != 0.0 || b->adj_force_seed[1] != 0.0 ||
                            b->adj_force_seed[2] != 0.0;
    bool done = n0 == 0.0 && !force_seed;
    while (!done && it < max_iters) {
        MTS_TRY(adjoint_substep(b, 0, it == 0));
        ++it;
        if (it == 1 && force_seed) {
            // an end-force seed enters through the first transposed kick: the
            // reference norm includes what it put into (u-bar, v-bar)
            MTS_TRY(adjoint_norm2(b, part, nrm));
            MTS_CUDA(cudaMemcpyAsync(h, nrm, 8, cudaMemcpyDeviceToHost, st));
            MTS_CUDA(cudaStreamSynchronize(st));
            n0 = std::max(n0, h[0]);
        }
        if (it % 8 == 0 || it == max_iters) {
            MTS_TRY(adjoint_norm2(b, part, nrm));
            MTS_CUDA(cudaMemcpyAsync(h, nrm, 8, cudaMemcpyDeviceToHost, st));
            MTS_CUDA(cudaStreamSynchronize(st));
            if (!std::isfinite(h[0])) {
                set_error("mts_adjoint_equilibrium: non-finite adjoint after %lld iterations",
                          (long long)it);
                return MTS_ERR_NONFINITE;
            }
            done = h[0] <= tol * tol * n0;
        }
    }
    double th[8];
    MTS_CUDA(cudaMemcpyAsync(th, b->adj_theta, sizeof(th), cudaMemcpyDeviceToHost, st));
    MTS_CUDA(cudaMemsetAsync(b->adj_theta, 0, sizeof(th), st));
    MTS_CUDA(cudaStreamSynchronize(st));
    for (int k = 0; k < 7; ++k) theta_bar[k] += th[k];
    for (int k = 0; k < 3; ++k) b->adj_force_seed[k] = 0.0;
    if (iters) *iters = it;
    if (!done) {
        set_error("mts_adjoint_equilibrium: adjoint not below tol after %lld iterations",
                  (long long)it);
        return MTS_ERR_TIMEOUT;
    }
    return MTS_OK;
}
