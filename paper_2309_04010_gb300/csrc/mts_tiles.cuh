// mts_tiles.cuh -- Morton-tile staging shared by the forward substep kernels
// and their adjoints: a CTA owns one tile of T consecutive particles, stages
// per-particle arrays of the tile's halo (the tile and all its neighbours) in
// shared memory, and walks each particle's neighbours through 16-bit local
// slots.
#pragma once

#include "mts_device.cuh"
#include "mts_internal.cuh"

namespace mts {

// byte offset of the second staged array: rounded up to 16 bytes so that
// 16-byte vector loads from it stay aligned for any halo size
template <class R, int P>
__host__ __device__ __forceinline__ size_t second_off(int max_halo) {
    return ((size_t)max_halo * P * sizeof(R) + 15) & ~size_t(15);
}

// --------------------------------------------------------------------- tiles
// A CTA owns one Morton tile of T = blockDim.x consecutive particles.  It
// stages the reference positions and one more per-particle array of the tile's
// halo (the tile and all its neighbours) in shared memory, then every
// neighbour access reads shared memory through a 16-bit local slot.  The
// positions come from the per-tile table halo_x (computed once in FP64
// relative to the tile's first particle), so in FP32 the separations keep
// their relative precision however far the tile is from the body's corner.
// Halo staging in two parts, so that the set-up data can move before the
// previous kernel of the chain has finished: stage_halo_pre loads the first
// kHaloPre x blockDim halo indices into registers and starts the copies of the
// X rows (set-up data) into shared memory; stage_halo_post, after the chain
// wait, starts the copies of the Y rows (state written by the previous
// kernel), stages any halo entries beyond the first part, and waits for every
// copy.  stage_halo runs both back to back.
constexpr int kHaloPre = 4;

template <class R>
struct HaloPre {
    long long h0;
    int nh;
    int g[kHaloPre];
};

template <class R, int P>
__device__ __forceinline__ HaloPre<R> stage_halo_pre(const Args<R> &A, R *sX) {
    HaloPre<R> h;
    const long long t = blockIdx.x;
    h.h0 = A.halo_off[t];
    h.nh = (int)(A.halo_off[t + 1] - h.h0);
#pragma unroll
    for (int u = 0; u < kHaloPre; ++u) {
        const int k = threadIdx.x + u * blockDim.x;
        h.g[u] = k < h.nh ? __ldg(A.halo_idx + h.h0 + k) : -1;
    }
#pragma unroll
    for (int u = 0; u < kHaloPre; ++u) {
        const int k = threadIdx.x + u * blockDim.x;
        if (h.g[u] >= 0 && sX) cp_async_reals<R, P>(sX + (size_t)k * P, A.halo_x + (size_t)(h.h0 + k) * P);
    }
    return h;
}

template <class R, int P, int NY>
__device__ __forceinline__ int stage_halo_post(const Args<R> &A, const HaloPre<R> &h, R *sX, R *sY,
                                               const R *Y) {
#pragma unroll
    for (int u = 0; u < kHaloPre; ++u) {
        const int k = threadIdx.x + u * blockDim.x;
        if (h.g[u] >= 0 && sY) cp_async_reals<R, NY>(sY + (size_t)k * NY, Y + (size_t)h.g[u] * NY);
    }
    for (int k = threadIdx.x + kHaloPre * blockDim.x; k < h.nh; k += blockDim.x) {
        const int g = __ldg(A.halo_idx + h.h0 + k);
        if (sX) cp_async_reals<R, P>(sX + (size_t)k * P, A.halo_x + (size_t)(h.h0 + k) * P);
        if (sY) cp_async_reals<R, NY>(sY + (size_t)k * NY, Y + (size_t)g * NY);
    }
    cp_async_wait_all();
    __syncthreads();
    return h.nh;
}

template <class R, int P, int NY>
__device__ __forceinline__ int stage_halo(const Args<R> &A, R *sX, R *sY, const R *Y) {
    const HaloPre<R> h = stage_halo_pre<R, P>(A, sX);
    return stage_halo_post<R, P, NY>(A, h, sX, sY, Y);
}

// Visit the neighbour slots of one particle, reading the index stream 8
// entries ahead into registers so that each warp keeps several index lines in
// flight (the loop is unrolled by 8 so every register index is static).
template <class Body>
__device__ __forceinline__ void for_each_neighbour(const uint16_t *row, int T, int w, Body body) {
    constexpr int K = 8;
    int cur[K], nxt[K];
#pragma unroll
    for (int u = 0; u < K; ++u) cur[u] = u < w ? (int)__ldg(row + u * T) : 0;
    for (int j0 = 0; j0 < w; j0 += K) {
#pragma unroll
        for (int u = 0; u < K; ++u)
            nxt[u] = (j0 + K + u < w) ? (int)__ldg(row + (j0 + K + u) * T) : 0;
#pragma unroll
        for (int u = 0; u < K; ++u)
            if (j0 + u < w) body(cur[u]);
#pragma unroll
        for (int u = 0; u < K; ++u) cur[u] = nxt[u];
    }
}

// The same visit with the whole chunks of 8 run without a per-entry test and
// the last, partial chunk tested entry by entry.  It issues ~18 % fewer
// instructions in the F gather (the stress kernel, bound by instruction issue:
// 2.4 % faster on the 2.5 M-particle plate); the force gather, whose shared-
// memory loads dominate, ran slower with it and keeps the form above.
template <class Body>
__device__ __forceinline__ void for_each_neighbour_chunks(const uint16_t *row, int T, int w, Body body) {
    constexpr int K = 8;
    int cur[K], nxt[K];
#pragma unroll
    for (int u = 0; u < K; ++u) cur[u] = u < w ? (int)__ldg(row + u * T) : 0;
    int j0 = 0;
    for (; j0 + K <= w; j0 += K) {
#pragma unroll
        for (int u = 0; u < K; ++u)
            nxt[u] = (j0 + K + u < w) ? (int)__ldg(row + (j0 + K + u) * T) : 0;
#pragma unroll
        for (int u = 0; u < K; ++u) body(cur[u]);
#pragma unroll
        for (int u = 0; u < K; ++u) cur[u] = nxt[u];
    }
#pragma unroll
    for (int u = 0; u < K - 1; ++u)
        if (u < w - j0) body(cur[u]);
}

}  // namespace mts
