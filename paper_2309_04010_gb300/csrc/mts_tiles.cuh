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
template <class R, int P, int NY>
__device__ __forceinline__ int stage_halo(const Args<R> &A, R *sX, R *sY, const R *Y) {
    const long long t = blockIdx.x;
    const long long h0 = A.halo_off[t];
    const int nh = (int)(A.halo_off[t + 1] - h0);
    // indices first (independent loads), then asynchronous row copies
    constexpr int U = 4;
    for (int k0 = threadIdx.x; k0 < nh; k0 += U * blockDim.x) {
        int g[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = k0 + u * blockDim.x;
            g[u] = k < nh ? __ldg(A.halo_idx + h0 + k) : -1;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = k0 + u * blockDim.x;
            if (g[u] < 0) continue;
            if (sX) cp_async_reals<R, P>(sX + (size_t)k * P, A.halo_x + (size_t)(h0 + k) * P);
            if (sY) cp_async_reals<R, NY>(sY + (size_t)k * NY, Y + (size_t)g[u] * NY);
        }
    }
    cp_async_wait_all();
    __syncthreads();
    return nh;
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
