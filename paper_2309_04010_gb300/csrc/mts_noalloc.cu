// mts_noalloc.cu -- kinetic energy and maximum speed of a caller-owned velocity
// array, computed without allocating memory.
//
// Who needs this: callers that cannot call cudaMalloc (or any allocator) at the
// point where they need the number -- for example code whose device memory is
// entirely owned by another allocator (a framework's caching allocator or a
// fixed arena that must not be bypassed or grown), code on a latency-critical
// path where the device-wide synchronisation of cudaMalloc/cudaFree is not
// acceptable, and code that must not be able to fail with out-of-memory once it
// has been set up.  They pass their own input and output buffers; the only
// working memory is the fixed array below, which belongs to this library.
//
// The reduction is the one the slow-step driver applies after every substep
// (block partials in a fixed tree order, then one block summing the partials
// in block order), so the result is deterministic for a given n.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "mts_device.cuh"
#include "mts_internal.cuh"

namespace {

using mts::cuda_fail;

constexpr int kMaxBlocks = 1024;   // partials held by the static scratch
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

// Static scratch: 1,024 (E_k, max |v|) partials = 16 KiB on every device that
// loads the library, kept until the process exits.  Every call writes all the
// partials it later reads, so nothing has to start at zero; calls that overlap
// on the GPU (e.g. on two streams) share this array and race.
static __device__ __align__(256) double g_partials[2 * kMaxBlocks];

std::mutex g_mu;
double *g_dev_ptr[kMaxDevices] = {nullptr};

template <class R, int D>
__global__ void __launch_bounds__(kThreads) k_ke_partials(const R *v, long long n, double half_m,
                                                          double *part) {
    double ke = 0.0, vmax = 0.0;
    for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < n;
         i += (long long)gridDim.x * kThreads) {
        // |v|^2 in the velocities' own precision, as the substep loop forms it
        R v2r = R(0);
#pragma unroll
        for (int k = 0; k < D; ++k) v2r += v[i * D + k] * v[i * D + k];
        const double v2 = (double)v2r;
        ke += half_m * v2;
        vmax = fmax(vmax, sqrt(v2));
    }
    __shared__ double sh[2][kThreads / 32];
    ke = mts::warp_sum(ke);
    vmax = mts::warp_max(vmax);
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = ke;
        sh[1][threadIdx.x >> 5] = vmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0, m = 0.0;
        for (int q = 0; q < kThreads / 32; ++q) {
            s += sh[0][q];
            m = fmax(m, sh[1][q]);
        }
        part[2 * blockIdx.x] = s;
        part[2 * blockIdx.x + 1] = m;
    }
}

__global__ void __launch_bounds__(kThreads) k_ke_final(const double *part, int nblk, double *out) {
    __shared__ double red[2][kThreads];
    double s = 0.0, m = 0.0;
    for (int q = threadIdx.x; q < nblk; q += kThreads) {
        s += part[2 * q];
        m = fmax(m, part[2 * q + 1]);
    }
    red[0][threadIdx.x] = s;
    red[1][threadIdx.x] = m;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            red[0][threadIdx.x] += red[0][threadIdx.x + w];
            red[1][threadIdx.x] = fmax(red[1][threadIdx.x], red[1][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = red[0][0];
        out[1] = red[1][0];
    }
}

// Device address of the static scratch on the current device.  The symbol's
// name in host code is only a stand-in; the address comes from
// cudaGetSymbolAddress, taken once per device with that device current.
mts_status scratch_address(double **out) {
    int dev = -1;
    MTS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        mts::set_error("mts_kinetic_energy_noalloc: device %d beyond the supported %d", dev,
                       kMaxDevices);
        return MTS_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_ptr[dev]) {
        void *p = nullptr;
        MTS_CUDA(cudaGetSymbolAddress(&p, g_partials));
        g_dev_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_dev_ptr[dev];
    return MTS_OK;
}

template <class R, int D>
mts_status launch(const void *v, long long n, double mass, double *out, cudaStream_t st,
                  double *part) {
    const long long want = (n + kThreads - 1) / kThreads;
    const int nblk = (int)(want < kMaxBlocks ? want : kMaxBlocks);
    k_ke_partials<R, D><<<nblk, kThreads, 0, st>>>(static_cast<const R *>(v), n, 0.5 * mass, part);
    MTS_CUDA(cudaGetLastError());
    k_ke_final<<<1, kThreads, 0, st>>>(part, nblk, out);
    MTS_CUDA(cudaGetLastError());
    return MTS_OK;
}

}  // namespace

extern "C" mts_status mts_kinetic_energy_noalloc(const void *v_dev, int32_t precision, int32_t dim,
                                                 int64_t n, double mass, double *out_dev,
                                                 void *cuda_stream) {
    if (!v_dev || !out_dev) {
        mts::set_error("mts_kinetic_energy_noalloc: NULL device pointer");
        return MTS_ERR_INVALID_ARG;
    }
    if ((precision != MTS_FP64 && precision != MTS_MIXED) || (dim != 2 && dim != 3)) {
        mts::set_error("mts_kinetic_energy_noalloc: precision %d / dim %d not supported", precision,
                       dim);
        return MTS_ERR_INVALID_ARG;
    }
    if (n < 1 || n > (int64_t)MTS_NOALLOC_MAX_N) {
        mts::set_error("mts_kinetic_energy_noalloc: n = %lld outside [1, %lld]", (long long)n,
                       (long long)MTS_NOALLOC_MAX_N);
        return MTS_ERR_INVALID_ARG;
    }
    if (!(mass >= 0.0) || !std::isfinite(mass)) {
        mts::set_error("mts_kinetic_energy_noalloc: mass must be finite and >= 0");
        return MTS_ERR_INVALID_ARG;
    }
    double *part = nullptr;
    MTS_TRY(scratch_address(&part));
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (precision == MTS_FP64)
        return dim == 2 ? launch<double, 2>(v_dev, n, mass, out_dev, st, part)
                        : launch<double, 3>(v_dev, n, mass, out_dev, st, part);
    return dim == 2 ? launch<float, 2>(v_dev, n, mass, out_dev, st, part)
                    : launch<float, 3>(v_dev, n, mass, out_dev, st, part);
}
