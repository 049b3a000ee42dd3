// residual_static.cu -- || a - b ||_2 without any device allocation.
//
// The same quantity as metos3d_residual (the residual norm the spin-up and the Newton
// solver report), for callers that cannot allocate device memory at call time: processes
// whose device memory is all owned by another allocator with a fixed budget, and callers
// that hold no library context (the other reductions use scratch a context allocated).
// The per-block partial sums live in one file-scope device array of fixed size instead of
// in allocated scratch.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "metos3d.h"

namespace {

constexpr int kThreadsPerBlock = 256;
constexpr int kPerThread = 8;
constexpr long long kPerBlock = (long long)kThreadsPerBlock * kPerThread;     // 2048 entries
constexpr int kMaxPartials = M3D_RESIDUAL_STATIC_MAX_BLOCKS;                  // 65536 partials, 512 KiB
constexpr int kMaxDevices = 64;

// Shared by every call on a device; it keeps the last call's partial sums.  Every call
// overwrites the partials it reads, so nothing has to start at zero.
static __device__ __align__(256) double g_partials[kMaxPartials];

std::mutex g_mutex;
double *g_partials_addr[kMaxDevices] = {nullptr};

__global__ void __launch_bounds__(kThreadsPerBlock) k_sqdiff_partials(const double *a, const double *b,
                                                                      long long len, double *part)
{
    __shared__ double ws[kThreadsPerBlock / 32];
    long long base = blockIdx.x * kPerBlock;
    double v = 0.0;
#pragma unroll
    for (int r = 0; r < kPerThread; r++) {
        long long i = base + (long long)r * kThreadsPerBlock + threadIdx.x;
        if (i < len) {
            double d = a[i] - b[i];
            v += d * d;
        }
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kThreadsPerBlock / 32; w++) s += ws[w];
        part[blockIdx.x] = s;
    }
}

// Fixed-order sum of the partials (thread t takes partials t, t + 256, ...), then sqrt.
__global__ void __launch_bounds__(kThreadsPerBlock) k_sum_partials_sqrt(const double *part, int np, double *out)
{
    __shared__ double ws[kThreadsPerBlock];
    double v = 0.0;
    for (int i = threadIdx.x; i < np; i += kThreadsPerBlock) v += part[i];
    ws[threadIdx.x] = v;
    __syncthreads();
    for (int s = kThreadsPerBlock / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) ws[threadIdx.x] += ws[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sqrt(ws[0]);
}

// Device address of g_partials on the current device, looked up once per device.
cudaError_t partials_address(double **addr)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_partials_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess) return e;
        g_partials_addr[dev] = (double *)p;
    }
    *addr = g_partials_addr[dev];
    return cudaSuccess;
}

thread_local char g_msg[256];

}  // namespace

extern "C" {

m3d_status metos3d_residual_static(const double *a, const double *b, long long len, double *norm_dev,
                                   void *stream)
{
    if (!norm_dev || len < 0 || (len > 0 && (!a || !b))) {
        snprintf(g_msg, sizeof g_msg, "metos3d_residual_static: null pointer or negative length");
        return M3D_ERR_ARG;
    }
    long long nblocks = (len + kPerBlock - 1) / kPerBlock;
    if (nblocks > kMaxPartials) {
        snprintf(g_msg, sizeof g_msg,
                 "metos3d_residual_static: %lld entries exceed the maximum of %lld (%d blocks of %lld)",
                 len, (long long)kMaxPartials * kPerBlock, kMaxPartials, kPerBlock);
        return M3D_ERR_ARG;
    }
    double *part = nullptr;
    cudaError_t e = partials_address(&part);
    if (e != cudaSuccess) {
        snprintf(g_msg, sizeof g_msg, "metos3d_residual_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        return M3D_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (nblocks > 0)
        k_sqdiff_partials<<<(unsigned)nblocks, kThreadsPerBlock, 0, s>>>(a, b, len, part);
    k_sum_partials_sqrt<<<1, kThreadsPerBlock, 0, s>>>(part, (int)nblocks, norm_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(g_msg, sizeof g_msg, "metos3d_residual_static: launch failed: %s", cudaGetErrorString(e));
        return M3D_ERR_CUDA;
    }
    return M3D_OK;
}

const char *metos3d_residual_static_error(void) { return g_msg; }

}  // extern "C"
