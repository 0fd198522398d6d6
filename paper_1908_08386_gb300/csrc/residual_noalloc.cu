// lbmfvm_residual_noalloc: the steady-state residual reduction on caller
// arrays, for callers that cannot allocate device memory.
//
// Some callers of this library cannot call cudaMalloc: code whose device
// memory is entirely owned by another allocator (a framework's caching
// allocator, or a fixed arena handed out at start-up, where a stray
// cudaMalloc would fail or fragment the pool) and latency-critical loops that
// cannot afford the implicit device-wide synchronisation of
// cudaMalloc/cudaFree.  This entry point allocates nothing: the reduction's
// scratch (per-block partial sums) lives in a file-scope __device__ array of
// fixed size that every GPU loading the library holds until the process
// exits.  The call waits for its stream and copies the two totals to the
// host before it returns.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "lbmfvm.h"

namespace lbmfvm_internal {
int fail_thread_msg(int code, const char *msg);
}

namespace {

constexpr int kThreads = 256;
constexpr int kBlocks = 512;               // pass-1 blocks; each leaves two partial sums
constexpr long long kMaxNodes = 1LL << 30; // largest n accepted
constexpr int kMaxDevices = 64;

// Scratch: partial sums (2 per block), then the two totals.  Every block
// writes its own slots on every call and the finishing pass reads only the
// slots written by this call, so nothing has to be cleared between calls.
__device__ __align__(256) double g_residual_scratch[2 * kBlocks + 2];

std::mutex g_mu;
double *g_scratch_addr[kMaxDevices];

// Pass 1: FP64 sums of |u - u_prev|^2 and |u|^2 over the selected nodes.
__global__ void __launch_bounds__(kThreads)
    noalloc_partials(const double *u, const double *v, const double *up, const double *vp, const uint8_t *sel,
                     long long n, double *scratch) {
    __shared__ double red[2][kThreads / 32];
    double num = 0.0, den = 0.0;
    for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads) {
        if (sel && !sel[i]) continue;
        const double du = u[i] - up[i], dv = v[i] - vp[i];
        num += du * du + dv * dv;
        den += u[i] * u[i] + v[i] * v[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_down_sync(0xffffffffu, num, o);
        den += __shfl_down_sync(0xffffffffu, den, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = num;
        red[1][threadIdx.x >> 5] = den;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < kThreads / 32; w++) {
            a += red[0][w];
            b += red[1][w];
        }
        scratch[2 * blockIdx.x] = a;
        scratch[2 * blockIdx.x + 1] = b;
    }
}

// Pass 2: one warp adds the partial sums of the nblocks blocks in a fixed order.
__global__ void noalloc_finish(double *scratch, int nblocks) {
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += 32) {
        a += scratch[2 * i];
        b += scratch[2 * i + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (threadIdx.x == 0) {
        scratch[2 * kBlocks] = a;
        scratch[2 * kBlocks + 1] = b;
    }
}

// Device address of the scratch array on the current device, looked up once
// per device.  The name g_residual_scratch is only a host-side stand-in.
int scratch_for_current_device(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        char msg[200];
        snprintf(msg, sizeof(msg), "cudaGetDevice failed: %s", cudaGetErrorString(e));
        return lbmfvm_internal::fail_thread_msg(LBMFVM_ERR_CUDA, msg);
    }
    if (dev < 0 || dev >= kMaxDevices)
        return lbmfvm_internal::fail_thread_msg(LBMFVM_ERR_ARG, "device ordinal beyond the supported 64 devices");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_residual_scratch);
        if (e != cudaSuccess || !p) {
            char msg[200];
            snprintf(msg, sizeof(msg), "cudaGetSymbolAddress of the residual scratch failed: %s",
                     cudaGetErrorString(e));
            return lbmfvm_internal::fail_thread_msg(LBMFVM_ERR_CUDA, msg);
        }
        g_scratch_addr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_addr[dev];
    return LBMFVM_OK;
}

}  // namespace

extern "C" int lbmfvm_residual_noalloc(const double *u, const double *v, const double *u_prev, const double *v_prev,
                                       const uint8_t *select, int64_t n, void *stream, double *r) {
    using lbmfvm_internal::fail_thread_msg;
    if (!r) return fail_thread_msg(LBMFVM_ERR_ARG, "r is NULL");
    *r = NAN;
    if (!u || !v || !u_prev || !v_prev) return fail_thread_msg(LBMFVM_ERR_ARG, "an input array is NULL");
    if (n < 1 || n > kMaxNodes) {
        char msg[160];
        snprintf(msg, sizeof(msg), "n = %lld is outside [1, %lld] (the size the static scratch supports)",
                 (long long)n, kMaxNodes);
        return fail_thread_msg(LBMFVM_ERR_ARG, msg);
    }
    double *scratch = nullptr;
    if (int rc = scratch_for_current_device(&scratch)) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    long long want = (n + kThreads - 1) / kThreads;
    const int blocks = want < kBlocks ? (int)want : kBlocks;
    noalloc_partials<<<blocks, kThreads, 0, s>>>(u, v, u_prev, v_prev, select, n, scratch);
    noalloc_finish<<<1, 32, 0, s>>>(scratch, blocks);
    double sums[2] = {0.0, 0.0};
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(sums, scratch + 2 * kBlocks, sizeof(sums), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        char msg[200];
        snprintf(msg, sizeof(msg), "residual without allocation failed: %s", cudaGetErrorString(e));
        return fail_thread_msg(LBMFVM_ERR_CUDA, msg);
    }
    if (!std::isfinite(sums[0]) || !std::isfinite(sums[1]))
        return fail_thread_msg(LBMFVM_ERR_DIVERGED, "non-finite velocity in the residual");
    *r = sums[1] > 0.0 ? std::sqrt(sums[0]) / std::sqrt(sums[1]) : (sums[0] == 0.0 ? 0.0 : INFINITY);
    return LBMFVM_OK;
}
