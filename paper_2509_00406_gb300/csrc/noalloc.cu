// noalloc.cu -- FP64 gradient 2-norm that allocates nothing.
//
// Some callers cannot call cudaMalloc at the point where they need this
// reduction: callers inside a real-time loop whose memory budget is fixed up
// front (an allocation there can stall or fail mid-loop), plug-ins running
// inside a host framework that owns the device's memory budget, and hosts
// that route every device allocation through their own pool and forbid the
// library from allocating behind it.
// adm_grad_norm_noalloc gives them a chunked sum-of-squares reduction like the
// one adm_eval_batch uses for its per-mesh gradient norms, all in FP64, with
// its scratch
// (one FP64 partial per chunk) in a fixed-size static device array of this
// file instead of a buffer owned by a handle.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "adm.h"

namespace {

constexpr int kNoAllocChunk = 8192;          // vector entries per partial sum
constexpr int kNoAllocMaxPartials = 4096;    // 32 KiB of partials -> n <= 33,554,432
constexpr int kNoAllocThreads = 256;

// Scratch shared by every call on a device, kept until the process exits.
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxPartials];

// Device address of g_noalloc_partials per device, resolved on the first call
// made with that device current (the name itself is only a host-side handle).
// The address is that of the module loaded in the device's primary context;
// a cudaDeviceReset unloads it, so the call is not for use after a reset.
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_partials_addr[kMaxDevices] = {};

template <int THREADS>
__device__ __forceinline__ double block_sum_fixed(double v)
{
    __shared__ double red[THREADS / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = threadIdx.x < THREADS / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;
}

// block b: sum of squares of v[b * chunk, min((b + 1) * chunk, n)) -> part[b]
template <typename T>
__global__ void __launch_bounds__(kNoAllocThreads) k_noalloc_sumsq(const T *v, int64_t n, double *part)
{
    const int64_t b0 = (int64_t)blockIdx.x * kNoAllocChunk;
    const int64_t b1 = b0 + kNoAllocChunk < n ? b0 + kNoAllocChunk : n;
    double s = 0.0;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += kNoAllocThreads) {
        const double x = (double)v[i];
        s += x * x;
    }
    s = block_sum_fixed<kNoAllocThreads>(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// one block: sqrt of the fixed-order sum of the first nb partials
__global__ void __launch_bounds__(1024) k_noalloc_finish(const double *part, int nb, double *out)
{
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += 1024) s += part[i];
    s = block_sum_fixed<1024>(s);
    if (threadIdx.x == 0) *out = ::sqrt(s);
}

adm_status partials_address(double **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ADM_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return ADM_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_partials_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) {
            cudaGetLastError();
            return ADM_ERR_CUDA;
        }
        g_partials_addr[dev] = (double *)p;
    }
    *out = g_partials_addr[dev];
    return ADM_OK;
}

}  // namespace

extern "C" adm_status adm_grad_norm_noalloc(const void *v_dev, int64_t n, adm_precision prec, double *norm_dev,
                                            void *stream)
{
    if (!norm_dev || n < 0 || (n > 0 && !v_dev) || (prec != ADM_FP32 && prec != ADM_FP64)) return ADM_ERR_ARG;
    const int64_t nb = (n + kNoAllocChunk - 1) / kNoAllocChunk;
    if (nb > kNoAllocMaxPartials) return ADM_ERR_ARG;  // n > 4096 * 8192 entries
    double *part = nullptr;
    adm_status s = partials_address(&part);
    if (s != ADM_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    // every partial read by the finishing kernel is written first by this
    // call, so nothing has to be cleared between calls
    if (nb > 0) {
        if (prec == ADM_FP32)
            k_noalloc_sumsq<float><<<(unsigned)nb, kNoAllocThreads, 0, st>>>((const float *)v_dev, n, part);
        else
            k_noalloc_sumsq<double><<<(unsigned)nb, kNoAllocThreads, 0, st>>>((const double *)v_dev, n, part);
    }
    k_noalloc_finish<<<1, 1024, 0, st>>>(part, (int)nb, norm_dev);
    return cudaGetLastError() == cudaSuccess ? ADM_OK : ADM_ERR_CUDA;
}
