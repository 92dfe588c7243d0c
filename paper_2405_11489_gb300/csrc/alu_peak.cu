// FMA throughput of the device's FP32 and FP64 CUDA-core pipes: the measured companion of the
// unit-count peaks against which the step kernel's ALU roofline is reported.  The paper has
// no counterpart; this is measurement plumbing.
//
// Every thread runs kChains independent FMA chains (a <- a * b + c) for iters trips of
// kUnroll steps each, so the pipe, not the dependency latency, limits the rate; b and c are
// kernel arguments (not constants the compiler could fold) and the chains' sum is compared
// with a value it never takes, so no chain is dead code.  Grid: kBlocksPerSm blocks of
// kThreads threads per SM, far more warps than the FMA latency needs.
#include <cuda_runtime.h>

#include "pond.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

__device__ double g_alu_sink;   // written only if the chains' sum hits an impossible value

template <class T>
__global__ void __launch_bounds__(kThreads) fma_chains(int iters, T b, T c)
{
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = T(threadIdx.x + k) * T(1e-6);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == T(-1234.5)) g_alu_sink = (double)s;
}

}  // namespace

extern "C" int pond_alu_peak(int32_t fp64, int32_t iters, void* cuda_stream, double* flop, float* ms)
{
    if (iters <= 0 || !flop || !ms || (fp64 != 0 && fp64 != 1)) return POND_EINVAL;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return POND_ECUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return POND_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return POND_ECUDA;
    }
    const dim3 grid(sms * kBlocksPerSm), block(kThreads);
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
        if (fp64) fma_chains<double><<<grid, block, 0, s>>>(iters, 0.9999999, 1e-7);
        else fma_chains<float><<<grid, block, 0, s>>>(iters, 0.9999f, 1e-4f);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return POND_ECUDA;
    *flop = 2.0 * kChains * kUnroll * (double)iters * (double)grid.x * kThreads;
    return POND_OK;
}
