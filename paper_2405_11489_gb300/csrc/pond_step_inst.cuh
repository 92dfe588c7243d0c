// Instantiates the step kernel for storage POND_S, arithmetic POND_R, lattice POND_Q1 and
// dimensionality POND_ONED (both interpolation orders); included by one translation unit each.
#include "pond_launch.h"
#include "pond_step.cuh"

#define POND_CAT3(a, b) a##_##b
#define POND_CAT(a, b) POND_CAT3(a, b)

namespace pond {

cudaError_t POND_CAT(step, POND_TAG)(const StepParams& p, int order, const Launch& l)
{
    if (order == 3)
        step_kernel<POND_S, POND_R, POND_Q1, 4, POND_ONED, step_threads(POND_ONED)><<<l.grid, l.block, l.smem, l.stream>>>(p);
    else
        step_kernel<POND_S, POND_R, POND_Q1, 3, POND_ONED, step_threads(POND_ONED)><<<l.grid, l.block, l.smem, l.stream>>>(p);
    return cudaGetLastError();
}

template <class K>
static cudaError_t set_smem_limit(K kernel, size_t optin, size_t* static_bytes)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    *static_bytes = fa.sharedSizeBytes;
    if (fa.sharedSizeBytes >= optin) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(optin - fa.sharedSizeBytes));
}

cudaError_t POND_CAT(smem, POND_TAG)(int order, size_t optin, size_t* static_bytes)
{
    if (order == 3)
        return set_smem_limit(step_kernel<POND_S, POND_R, POND_Q1, 4, POND_ONED, step_threads(POND_ONED)>, optin,
                              static_bytes);
    return set_smem_limit(step_kernel<POND_S, POND_R, POND_Q1, 3, POND_ONED, step_threads(POND_ONED)>, optin,
                          static_bytes);
}

}  // namespace pond
