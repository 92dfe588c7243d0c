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
        step_kernel<POND_S, POND_R, POND_Q1, 4, POND_ONED, kStepThreads><<<l.grid, l.block, l.smem, l.stream>>>(p);
    else
        step_kernel<POND_S, POND_R, POND_Q1, 3, POND_ONED, kStepThreads><<<l.grid, l.block, l.smem, l.stream>>>(p);
    return cudaGetLastError();
}

cudaError_t POND_CAT(smem, POND_TAG)(int order, size_t bytes)
{
    if (order == 3)
        return cudaFuncSetAttribute(step_kernel<POND_S, POND_R, POND_Q1, 4, POND_ONED, kStepThreads>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return cudaFuncSetAttribute(step_kernel<POND_S, POND_R, POND_Q1, 3, POND_ONED, kStepThreads>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace pond
