// Instantiates the step kernel for storage POND_S, arithmetic POND_R, lattice POND_Q1 and
// dimensionality POND_ONED (both interpolation orders); included by one translation unit each.
#include "pond_launch.h"
#include "pond_step.cuh"

#define POND_CAT3(a, b) a##_##b
#define POND_CAT(a, b) POND_CAT3(a, b)

namespace pond {

template <int P, bool PRED>
static void launch_step(const StepParams& p, const Launch& l)
{
    step_kernel<POND_S, POND_R, POND_Q1, P, POND_ONED, step_threads(POND_ONED), PRED><<<l.grid, l.block, l.smem, l.stream>>>(p);
}

cudaError_t POND_CAT(step, POND_TAG)(const StepParams& p, int order, bool pred, const Launch& l)
{
    if (order == 3) {
        if (pred) launch_step<4, true>(p, l); else launch_step<4, false>(p, l);
    } else {
        if (pred) launch_step<3, true>(p, l); else launch_step<3, false>(p, l);
    }
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

// Sets the limit of the step kernel and of its predictor variant; *static_bytes is the larger
// static part of the two.
template <int P>
static cudaError_t set_smem_limits(size_t optin, size_t* static_bytes)
{
    size_t s0 = 0, s1 = 0;
    cudaError_t e = set_smem_limit(step_kernel<POND_S, POND_R, POND_Q1, P, POND_ONED, step_threads(POND_ONED), false>,
                                   optin, &s0);
    if (e == cudaSuccess)
        e = set_smem_limit(step_kernel<POND_S, POND_R, POND_Q1, P, POND_ONED, step_threads(POND_ONED), true>, optin,
                           &s1);
    *static_bytes = s0 > s1 ? s0 : s1;
    return e;
}

cudaError_t POND_CAT(smem, POND_TAG)(int order, size_t optin, size_t* static_bytes)
{
    return order == 3 ? set_smem_limits<4>(optin, static_bytes) : set_smem_limits<3>(optin, static_bytes);
}

}  // namespace pond
