// Launch entry points of the kernels.  Step kernels are instantiated per storage precision,
// lattice and grid dimensionality, auxiliary kernels per precision, each set in its own
// translation unit so that the build runs in parallel.
#pragma once

#include "pond_device.cuh"

namespace pond {

struct StepParams;
struct AuxParams;
struct CaseDesc;

// Threads per CTA of the step kernel (tile_x * tile_y).  The kernel holds about 255
// registers a thread, so an SM keeps 256 of its threads: one CTA of 256 on 2-D grids, two of
// 128 on quasi-1-D grids, where one CTA's staging then overlaps the other's stencil work and
// the last tile of a short tube leaves fewer lanes idle (256 uneven tubes: 2250 -> 2560 MLUPS;
// on 2-D grids 128-node tiles stage 39 % more halo and ran 1-2 % slower).
constexpr int kStepThreads2D = 256;
constexpr int kStepThreads1D = 128;
constexpr int step_threads(bool one_d) { return one_d ? kStepThreads1D : kStepThreads2D; }
// CTAs of the step kernel resident per SM, the launch bound it is compiled for: one on 2-D
// grids and two on quasi-1-D grids (registers: about 255 a thread), three on quasi-1-D D2Q16
// grids with FP32 arithmetic, whose kernel is held to 168 registers (90 B of spills; the 256
// tubes 2410 -> 2820 MLUPS; four per SM spilled 400 B and ran at 2360).
constexpr int step_blocks_per_sm(bool one_d, bool d2q25, bool fp64)
{
    return !one_d ? 1 : (!d2q25 && !fp64) ? 3 : 2;
}

struct Launch {
    dim3 grid, block;
    size_t smem;
    cudaStream_t stream;
};

// pred: the internal split's predictor pass instead of a step (see step_kernel).
typedef cudaError_t (*StepFn)(const StepParams& p, int order, bool pred, const Launch& l);
// Raises the step kernel's dynamic shared-memory limit to what the device allows per block
// (optin) less the kernel's static shared memory, which it reports in *static_bytes.
typedef cudaError_t (*SmemFn)(int order, size_t optin, size_t* static_bytes);

#define POND_DECLARE_STEP(TAG)                                               \
    cudaError_t step_##TAG(const StepParams& p, int order, bool pred, const Launch& l); \
    cudaError_t smem_##TAG(int order, size_t optin, size_t* static_bytes);

#define POND_DECLARE_STEP_ALL(PREC) \
    POND_DECLARE_STEP(PREC##_q4_2d) \
    POND_DECLARE_STEP(PREC##_q4_1d) \
    POND_DECLARE_STEP(PREC##_q5_2d) \
    POND_DECLARE_STEP(PREC##_q5_1d)

POND_DECLARE_STEP_ALL(f64)
POND_DECLARE_STEP_ALL(f32)
POND_DECLARE_STEP_ALL(f16)
POND_DECLARE_STEP_ALL(bf16)

#define POND_DECLARE_AUX(PREC)                                                                   \
    cudaError_t init_##PREC(const AuxParams& p, const double* rho, const double* ux,             \
                            const double* uy, const double* T, cudaStream_t s);                  \
    cudaError_t set_pops_##PREC(const AuxParams& p, const double* f, const double* g,            \
                                const double* ux, const double* uy, const double* T,             \
                                cudaStream_t s);                                                 \
    cudaError_t moments_##PREC(const AuxParams& p, double* rho, double* ux, double* uy,          \
                               double* T, cudaStream_t s);                                       \
    cudaError_t get_pops_##PREC(const AuxParams& p, double* f, double* g, double* ux,            \
                                double* uy, double* T, cudaStream_t s);                          \
    cudaError_t internal_source_##PREC(const AuxParams& p, cudaStream_t s);                        \
    cudaError_t internal_source_batch_##PREC(const CaseDesc* cases, const int* block_start,        \
                                             int ncase, int flip, int blocks, cudaStream_t s);     \
    cudaError_t init_batch_##PREC(const CaseDesc* cases, const int* block_start, int c0, int c1,   \
                                  int block0, int blocks, int flip, const MemberFields& fld,       \
                                  cudaStream_t s);                                                 \
    cudaError_t moments_batch_##PREC(const CaseDesc* cases, const int* block_start, int c0, int c1, \
                                     int block0, int blocks, int flip, const MemberFields& fld,    \
                                     cudaStream_t s);

POND_DECLARE_AUX(f64)
POND_DECLARE_AUX(f32)
POND_DECLARE_AUX(f16)
POND_DECLARE_AUX(bf16)

}  // namespace pond
