// Instantiates the auxiliary kernels for storage POND_S (suffix POND_PREC).
#include "pond_aux.cuh"
#include "pond_launch.h"

#define POND_CAT3(a, b) a##_##b
#define POND_CAT(a, b) POND_CAT3(a, b)

namespace pond {

static inline unsigned blocks_for(long long n) { return (unsigned)((n + 255) / 256); }

cudaError_t POND_CAT(init, POND_PREC)(const AuxParams& p, const double* rho, const double* ux,
                                      const double* uy, const double* T, cudaStream_t s)
{
    init_kernel<POND_S><<<blocks_for(p.N), 256, 0, s>>>(p, rho, ux, uy, T);
    return cudaGetLastError();
}

cudaError_t POND_CAT(set_pops, POND_PREC)(const AuxParams& p, const double* f, const double* g,
                                          const double* ux, const double* uy, const double* T,
                                          cudaStream_t s)
{
    set_pops_kernel<POND_S><<<blocks_for(p.N), 256, 0, s>>>(p, f, g, ux, uy, T);
    return cudaGetLastError();
}

cudaError_t POND_CAT(moments, POND_PREC)(const AuxParams& p, double* rho, double* ux, double* uy,
                                         double* T, cudaStream_t s)
{
    moments_kernel<POND_S><<<blocks_for(p.N), 256, 0, s>>>(p, rho, ux, uy, T);
    return cudaGetLastError();
}

cudaError_t POND_CAT(get_pops, POND_PREC)(const AuxParams& p, double* f, double* g, double* ux,
                                          double* uy, double* T, cudaStream_t s)
{
    get_pops_kernel<POND_S><<<blocks_for(p.N), 256, 0, s>>>(p, f, g, ux, uy, T);
    return cudaGetLastError();
}

cudaError_t POND_CAT(internal_source, POND_PREC)(const AuxParams& p, cudaStream_t s)
{
    internal_source_kernel<POND_S><<<blocks_for(p.N), 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t POND_CAT(internal_source_batch, POND_PREC)(const CaseDesc* cases, const int* block_start,
                                                       int ncase, int flip, int blocks, cudaStream_t s)
{
    internal_source_batch_kernel<POND_S><<<blocks, 256, 0, s>>>(cases, block_start, ncase, flip);
    return cudaGetLastError();
}

cudaError_t POND_CAT(init_batch, POND_PREC)(const CaseDesc* cases, const int* block_start, int c0, int c1,
                                            int block0, int blocks, int flip, const MemberFields& fld,
                                            cudaStream_t s)
{
    init_batch_kernel<POND_S><<<blocks, 256, 0, s>>>(cases, block_start, c0, c1, block0, flip, fld);
    return cudaGetLastError();
}

cudaError_t POND_CAT(moments_batch, POND_PREC)(const CaseDesc* cases, const int* block_start, int c0, int c1,
                                               int block0, int blocks, int flip, const MemberFields& fld,
                                               cudaStream_t s)
{
    moments_batch_kernel<POND_S><<<blocks, 256, 0, s>>>(cases, block_start, c0, c1, block0, flip, fld);
    return cudaGetLastError();
}

}  // namespace pond
