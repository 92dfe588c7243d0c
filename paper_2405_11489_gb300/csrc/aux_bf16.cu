// Auxiliary kernels, non-equilibrium storage __nv_bfloat16.
#define POND_S __nv_bfloat16
#define POND_PREC bf16
#include "pond_aux_inst.cuh"
