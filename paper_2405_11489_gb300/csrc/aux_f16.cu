// Auxiliary kernels, non-equilibrium storage __half.
#define POND_S __half
#define POND_PREC f16
#include "pond_aux_inst.cuh"
