// Auxiliary kernels, non-equilibrium storage float.
#define POND_S float
#define POND_PREC f32
#include "pond_aux_inst.cuh"
