// Auxiliary kernels, non-equilibrium storage double.
#define POND_S double
#define POND_PREC f64
#include "pond_aux_inst.cuh"
