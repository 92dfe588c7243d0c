// Step kernel: storage __half, arithmetic float, D1Q4-based lattice, 1d grids.
#define POND_S __half
#define POND_R float
#define POND_Q1 4
#define POND_ONED true
#define POND_TAG f16_q4_1d
#include "pond_step_inst.cuh"
