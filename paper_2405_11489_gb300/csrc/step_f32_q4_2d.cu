// Step kernel: storage float, arithmetic float, D1Q4-based lattice, 2d grids.
#define POND_S float
#define POND_R float
#define POND_Q1 4
#define POND_ONED false
#define POND_TAG f32_q4_2d
#include "pond_step_inst.cuh"
